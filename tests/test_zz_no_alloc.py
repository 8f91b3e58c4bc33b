"""The allocation-free colouring entry point against the regular one, through the C-ABI.

css_color_graph_noalloc is for callers that may not allocate device memory (their own
allocator owns the device, or their loop must not pay for cudaMalloc): it keeps its scratch
in a fixed array inside the library.  Two calls in a row must both reproduce css_color_graph
exactly (colours are integers, compared bit for bit), and sizes beyond the fixed capacity
must be refused.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def lib(torch):
    import paper_2605_20918_gb300 as css
    from paper_2605_20918_gb300 import build
    build.build()
    L = css.load_library()
    L.css_color_graph_noalloc.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p,
                                          C.POINTER(C.c_int32), C.c_void_p]
    L.css_color_graph_noalloc.restype = C.c_int
    return L


def _graph(n, p, seed):
    rng = np.random.default_rng(seed)
    A = np.triu(rng.random((n, n)) < p, 1)
    A = A | A.T
    ptr = np.concatenate([[0], np.cumsum(A.sum(1))]).astype(np.int32)
    adj = np.concatenate([np.nonzero(A[i])[0] for i in range(n)] + [np.zeros(0, np.int64)]).astype(np.int32)
    return ptr, adj


def _noalloc(torch, lib, ptr, adj, seed):
    n = ptr.shape[0] - 1
    dp = torch.as_tensor(ptr, device="cuda")
    da = torch.as_tensor(adj if adj.size else np.zeros(1, np.int32), device="cuda")
    col = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    nc = C.c_int32()
    st = lib.css_color_graph_noalloc(n, C.c_void_p(dp.data_ptr()), C.c_void_p(da.data_ptr()), C.c_uint64(seed),
                                     C.c_void_p(col.data_ptr()), C.byref(nc),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, st
    return col.cpu().numpy(), nc.value


def _regular(torch, ptr, adj, seed):
    import paper_2605_20918_gb300 as css
    n = ptr.shape[0] - 1
    col = torch.empty(n, dtype=torch.int32, device="cuda")
    with css.Context(0) as ctx:
        nc = ctx.color_graph(torch.as_tensor(ptr, device="cuda"), torch.as_tensor(adj, device="cuda"), seed, col)
    return col.cpu().numpy(), nc


def test_two_calls_in_a_row_match_the_regular_entry_point(torch, lib):
    for n, p, seed in [(3000, 0.01, 5), (600, 0.2, 9)]:
        ptr, adj = _graph(n, p, seed)
        ref, nref = _regular(torch, ptr, adj, 1004)
        for _ in range(2):  # the second call starts from the first call's leftover scratch
            got, ng = _noalloc(torch, lib, ptr, adj, 1004)
            assert ng == nref and np.array_equal(got, ref)


def test_a_warm_call_allocates_no_device_memory(torch, lib):
    """The property the entry point exists for: once its inputs and outputs exist, a call takes
    no device memory (free bytes as the driver reports them, and torch's caching allocator)."""
    ptr, adj = _graph(2000, 0.02, 3)
    dp = torch.as_tensor(ptr, device="cuda")
    da = torch.as_tensor(adj, device="cuda")
    col = torch.empty(2000, dtype=torch.int32, device="cuda")
    nc = C.c_int32()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        return lib.css_color_graph_noalloc(2000, C.c_void_p(dp.data_ptr()), C.c_void_p(da.data_ptr()),
                                           C.c_uint64(11), C.c_void_p(col.data_ptr()), C.byref(nc), stream)

    assert call() == 0  # warm: the library is loaded and the scratch address looked up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        assert call() == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_reserved() == reserved0


def test_refuses_a_malformed_graph(torch, lib):
    """A neighbour outside [0, n) or a decreasing adj_ptr is refused on the device before any
    round reads through it, and the next call on a good graph is unaffected."""
    ptr, adj = _graph(500, 0.05, 4)
    ref, nref = _regular(torch, ptr, adj, 21)
    bad_adj = adj.copy()
    bad_adj[len(bad_adj) // 2] = 500  # one past the last vertex
    bad_ptr = ptr.copy()
    bad_ptr[100] = bad_ptr[101] + 1  # decreasing
    for p_, a_ in ((ptr, bad_adj), (bad_ptr, adj)):
        dp = torch.as_tensor(p_, device="cuda")
        da = torch.as_tensor(a_, device="cuda")
        col = torch.empty(500, dtype=torch.int32, device="cuda")
        nc = C.c_int32()
        st = lib.css_color_graph_noalloc(500, C.c_void_p(dp.data_ptr()), C.c_void_p(da.data_ptr()), C.c_uint64(21),
                                         C.c_void_p(col.data_ptr()), C.byref(nc), None)
        assert st == 1  # CSS_ERR_INVALID_ARG
    got, ng = _noalloc(torch, lib, ptr, adj, 21)
    assert ng == nref and np.array_equal(got, ref)


def test_geometric_graph_and_repeat(torch, lib):
    import oracle
    from paper_2605_20918_gb300 import synth
    g = synth.water_box(4096)
    ptr, adj = oracle.neighbours(g.pos, g.box, 10.0)
    ref, nref = _regular(torch, ptr, adj, 77)
    for _ in range(2):
        got, ng = _noalloc(torch, lib, ptr, adj, 77)
        assert ng == nref and np.array_equal(got, ref)


def test_refuses_graphs_beyond_its_fixed_scratch(torch, lib):
    n = 262144 + 1
    dummy = torch.zeros(8, dtype=torch.int32, device="cuda")
    nc = C.c_int32()
    st = lib.css_color_graph_noalloc(n, C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()), C.c_uint64(1),
                                     C.c_void_p(dummy.data_ptr()), C.byref(nc), None)
    assert st == 1  # CSS_ERR_INVALID_ARG, refused on the host before any launch
