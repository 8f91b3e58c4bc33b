"""The block-Lanczos phase as one CUDA graph per call (env CSS_GRAPH=1 at css_create; the
default for a single system): results bitwise equal to launching the kernels one by one
(CSS_GRAPH=0), for a single system with the stored sampled rows, with the regenerating second
pass, and for a batch whose systems run on side streams; a second call of the same shape updates
the previous call's graph in place; by default a batch runs its kernels one by one."""
import os

import numpy as np
import pytest

import oracle
from paper_2605_20918_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def css(torch):
    import paper_2605_20918_gb300 as m
    from paper_2605_20918_gb300 import build
    build.build()
    return m


def _ctx(css, graph):
    os.environ["CSS_GRAPH"] = "1" if graph else "0"
    try:
        return css.Context(0)
    finally:
        os.environ.pop("CSS_GRAPH", None)


def _inputs(torch, css, n, kind, r_col):
    g = synth.water_box(n)
    H = synth.hamiltonian(g, kind)
    col, nc = oracle.color(g.pos, g.box, r_col, 1004)
    s = oracle.probes(col, H.b, 1005)
    dev = torch.device("cuda:0")
    return (css.DeviceBSR.from_host(H, dev), torch.as_tensor(col, device=dev), torch.as_tensor(s, device=dev), nc,
            H, synth.n_electrons(n))


@pytest.mark.parametrize("n,kind,r_col,m,prec,flags", [
    (216, "minimal", 8.0, 20, "CSS_MIXED_FP32", 0),
    (125, "dzp", 10.0, 12, "CSS_MIXED_FP32", 0),
    (125, "dzp", 10.0, 12, "CSS_FP64", 0),
    (343, "minimal", 8.0, 16, "CSS_FP64", 2),       # CSS_TWO_PASS: two captured phases per call
])
def test_graph_equals_eager_bitwise(torch, css, n, kind, r_col, m, prec, flags):
    Hd, col, s, nc, H, ne = _inputs(torch, css, n, kind, r_col)
    out = {}
    for graph in (False, True):
        c = _ctx(css, graph)
        try:
            Ps = []
            for _ in range(2):
                P = torch.full((H.nnzb, H.b, H.b), float("nan"), dtype=torch.float64, device="cuda")
                r = c.density(Hd, col, s, nc, P, kT=0.05, n_elec=ne, m=m, precision=getattr(css, prec),
                              flags=css.CSS_SYMMETRIZE | flags)
                Ps.append((P.cpu().numpy(), r["mu"], r["trP"]))
            info = c.info()
        finally:
            c.close()
        out[graph] = (Ps, info)
    (e, ie), (g, ig) = out[False], out[True]
    for a, b in zip(e, g):
        assert np.array_equal(a[0], b[0])
        assert a[1] == b[1] and a[2] == b[2]
    assert ie["graph_launches"] == 0
    phases = 2 if flags & 2 else 1
    assert ig["graph_launches"] == 2 * phases
    # the second call's graph of each mode updates the first one's in place
    assert ig["graph_instantiations"] == phases


def test_graph_batch_on_side_streams_equals_eager(torch, css):
    systems = [_inputs(torch, css, n, "minimal", 10.0) for n in (343, 125, 64, 216)]
    res = {}
    for graph in (False, True):
        c = _ctx(css, graph)
        try:
            Ps = [torch.empty((x[4].nnzb, 6, 6), dtype=torch.float64, device="cuda") for x in systems]
            r = c.density_batch([x[0] for x in systems], [x[1] for x in systems], [x[2] for x in systems],
                                [x[3] for x in systems], Ps, [dict(kT=0.05, n_elec=x[5]) for x in systems], m=20,
                                precision=css.CSS_MIXED_FP32)
            res[graph] = ([p.cpu().numpy() for p in Ps], r["mu"], c.info()["graph_launches"])
        finally:
            c.close()
    for a, b in zip(res[False][0], res[True][0]):
        assert np.array_equal(a, b)
    assert res[False][1] == res[True][1]
    assert res[False][2] == 0 and res[True][2] == 1
    os.environ.pop("CSS_GRAPH", None)
    c = css.Context(0)
    try:
        Ps = [torch.empty((x[4].nnzb, 6, 6), dtype=torch.float64, device="cuda") for x in systems]
        c.density_batch([x[0] for x in systems], [x[1] for x in systems], [x[2] for x in systems],
                        [x[3] for x in systems], Ps, [dict(kT=0.05, n_elec=x[5]) for x in systems], m=20,
                        precision=css.CSS_MIXED_FP32)
        assert c.info()["graph_launches"] == 0  # the default for a batch
        for a, p in zip(res[False][0], Ps):
            assert np.array_equal(a, p.cpu().numpy())
    finally:
        c.close()
