"""Failure detection on the GPU without a fault: the library's bounded device waits and its
device-side input checks return a status, and the context and the device stay usable.

* A grid barrier that can never complete: with CSS_TEST_MU_BARRIER_EXTRA=1 in the environment at
  css_create, the mu bisection's grid barrier waits for one CTA more than the cooperative launch
  has (a flag that nothing sets).  The wait must run out after its bounded number of polls and the
  call must return CSS_ERR_TIMEOUT; a context created afterwards without the variable must still
  give the oracle's density matrix.
* A ring of H blocks whose "empty" barriers can never complete: with CSS_TEST_SPMM_EMPTY_EXTRA=1
  at css_create, the exact-width FP32 H*V's barriers wait for one warp more than a CTA has; the
  copying thread's bounded wait must run out, the CTAs drain their copies, write zeros and return,
  and the call must return CSS_ERR_TIMEOUT with the device still usable.
* A malformed explicit graph (a neighbour outside [0, n), a decreasing adj_ptr) must be refused
  with CSS_ERR_INVALID_ARG before any Jones-Plassmann round reads through it.
"""
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
    oracle.build()
    return m


def _system(torch, n=64):
    g = synth.water_box(n)
    H = synth.hamiltonian(g, "minimal")
    col, nc = oracle.color(g.pos, g.box, 8.0, 1004)
    sign = oracle.probes(col, H.b, 1005)
    return g, H, col, nc, sign


def test_mu_barrier_timeout_returns_a_status_and_the_device_stays_usable(torch, css):
    g, H, col, nc, sign = _system(torch)
    ne = synth.n_electrons(g.n_mol)
    os.environ["CSS_TEST_MU_BARRIER_EXTRA"] = "1"
    try:
        bad = css.Context(0)
    finally:
        del os.environ["CSS_TEST_MU_BARRIER_EXTRA"]
    Hd = css.DeviceBSR.from_host(H)
    dcol = torch.as_tensor(col, device="cuda")
    dsign = torch.as_tensor(sign, device="cuda")
    P = torch.empty((H.nnzb, H.b, H.b), dtype=torch.float64, device="cuda")
    with pytest.raises(css.CSSError) as ei:
        bad.density(Hd, dcol, dsign, nc, P, kT=0.05, n_elec=ne, m=8, precision=css.CSS_FP64)
    assert ei.value.status == css.CSS_ERR_TIMEOUT
    bad.close()
    torch.cuda.synchronize()  # no sticky CUDA error
    with css.Context(0) as ctx:
        r = ctx.density(Hd, dcol, dsign, nc, P, kT=0.05, n_elec=ne, m=8, precision=css.CSS_FP64)
        torch.cuda.synchronize()
    ref = oracle.density(H, col, sign, nc, kT=0.05, n_elec=ne, m=8)
    assert float(np.abs(P.cpu().numpy() - ref["P"]).max()) < 1e-10
    assert abs(r["trP"] - ref["trP"]) < 1e-9


def test_hv_ring_timeout_returns_a_status_and_the_device_stays_usable(torch, css):
    g, H, col, nc, sign = _system(torch)
    ne = synth.n_electrons(g.n_mol)
    os.environ["CSS_TEST_SPMM_EMPTY_EXTRA"] = "1"
    try:
        bad = css.Context(0)
    finally:
        del os.environ["CSS_TEST_SPMM_EMPTY_EXTRA"]
    Hd = css.DeviceBSR.from_host(H)
    dcol = torch.as_tensor(col, device="cuda")
    dsign = torch.as_tensor(sign, device="cuda")
    P = torch.empty((H.nnzb, H.b, H.b), dtype=torch.float64, device="cuda")
    with pytest.raises(css.CSSError) as ei:
        bad.density(Hd, dcol, dsign, nc, P, kT=0.05, n_elec=ne, m=8, precision=css.CSS_MIXED_FP32)
    assert ei.value.status == css.CSS_ERR_TIMEOUT
    bad.close()
    torch.cuda.synchronize()  # no sticky CUDA error
    with css.Context(0) as ctx:
        ctx.density(Hd, dcol, dsign, nc, P, kT=0.05, n_elec=ne, m=8, precision=css.CSS_MIXED_FP32)
        torch.cuda.synchronize()
    ref = oracle.density(H, col, sign, nc, kT=0.05, n_elec=ne, m=8)
    assert float(np.abs(P.cpu().numpy() - ref["P"]).max()) < 1e-6


def test_malformed_graph_is_refused_before_the_rounds(torch, css):
    rng = np.random.default_rng(8)
    n = 400
    A = np.triu(rng.random((n, n)) < 0.05, 1)
    A = A | A.T
    ptr = np.concatenate([[0], np.cumsum(A.sum(1))]).astype(np.int32)
    adj = np.concatenate([np.nonzero(A[i])[0] for i in range(n)]).astype(np.int32)
    bad_adj = adj.copy()
    bad_adj[7] = -1
    bad_ptr = ptr.copy()
    bad_ptr[50] = bad_ptr[51] + 1
    col = torch.empty(n, dtype=torch.int32, device="cuda")
    with css.Context(0) as ctx:
        for p_, a_ in ((ptr, bad_adj), (bad_ptr, adj)):
            with pytest.raises(css.CSSError) as ei:
                ctx.color_graph(torch.as_tensor(p_, device="cuda"), torch.as_tensor(a_, device="cuda"), 5, col)
            assert ei.value.status == css.CSS_ERR_INVALID_ARG
        nc = ctx.color_graph(torch.as_tensor(ptr, device="cuda"), torch.as_tensor(adj, device="cuda"), 5, col)
    ref, nref = oracle.color_graph(ptr, adj, 5)
    assert nc == nref and np.array_equal(col.cpu().numpy(), ref)
