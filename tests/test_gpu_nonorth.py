"""GPU parity of the density matrix of a non-orthogonal basis (css_density_nonorth) against the
oracle (css_ref_density_nonorth), on the same S~^(-1/2) and H' inputs (the oracle's, uploaded),
so that only the new path is compared: FP64 P within 1e-10 of its scale, mixed within 5e-6; Tr(rho
S), Tr(rho H) and mu alike.

The mixed tolerance follows from the arithmetic: besides the FP32 Lanczos recurrence on H' that the
orthogonal density also has (1e-6), the non-orthogonal density passes through four FP32 sparse
products outside the recurrence (r~ = S~^(-1/2) R, S R and u = S~^(-1/2)^T S R for the start block and
the electron-count weights, and X = S~^(-1/2) X~ on the result itself), each rounding a sum of
b x neighbours x m terms at 2^-24, about 2^-24 sqrt(6 * 6 * 12) = 1.2e-6 apiece: the same 5e-6
bound as H' (whose two FP32 products carry the same error).
"""
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


@pytest.fixture(scope="module")
def ctx(css):
    c = css.Context(0)
    yield c
    c.close()


CASES = [
    # n_mol, box, S cut-off, H cut-off, R_col^S, R_col, m, solve_mu, flags
    (6, 6.0, 20.0, 20.0, 100.0, 100.0, 6, False, 1),     # full patterns, full Krylov
    (6, 6.0, 20.0, 20.0, 100.0, 100.0, 6, True, 1),
    (12, 9.0, 4.5, 5.0, 100.0, 3.5, 12, False, 0),     # shared density colours, full Krylov
    (12, 9.0, 4.5, 5.0, 100.0, 3.5, 12, False, 1),
    (27, None, 4.5, 6.0, 6.0, 5.0, 3, True, 1),        # truncated Krylov, mu solved
    (27, None, 4.5, 6.0, 6.0, 5.0, 4, True, 0),
]


def _system(n, box, rs, rh, rcs, rc):
    g = synth.water_box(n, box=box)
    S = synth.overlap(g, r_cut=rs)
    H = synth.hamiltonian(g, r_cut=rh)
    colS, ncS = oracle.color(g.pos, g.box, rcs, 1004)
    hp = oracle.hprime(S, H, colS, oracle.probes(colS, S.b, 1005), ncS, m=6)
    col, nc = oracle.color(g.pos, g.box, rc, 2004)
    return g, S, H, hp, col, oracle.probes(col, H.b, 2005), nc


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,box,rs,rh,rcs,rc,m,solve,flags", CASES)
def test_nonorth_matches_oracle(torch, css, ctx, n, box, rs, rh, rcs, rc, m, solve, flags, prec):
    g, S, H, hp, col, s, nc = _system(n, box, rs, rh, rcs, rc)
    ne = synth.n_electrons(n)
    kw = dict(kT=0.05, m=m, flags=flags)
    kw.update({"n_elec": ne} if solve else {"mu": -5.0, "solve_mu": False})
    ref = oracle.density_nonorth(S, hp["Sinv"], H, hp["Hp"], col, s, nc, **kw)
    dev = "cuda"
    Sd = css.DeviceBSR.from_host(S, dev)
    Hpd = css.DeviceBSR.from_host(synth.BSR(H.n_brow, H.b, H.row_ptr, H.col_idx, hp["Hp"]), dev)
    P = torch.full((H.nnzb, H.b, H.b), float("nan"), dtype=torch.float64, device=dev)
    p = css.CSS_FP64 if prec == "fp64" else css.CSS_MIXED_FP32
    r = ctx.density_nonorth(Sd, torch.as_tensor(hp["Sinv"], device=dev), Hpd, torch.as_tensor(H.val, device=dev),
                            torch.as_tensor(col, device=dev), torch.as_tensor(s, device=dev), nc, P, precision=p,
                            **kw)
    torch.cuda.synchronize()
    scale = max(1.0, float(np.abs(ref["P"]).max()))
    tol = 1e-10 if prec == "fp64" else 5e-6
    assert float(np.abs(P.cpu().numpy() - ref["P"]).max()) <= tol * scale
    assert abs(r["trPS"] - ref["trPS"]) <= tol * scale * n * H.b
    assert abs(r["trPH"] - ref["trPH"]) <= tol * scale * n * H.b * 30.0
    if solve:
        assert abs(r["trPS"] - 0.5 * ne) <= 1e-4 * ne / 2 + tol * scale * n * H.b


def test_nonorth_with_identity_overlap_is_the_orthogonal_density(torch, css, ctx):
    """S = S~^(-1/2) = I and H' = H: the GPU result equals css_density's on the same inputs."""
    g = synth.water_box(27)
    H = synth.hamiltonian(g)
    n, b = H.n_brow, H.b
    eye = synth.BSR(n, b, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
                    np.broadcast_to(np.eye(b), (n, b, b)).copy())
    col, nc = oracle.color(g.pos, g.box, 5.0, 2004)
    s = oracle.probes(col, b, 2005)
    dev = "cuda"
    Hd = css.DeviceBSR.from_host(H, dev)
    Ed = css.DeviceBSR.from_host(eye, dev)
    c, sg = torch.as_tensor(col, device=dev), torch.as_tensor(s, device=dev)
    P1 = torch.empty((H.nnzb, b, b), dtype=torch.float64, device=dev)
    P2 = torch.empty_like(P1)
    ne = synth.n_electrons(27)
    r1 = ctx.density_nonorth(Ed, torch.as_tensor(eye.val, device=dev), Hd, Hd.val, c, sg, nc, P1, kT=0.05, n_elec=ne,
                             m=5)
    r2 = ctx.density(Hd, c, sg, nc, P2, kT=0.05, n_elec=ne, m=5)
    torch.cuda.synchronize()
    assert float((P1 - P2).abs().max().item()) <= 1e-10
    assert abs(r1["mu"] - r2["mu"]) <= 1e-9 and abs(r1["trPS"] - r2["trP"]) <= 1e-9
