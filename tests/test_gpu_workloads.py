"""Full-size parity of the other synthetic workloads (GPU; about a minute each):

* 4,096 molecules x 23 orbitals (N = 94,208), R_col = 10 A, m = 40: the first block-Lanczos
  blocks of sampled colours against the oracle on the full matrix, mixed P against FP64 P at
  the same mu, symmetry, Tr P and the Ritz weights;
* 32 systems of 205-4,469 molecules (6 orbitals, log-uniform sizes, R_col = 10 A, m = 30) in
  one css_density_batch call: three systems (smallest, middle, largest) against the oracle's
  full density in FP64, every system's Tr P, and the mixed batch against the FP64 batch at the
  same mu;
* 1,000,000 molecules x 6 orbitals (N = 6,000,000), R_col = 10 A, m = 30, mixed precision with
  the regenerating second Lanczos pass: the first blocks of a sampled colour against the
  oracle on the full matrix, Tr P = N_e/2, symmetry, the Ritz weights, and the band energy per
  molecule against the oracle's on a 512-molecule system from the same generator (finite-size
  and seed spread of that intensive quantity, measured with the oracle from 512 to 4,000
  molecules: 0.05 eV; tolerance 0.2 eV).
"""
import numpy as np
import pytest

import oracle
from paper_2605_20918_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

STEPS = 3  # oracle block-Lanczos steps per sampled colour


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


def _colour(torch, ctx, g, r_col, b):
    col = torch.empty(g.n_mol, dtype=torch.int32, device="cuda")
    sign = torch.empty(g.n_mol * b, dtype=torch.int8, device="cuda")
    nc = ctx.color(torch.as_tensor(g.pos, device="cuda"), g.box, r_col, 1004, col)
    ctx.probes(col, b, 1005, sign)
    return col, sign, nc


def _check_first_blocks(H, col, sign, c, A, B, tol):
    b = H.b
    T = oracle.lanczos(H, col, sign, c, STEPS)
    scale = max(float(np.abs(T[:b, :b]).max()), 1.0)
    for j in range(STEPS):
        assert np.abs(A[c, j] - T[j * b:(j + 1) * b, j * b:(j + 1) * b]).max() <= tol * scale, ("A", c, j)
    for j in range(STEPS - 1):
        assert np.abs(B[c, j] - T[(j + 1) * b:(j + 2) * b, j * b:(j + 1) * b]).max() <= tol * scale, ("B", c, j)


def _transpose_map(H):
    rows = np.repeat(np.arange(H.n_brow), np.diff(H.row_ptr))
    key = rows.astype(np.int64) * H.n_brow + H.col_idx
    tkey = H.col_idx.astype(np.int64) * H.n_brow + rows
    order = np.argsort(key)
    return order[np.searchsorted(key[order], tkey)]


def _check_ritz_weights(ctx, col_host, nc, b):
    cnt = np.bincount(col_host, minlength=nc)
    for c, (lam, w) in enumerate(ctx.ritz()):
        assert np.isfinite(lam).all() and (w >= -1e-12).all()
        assert abs(w.sum() - b * cnt[c]) <= 1e-9 * b * max(cnt[c], 1), c


def test_4096_molecules_23_orbitals(torch, css):
    g = synth.water_box(4096)
    H = synth.hamiltonian(g, "dzp")
    ne = synth.n_electrons(4096)
    with css.Context(0) as ctx:
        col, sign, nc = _colour(torch, ctx, g, 10.0, H.b)
        Hd = css.DeviceBSR.from_host(H)
        Pm = torch.empty((H.nnzb, H.b, H.b), dtype=torch.float64, device="cuda")
        rm = ctx.density(Hd, col, sign, nc, Pm, kT=0.05, n_elec=ne, m=40, precision=css.CSS_MIXED_FP32)
        Am, Bm, _ = ctx.projected()
        _check_ritz_weights(ctx, col.cpu().numpy(), nc, H.b)
        P64 = torch.empty_like(Pm)
        r64 = ctx.density(Hd, col, sign, nc, P64, kT=0.05, n_elec=ne, m=40, precision=css.CSS_FP64, mu=rm["mu"],
                          solve_mu=False)
        A64, B64, _ = ctx.projected()
        torch.cuda.synchronize()
        ch, sh = col.cpu().numpy(), sign.cpu().numpy()
        for c in (0, nc - 1):
            _check_first_blocks(H, ch, sh, c, A64, B64, 1e-10)
            _check_first_blocks(H, ch, sh, c, Am, Bm, 1e-5)
        assert float((Pm - P64).abs().max().item()) <= 1e-6
        assert abs(2.0 * (rm["trPH"] - r64["trPH"])) / 4096 <= 1e-5
        assert abs(rm["trP"] - ne / 2) <= 1e-4 * ne / 2
        t = torch.as_tensor(_transpose_map(H), device="cuda")
        assert float((Pm - Pm[t].transpose(1, 2)).abs().max().item()) == 0.0


def test_batch_of_32_uneven_systems(torch, css):
    sizes = synth.log_uniform_sizes(32)
    systems = []
    for i, n_i in enumerate(sizes):
        gi = synth.water_box(int(n_i), seed=1001 + i)
        systems.append((gi, synth.hamiltonian(gi, "minimal")))
    with css.Context(0) as ctx:
        Hs, cols, signs, ncs, fs = [], [], [], [], []
        for gi, Hi in systems:
            c, s, nc = _colour(torch, ctx, gi, 10.0, Hi.b)
            Hs.append(css.DeviceBSR.from_host(Hi))
            cols.append(c)
            signs.append(s)
            ncs.append(nc)
            fs.append({"kT": 0.05, "n_elec": synth.n_electrons(gi.n_mol), "solve_mu": True})
        P64 = [torch.empty((H.nnzb, H.b, H.b), dtype=torch.float64, device="cuda") for _, H in systems]
        r64 = ctx.density_batch(Hs, cols, signs, ncs, P64, fs, m=30, precision=css.CSS_FP64)
        Pm = [torch.empty_like(p) for p in P64]
        fm = [{"kT": 0.05, "mu": mu, "solve_mu": False} for mu in r64["mu"]]
        rm = ctx.density_batch(Hs, cols, signs, ncs, Pm, fm, m=30, precision=css.CSS_MIXED_FP32)
        torch.cuda.synchronize()
        for i, (gi, Hi) in enumerate(systems):
            ne = synth.n_electrons(gi.n_mol)
            assert abs(r64["trP"][i] - ne / 2) <= 1e-4 * ne / 2, i
            assert float((Pm[i] - P64[i]).abs().max().item()) <= 1e-6, i
            assert abs(2.0 * (rm["trPH"][i] - r64["trPH"][i])) / gi.n_mol <= 1e-5, i
        order = np.argsort(sizes)
        for i in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
            gi, Hi = systems[i]
            ref = oracle.density(Hi, cols[i].cpu().numpy(), signs[i].cpu().numpy(), ncs[i], kT=0.05,
                                 n_elec=synth.n_electrons(gi.n_mol), m=30)
            assert float(np.abs(P64[i].cpu().numpy() - ref["P"]).max()) <= 1e-10, i
            assert abs(r64["trPH"][i] - ref["trPH"]) <= 1e-9 * max(1.0, abs(ref["trPH"])), i


def test_million_molecules_two_pass(torch, css):
    n = 1_000_000
    g = synth.water_box(n)
    H = synth.hamiltonian(g, "minimal")
    ne = synth.n_electrons(n)
    with css.Context(0) as ctx:
        col, sign, nc = _colour(torch, ctx, g, 10.0, H.b)
        Hd = css.DeviceBSR.from_host(H)
        P = torch.empty((H.nnzb, H.b, H.b), dtype=torch.float64, device="cuda")
        r = ctx.density(Hd, col, sign, nc, P, kT=0.05, n_elec=ne, m=30, precision=css.CSS_MIXED_FP32,
                        flags=css.CSS_SYMMETRIZE | css.CSS_TWO_PASS)
        A, B, _ = ctx.projected()
        ch = col.cpu().numpy()
        _check_ritz_weights(ctx, ch, nc, H.b)
        assert torch.isfinite(P).all().item()
        t = torch.as_tensor(_transpose_map(H), device="cuda")
        assert float((P - P[t].transpose(1, 2)).abs().max().item()) == 0.0
        del t, P
        torch.cuda.synchronize()
    assert abs(r["trP"] - ne / 2) <= 1e-4 * ne / 2
    _check_first_blocks(H, ch, sign.cpu().numpy(), 0, A, B, 1e-5)
    del H
    gs = synth.water_box(512)
    Hs = synth.hamiltonian(gs, "minimal")
    cs, ncs = oracle.color(gs.pos, gs.box, 10.0, 1004)
    ref = oracle.density(Hs, cs, oracle.probes(cs, Hs.b, 1005), ncs, kT=0.05, n_elec=synth.n_electrons(512), m=30)
    assert abs(2.0 * r["trPH"] / n - 2.0 * ref["trPH"] / 512) <= 0.2
