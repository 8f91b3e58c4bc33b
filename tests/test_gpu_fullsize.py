"""Full-size checks in the configuration bench.py times: 10,000 molecules x 23 orbitals
(N = 230,000), R_col = 10 A, m = 40, kT = 0.05 eV, mu solved.

The oracle needs minutes per colour at this size.  Two kinds of oracle comparison:

* the unsymmetrised columns of two colours (first and last: every block P~_IJ with colour(J) = c,
  Eq. 2 and Eq. 6) at a fixed mu of -4.0 eV, against values the oracle wrote into
  tests/golden/fullsize_10k_colours.npz (tests/golden/make_fullsize_golden.py calls only the oracle
  and the input generator): 32 sampled blocks per colour element by element (FP64 1e-10, mixed
  1e-6) and Tr / Tr(H .) over all of the colour's blocks;
* the first block-Lanczos steps of sampled colours on the full matrix (paragraph after Eq. 4),
  computed by the oracle during the test, against the GPU's projected blocks A_0..A_2, B_0, B_1.

The rest is checked through properties that hold at any size: the symmetrised P is symmetric on
the pattern, Tr P matches N_e/2 (the mu rule), the Ritz weights of each colour sum to b|c|
(Eq. 7), and the mixed-precision P equals the FP64 P, each with its own solved mu (the product as
called), within 1e-6 max-abs and 1e-5 eV/molecule.
"""
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2605_20918_gb300 import synth

pytestmark = pytest.mark.gpu

N_MOL, R_COL, M, KT = 10000, 10.0, 40, 0.05
STEPS = 3  # oracle block-Lanczos steps per sampled colour
GOLDEN = Path(__file__).resolve().parent / "golden" / "fullsize_10k_colours.npz"


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def run(torch):
    """One mixed (solved mu) and one FP64 (same mu) P build of the 10k workload on the GPU."""
    import paper_2605_20918_gb300 as css
    from paper_2605_20918_gb300 import build
    build.build()
    oracle.build()
    g = synth.water_box(N_MOL)
    H = synth.hamiltonian(g, "dzp")
    ctx = css.Context(0)
    dev = "cuda"
    col = torch.empty(N_MOL, dtype=torch.int32, device=dev)
    sign = torch.empty(N_MOL * H.b, dtype=torch.int8, device=dev)
    nc = ctx.color(torch.as_tensor(g.pos, device=dev), g.box, R_COL, 1004, col)
    ctx.probes(col, H.b, 1005, sign)
    Hd = css.DeviceBSR.from_host(H)
    ne = synth.n_electrons(N_MOL)
    Pm = torch.empty((H.nnzb, H.b, H.b), dtype=torch.float64, device=dev)
    rm = ctx.density(Hd, col, sign, nc, Pm, kT=KT, n_elec=ne, m=M, precision=css.CSS_MIXED_FP32)
    Am, Bm, nbm = ctx.projected()
    ritz_m = ctx.ritz()
    P64 = torch.empty_like(Pm)
    r64 = ctx.density(Hd, col, sign, nc, P64, kT=KT, n_elec=ne, m=M, precision=css.CSS_FP64)
    A64, B64, nb64 = ctx.projected()
    # unsymmetrised, at the fixed mu of the stored oracle columns
    gold = np.load(GOLDEN)
    Pt = {}
    for name, prec in (("fp64", css.CSS_FP64), ("mixed", css.CSS_MIXED_FP32)):
        Pt[name] = torch.empty_like(Pm)
        ctx.density(Hd, col, sign, nc, Pt[name], mu=float(gold["mu"]), kT=float(gold["kT"]), solve_mu=False,
                    m=int(gold["m"]), precision=prec, flags=0)
    torch.cuda.synchronize()
    out = dict(g=g, H=H, nc=nc, col=col.cpu().numpy(), sign=sign.cpu().numpy(), ne=ne, rm=rm, r64=r64,
               Pm=Pm, P64=P64, Am=Am, Bm=Bm, nbm=nbm, A64=A64, B64=B64, nb64=nb64, ritz_m=ritz_m, gold=gold,
               Pt64=Pt["fp64"], Ptm=Pt["mixed"])
    yield out
    ctx.close()


def _oracle_blocks(run, c):
    H, b = run["H"], run["H"].b
    T = oracle.lanczos(H, run["col"], run["sign"], c, STEPS)
    A = [T[j * b:(j + 1) * b, j * b:(j + 1) * b] for j in range(STEPS)]
    B = [T[(j + 1) * b:(j + 2) * b, j * b:(j + 1) * b] for j in range(STEPS - 1)]
    return A, B


@pytest.mark.parametrize("which", [0, -1])
def test_first_lanczos_blocks_match_the_oracle(run, which):
    """A_0..A_2 and B_0, B_1 of a sampled colour (first and last) against the oracle's own
    block-Lanczos steps on the full 230,000-row matrix: FP64 to 1e-10 relative to ||H||, the
    mixed path to FP32 level (1e-5)."""
    c = which % run["nc"]
    A, B = _oracle_blocks(run, c)
    scale = max(np.abs(A[0]).max(), 1.0)
    for j in range(STEPS):
        assert np.abs(run["A64"][c, j] - A[j]).max() <= 1e-10 * scale, ("A", j)
        assert np.abs(run["Am"][c, j] - A[j]).max() <= 1e-5 * scale, ("A mixed", j)
    for j in range(STEPS - 1):
        assert np.abs(run["B64"][c, j] - B[j]).max() <= 1e-10 * scale, ("B", j)
        assert np.abs(run["Bm"][c, j] - B[j]).max() <= 1e-5 * scale, ("B mixed", j)


def test_colour_columns_match_the_oracle(run, torch):
    """Unsymmetrised columns of the first and the last colour against the oracle's (fixed mu):
    sampled blocks element by element, and the colour's share of Tr P~ and Tr(P~ H) over all of
    its blocks."""
    gold, H = run["gold"], run["H"]
    assert run["nc"] == int(gold["n_colours"])
    cs = int((run["col"].astype(np.int64) * np.arange(N_MOL, dtype=np.int64)).sum())
    assert cs == int(gold["colour_checksum"])  # the same colouring as the oracle's
    rows = np.repeat(np.arange(H.n_brow), np.diff(H.row_ptr))
    Hv = torch.as_tensor(H.val, device="cuda")
    for c in gold["colours"]:
        c = int(c)
        blk = gold[f"blocks_{c}"]
        ref = gold[f"P_{c}"]
        mask = torch.as_tensor(run["col"][H.col_idx] == c, device="cuda")
        diag = torch.as_tensor((run["col"][H.col_idx] == c) & (rows == H.col_idx), device="cuda")
        for name, tol in (("Pt64", 1e-10), ("Ptm", 1e-6)):
            got = run[name][torch.as_tensor(blk, device="cuda")].cpu().numpy()
            assert float(np.abs(got - ref).max()) <= tol, (name, c, float(np.abs(got - ref).max()))
            P = run[name]
            trp = float(torch.diagonal(P[diag], dim1=1, dim2=2).sum().item())
            trph = float((P[mask] * Hv[mask]).sum().item())
            assert abs(trp - float(gold[f"trP_{c}"])) <= tol * int(gold[f"nblocks_{c}"]), (name, c, trp)
            assert abs(trph - float(gold[f"trPH_{c}"])) <= 30.0 * tol * int(gold[f"nblocks_{c}"]), (name, c, trph)


def test_mixed_equals_fp64_with_mu_solved(run, torch):
    """The product as called in both precisions (each solves its own mu): P within 1e-6 max-abs,
    band energy within 1e-5 eV per molecule, and the two chemical potentials close."""
    dP = float((run["Pm"] - run["P64"]).abs().max().item())
    dE = abs(2.0 * (run["rm"]["trPH"] - run["r64"]["trPH"])) / N_MOL
    assert dP <= 1e-6, dP
    assert dE <= 1e-5, dE
    assert abs(run["rm"]["mu"] - run["r64"]["mu"]) <= 1e-3


def test_symmetric_on_the_pattern(run, torch):
    H = run["H"]
    rows = np.repeat(np.arange(H.n_brow), np.diff(H.row_ptr))
    key = rows.astype(np.int64) * H.n_brow + H.col_idx
    tkey = H.col_idx.astype(np.int64) * H.n_brow + rows
    order = np.argsort(key)
    trans = order[np.searchsorted(key[order], tkey)]
    t = torch.as_tensor(trans, device="cuda")
    for P in (run["Pm"], run["P64"]):
        assert torch.isfinite(P).all().item()
        assert float((P - P[t].transpose(1, 2)).abs().max().item()) == 0.0


def test_electron_count_and_ritz_weights(run):
    # the mu rule: |N(mu) - N_e/2| <= 1e-4 N_e/2 on the Ritz quadrature; Tr P follows it up to
    # the contamination of the sampled reconstruction
    assert abs(run["rm"]["trP"] - run["ne"] / 2) <= 1e-4 * run["ne"] / 2
    cnt = np.bincount(run["col"], minlength=run["nc"])
    b = run["H"].b
    for c, (lam, w) in enumerate(run["ritz_m"]):
        assert np.isfinite(lam).all() and (w >= -1e-12).all()
        assert abs(w.sum() - b * cnt[c]) <= 1e-9 * b * cnt[c], c
