"""GPU parity: the CUDA path through the C-ABI against the FP64 CPU oracle.

Colours and probe signs bit-exact; P within 1e-10 max-abs in FP64 mode; within 1e-6 max-abs
and 1e-5 eV/molecule band energy in mixed mode (FP32 H*V and Krylov vectors).
"""
import numpy as np
import pytest

import oracle
from paper_2605_20918_gb300 import synth
from tests.dense_truth import Dense, fermi

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
MIXED_P_TOL = 1e-6
MIXED_E_TOL = 1e-5   # eV per molecule, band energy 2 Tr(PH) / n_mol


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


def gpu_colour(torch, ctx, g, r_col, seed=1004):
    xyz = torch.as_tensor(g.pos, device="cuda")
    col = torch.empty(g.n_mol, dtype=torch.int32, device="cuda")
    nc = ctx.color(xyz, g.box, r_col, seed, col)
    return col.cpu().numpy(), nc


def gpu_density(torch, css, ctx, H, col, sign, nc, **kw):
    Hd = css.DeviceBSR.from_host(H)
    c = torch.as_tensor(col, device="cuda")
    s = torch.as_tensor(sign, device="cuda")
    P = torch.full((H.nnzb, H.b, H.b), float("nan"), dtype=torch.float64, device="cuda")
    r = ctx.density(Hd, c, s, nc, P, **kw)
    torch.cuda.synchronize()
    r["P"] = P.cpu().numpy()
    return r


# ---------------------------------------------------------------------- colouring
@pytest.mark.parametrize("n,r_col", [(1, 8.0), (27, 100.0), (64, 8.0), (216, 8.0), (1000, 10.0), (4096, 10.0),
                                     (10000, 10.0)])
def test_colour_bit_exact(torch, css, ctx, n, r_col):
    g = synth.water_box(n)
    col, nc = gpu_colour(torch, ctx, g, r_col)
    ref, nref = oracle.color(g.pos, g.box, r_col, 1004)
    assert nc == nref
    assert np.array_equal(col, ref)


def test_colour_bit_exact_md_step_and_seed(torch, css, ctx):
    seq = list(synth.md_sequence(512, 3))
    for t, g in enumerate(seq):
        col, nc = gpu_colour(torch, ctx, g, 10.0, seed=7 + t)
        ref, nref = oracle.color(g.pos, g.box, 10.0, 7 + t)
        assert nc == nref and np.array_equal(col, ref)


@pytest.mark.parametrize("n,p", [(1, 0.0), (50, 0.1), (200, 0.3), (64, 1.0)])
def test_colour_graph_bit_exact(torch, css, ctx, n, p):
    rng = np.random.default_rng(n)
    A = np.triu(rng.random((n, n)) < p, 1)
    A = A | A.T
    ptr = np.concatenate([[0], np.cumsum(A.sum(1))]).astype(np.int32)
    adj = np.concatenate([np.nonzero(A[i])[0] for i in range(n)] + [np.zeros(0, np.int64)]).astype(np.int32)
    col = torch.empty(n, dtype=torch.int32, device="cuda")
    nc = ctx.color_graph(torch.as_tensor(ptr, device="cuda"), torch.as_tensor(adj, device="cuda"), 99, col)
    ref, nref = oracle.color_graph(ptr, adj, 99)
    assert nc == nref and np.array_equal(col.cpu().numpy(), ref)


@pytest.mark.parametrize("b,flags", [(6, 0), (23, 0), (23, 1)])
def test_probe_signs_bit_exact(torch, css, ctx, b, flags):
    col = torch.zeros(777, dtype=torch.int32, device="cuda")
    s = torch.empty(777 * b, dtype=torch.int8, device="cuda")
    ctx.probes(col, b, 1005, s, flags=flags)
    ref = oracle.probes(np.zeros(777, np.int32), b, 1005, flags)
    assert np.array_equal(s.cpu().numpy(), ref)


# ------------------------------------------------------------------------- FP64
def _system(n, kind, r_col, **hk):
    g = synth.water_box(n, box=hk.pop("box", None))
    H = synth.hamiltonian(g, kind, **hk)
    col, nc = oracle.color(g.pos, g.box, r_col, 1004)
    s = oracle.probes(col, H.b, 1005)
    return g, H, col, s, nc


FP64_CASES = [
    # (n_mol, kind, R_col, m, extra density kwargs, hamiltonian kwargs)
    (64, "minimal", 8.0, 8, {}, {}),
    (64, "minimal", 8.0, 30, {}, {}),                              # the 64-molecule workload
    (125, "minimal", 8.0, 12, {"flags": 0}, {}),                   # no symmetrisation
    (27, "dzp", 6.0, 4, {}, {}),
    (64, "dzp", 10.0, 6, {"solve_mu": False, "mu": -4.0}, {}),
    (64, "minimal", 8.0, 10, {"flags": 1 | 4}, {}),                # local reorthogonalisation
    (64, "minimal", 8.0, 10, {"flags": 1 | 2}, {}),                # two-pass basis regeneration
    (27, "minimal", 6.0, 10, {}, {"coupling": 0.0}),              # breakdown (invariant subspaces)
    (64, "minimal", 8.0, 8, {"kT": 0.0, "solve_mu": False, "mu": -4.5}, {}),  # T = 0 step function
    (200, "minimal", 10.0, 6, {"kT": 0.3}, {}),
]


@pytest.mark.parametrize("n,kind,r_col,m,kw,hk", FP64_CASES)
def test_density_fp64_matches_oracle(torch, css, ctx, n, kind, r_col, m, kw, hk):
    g, H, col, s, nc = _system(n, kind, r_col, **hk)
    ne = synth.n_electrons(n)
    args = dict(kT=0.05, n_elec=ne, solve_mu=True, m=m, flags=1)
    args.update(kw)
    ref = oracle.density(H, col, s, nc, mu=args.get("mu", 0.0), kT=args["kT"], n_elec=ne,
                         solve_mu=args["solve_mu"], m=m, flags=args["flags"] & ~2)
    got = gpu_density(torch, css, ctx, H, col, s, nc, precision=css.CSS_FP64, **args)
    err = float(np.abs(got["P"] - ref["P"]).max())
    assert err < FP64_TOL, err
    assert abs(got["trP"] - ref["trP"]) < 1e-8
    assert abs(got["trPH"] - ref["trPH"]) < 1e-7
    assert (got["status"] == css.CSS_WARN_BREAKDOWN) == (ref["n_breakdown"] > 0)


@pytest.mark.parametrize("n,kind,r_col,m,kw,hk", FP64_CASES)
def test_density_fp64_split_matches_oracle(torch, css, ctx, n, kind, r_col, m, kw, hk):
    """CSS_FP64_SPLIT: FP64 everywhere but the recurrence's H*V, which runs on the FP32 FMA pipe with
    every value as an FP32 hi + lo pair, error-free products and TwoSum accumulation; the FP64
    tolerances against the oracle on every FP64 case (6 and 23 orbitals, breakdown, two-pass,
    T = 0, no symmetrisation)."""
    g, H, col, s, nc = _system(n, kind, r_col, **hk)
    ne = synth.n_electrons(n)
    args = dict(kT=0.05, n_elec=ne, solve_mu=True, m=m, flags=1)
    args.update(kw)
    ref = oracle.density(H, col, s, nc, mu=args.get("mu", 0.0), kT=args["kT"], n_elec=ne,
                         solve_mu=args["solve_mu"], m=m, flags=args["flags"] & ~2)
    got = gpu_density(torch, css, ctx, H, col, s, nc, precision=css.CSS_FP64_SPLIT, **args)
    err = float(np.abs(got["P"] - ref["P"]).max())
    assert err < FP64_TOL, err
    assert abs(got["trP"] - ref["trP"]) < 1e-8
    assert abs(got["trPH"] - ref["trPH"]) < 1e-7
    assert (got["status"] == css.CSS_WARN_BREAKDOWN) == (ref["n_breakdown"] > 0)


def test_fp64_split_batch_equals_single(torch, css, ctx):
    """A batch of two systems under CSS_FP64_SPLIT (their passes in turn on one stream) gives each
    system's single-call P to the batch tolerance of the FP64 mode."""
    sysd = [_system(n, "dzp", 8.0) for n in (64, 27)]
    dev = torch.device("cuda:0")
    singles, Hs, cs, ss, ncs, Ps, fs = [], [], [], [], [], [], []
    for g, H, col, s, nc in sysd:
        ne = synth.n_electrons(g.n_mol)
        singles.append(gpu_density(torch, css, ctx, H, col, s, nc, kT=0.05, n_elec=ne, m=6,
                                   precision=css.CSS_FP64_SPLIT)["P"])
        Hs.append(css.DeviceBSR.from_host(H, dev))
        cs.append(torch.as_tensor(col, device=dev))
        ss.append(torch.as_tensor(s, device=dev))
        ncs.append(nc)
        Ps.append(torch.empty((H.nnzb, H.b, H.b), dtype=torch.float64, device=dev))
        fs.append(dict(kT=0.05, n_elec=ne))
    ctx.density_batch(Hs, cs, ss, ncs, Ps, fs, m=6, precision=css.CSS_FP64_SPLIT)
    for a, p in zip(singles, Ps):
        assert np.abs(a - p.cpu().numpy()).max() < 1e-12


def test_fp64_split_refuses_other_block_widths(torch, css, ctx):
    """The split-FP64 H*V exists for b = 6 and b = 23; another b is refused with CSS_ERR_UNSUPPORTED."""
    g = synth.water_box(27)
    lv = np.sort(np.random.default_rng(5).uniform(-12, 8, size=(27, 5)), axis=1)
    H = synth.hamiltonian(g, levels=lv)
    col, nc = oracle.color(g.pos, g.box, 6.0, 1004)
    s = oracle.probes(col, 5, 1005)
    with pytest.raises(css.CSSError) as e:
        gpu_density(torch, css, ctx, H, col, s, nc, mu=-1.0, kT=0.1, solve_mu=False, m=4,
                    precision=css.CSS_FP64_SPLIT)
    assert e.value.status == 7


def test_degenerate_colouring_is_exact_f_of_H(torch, css, ctx):
    g = synth.water_box(8)
    H = synth.hamiltonian(g)
    col, nc = gpu_colour(torch, ctx, g, 100.0)
    s = oracle.probes(col, H.b, 1005)
    got = gpu_density(torch, css, ctx, H, col, s, nc, kT=0.05, n_elec=64.0, m=8, precision=css.CSS_FP64)
    dn = Dense(H)
    ref = dn.on_pattern(dn.f(dn.mu_exact(64.0, 0.05), 0.05))
    assert np.abs(got["P"] - ref).max() < 1e-10


def test_two_level_closed_form(torch, css, ctx):
    a, d, t = -1.3, 0.4, 0.7
    H = synth.BSR(n_brow=2, b=1, row_ptr=np.array([0, 2, 4], np.int32), col_idx=np.array([0, 1, 0, 1], np.int32),
                  val=np.array([a, t, t, d], float).reshape(4, 1, 1))
    got = gpu_density(torch, css, ctx, H, np.array([0, 1], np.int32), np.array([1, -1], np.int8), 2, mu=-0.2,
                      kT=0.25, solve_mu=False, m=2, precision=css.CSS_FP64)
    w, V = np.linalg.eigh(H.dense())
    F = (V * fermi(w, -0.2, 0.25)) @ V.T
    assert np.abs(got["P"].ravel() - F.ravel()).max() < 1e-13


@pytest.mark.parametrize("b", [2, 5, 9, 17, 32])
def test_generic_block_widths(torch, css, ctx, b):
    n = 27
    g = synth.water_box(n)
    lv = np.sort(np.random.default_rng(b).uniform(-12, 8, size=(n, b)), axis=1)
    H = synth.hamiltonian(g, levels=lv)
    col, nc = oracle.color(g.pos, g.box, 6.0, 1004)
    s = oracle.probes(col, b, 1005)
    m = max(2, 64 // b)
    ref = oracle.density(H, col, s, nc, mu=-1.0, kT=0.1, solve_mu=False, m=m)
    got = gpu_density(torch, css, ctx, H, col, s, nc, mu=-1.0, kT=0.1, solve_mu=False, m=m, precision=css.CSS_FP64)
    assert np.abs(got["P"] - ref["P"]).max() < FP64_TOL


def test_empty_colours_change_nothing(torch, css, ctx):
    g, H, col, s, nc = _system(64, "minimal", 8.0)
    a = gpu_density(torch, css, ctx, H, col, s, nc, kT=0.05, n_elec=512.0, m=8)
    b = gpu_density(torch, css, ctx, H, col, s, nc + 3, kT=0.05, n_elec=512.0, m=8)
    assert np.array_equal(a["P"], b["P"])


def test_bitwise_repeatable(torch, css, ctx):
    g, H, col, s, nc = _system(125, "minimal", 8.0)
    a = gpu_density(torch, css, ctx, H, col, s, nc, kT=0.05, n_elec=1000.0, m=10)
    b = gpu_density(torch, css, ctx, H, col, s, nc, kT=0.05, n_elec=1000.0, m=10)
    assert np.array_equal(a["P"], b["P"]) and a["mu"] == b["mu"]


# ------------------------------------------------------------------------ mixed
@pytest.mark.parametrize("n,kind,r_col,m,solve", [(64, "minimal", 8.0, 30, True), (343, "minimal", 10.0, 20, True),
                                                   (125, "dzp", 10.0, 40, True), (125, "dzp", 10.0, 8, False)])
def test_density_mixed_within_tolerance(torch, css, ctx, n, kind, r_col, m, solve):
    g, H, col, s, nc = _system(n, kind, r_col)
    ne = synth.n_electrons(n)
    ref = oracle.density(H, col, s, nc, kT=0.05, n_elec=ne, m=m, mu=-4.0, solve_mu=solve)
    got = gpu_density(torch, css, ctx, H, col, s, nc, kT=0.05, n_elec=ne, m=m, mu=-4.0, solve_mu=solve,
                      precision=css.CSS_MIXED_FP32)
    dP = float(np.abs(got["P"] - ref["P"]).max())
    dE = abs(2 * got["trPH"] - 2 * ref["trPH"]) / n
    assert dP < MIXED_P_TOL, dP
    assert dE < MIXED_E_TOL, dE
    assert abs(got["trP"] - ref["trP"]) < 1e-4


@pytest.mark.parametrize("env", ["CSS_HV_TC", "CSS_ROWS_STREAM"])
@pytest.mark.parametrize("n,r_col,m,solve", [(125, 10.0, 40, True), (64, 10.0, 8, False)])
def test_alternative_fp32_kernels_match_oracle(torch, css, n, r_col, m, solve, env):
    """The opt-in FP32 kernels for 17 <= b <= 24 (selected by an environment variable at
    css_create): H*V on the tensor cores (tcgen05, 3xTF32 with the on-site blocks in three parts)
    and the streaming row passes; each against the oracle like the default mixed path, with the
    stored sampled rows and with the regenerating second pass."""
    import os
    g, H, col, s, nc = _system(n, "dzp", r_col)
    ne = synth.n_electrons(n)
    ref = oracle.density(H, col, s, nc, kT=0.05, n_elec=ne, m=m, mu=-4.0, solve_mu=solve)
    os.environ[env] = "1"
    try:
        c2 = css.Context(0)
    finally:
        del os.environ[env]
    try:
        got = gpu_density(torch, css, c2, H, col, s, nc, kT=0.05, n_elec=ne, m=m, mu=-4.0, solve_mu=solve,
                          precision=css.CSS_MIXED_FP32)
        two = gpu_density(torch, css, c2, H, col, s, nc, kT=0.05, n_elec=ne, m=m, mu=-4.0, solve_mu=solve,
                          precision=css.CSS_MIXED_FP32, flags=css.CSS_SYMMETRIZE | css.CSS_TWO_PASS)
    finally:
        c2.close()
    dP = float(np.abs(got["P"] - ref["P"]).max())
    assert dP < MIXED_P_TOL, dP
    assert abs(2 * got["trPH"] - 2 * ref["trPH"]) / n < MIXED_E_TOL
    assert abs(got["trP"] - ref["trP"]) < 1e-4
    assert float(np.abs(two["P"] - ref["P"]).max()) < MIXED_P_TOL


@pytest.mark.parametrize("n,r_col,m,solve", [(125, 10.0, 40, True), (216, 10.0, 12, False)])
def test_3xtf32_precision_matches_oracle(torch, css, ctx, n, r_col, m, solve):
    """CSS_MIXED_3XTF32: the recurrence's H*V on the tensor cores (TF32 products of split
    operands, FP32 accumulation), everything else as in the FP32 mode; against the oracle at the
    mixed-precision tolerances, single system and a batch of two."""
    g, H, col, s, nc = _system(n, "dzp", r_col)
    ne = synth.n_electrons(n)
    ref = oracle.density(H, col, s, nc, kT=0.05, n_elec=ne, m=m, mu=-4.0, solve_mu=solve)
    got = gpu_density(torch, css, ctx, H, col, s, nc, kT=0.05, n_elec=ne, m=m, mu=-4.0, solve_mu=solve,
                      precision=css.CSS_MIXED_3XTF32)
    dP = float(np.abs(got["P"] - ref["P"]).max())
    assert dP < MIXED_P_TOL, dP
    assert abs(2 * got["trPH"] - 2 * ref["trPH"]) / n < MIXED_E_TOL
    assert abs(got["trP"] - ref["trP"]) < 1e-4
    dev = torch.device("cuda:0")
    Hd = css.DeviceBSR.from_host(H, dev)
    cd = torch.as_tensor(col, device=dev)
    sd = torch.as_tensor(s, device=dev)
    Ps = [torch.empty((H.nnzb, H.b, H.b), dtype=torch.float64, device=dev) for _ in range(2)]
    f = dict(mu=-4.0, kT=0.05, n_elec=ne, solve_mu=solve)
    ctx.density_batch([Hd, Hd], [cd, cd], [sd, sd], [nc, nc], Ps, [f, f], m=m, precision=css.CSS_MIXED_3XTF32)
    for p in Ps:
        assert float(np.abs(p.cpu().numpy() - ref["P"]).max()) < MIXED_P_TOL


def test_3xtf32_precision_refuses_other_block_widths(torch, css, ctx):
    """The tensor-core H*V covers 17 <= b <= 24; CSS_MIXED_3XTF32 with the 6-orbital basis is
    refused with CSS_ERR_UNSUPPORTED rather than run on another kernel."""
    g, H, col, s, nc = _system(27, "minimal", 8.0)
    with pytest.raises(css.CSSError) as e:
        gpu_density(torch, css, ctx, H, col, s, nc, kT=0.05, n_elec=synth.n_electrons(27), m=6,
                    precision=css.CSS_MIXED_3XTF32)
    assert e.value.status == 7


@pytest.mark.parametrize("n,kind,r_col,m", [(125, "dzp", 10.0, 12), (343, "minimal", 8.0, 12), (27, "dzp", 6.0, 6)])
def test_exact_width_hv_equals_the_padded_kernel_bitwise(torch, css, n, kind, r_col, m):
    """FP32 H*V for b = 6 and b = 23 runs by default in the exact-width kernel (packed FMAs over
    column pairs, no padded rows or columns); the padded kernel (CSS_SPMM_VARIANT=0 at css_create)
    forms every output from the same IEEE FMAs in the same order, so the mixed P must be bitwise
    the same, for every launch variant of the exact-width kernel (CSS_SPMM_DUP_VARIANT=0..3) and
    with the regenerating second pass.  The column counts span several CTA tiles with a ragged
    last one."""
    import os
    g, H, col, s, nc = _system(n, kind, r_col)
    ne = synth.n_electrons(n)
    kw = dict(kT=0.05, n_elec=ne, m=m, precision=css.CSS_MIXED_FP32)

    def run(env, flags=css.CSS_SYMMETRIZE):
        os.environ.update(env)
        try:
            c2 = css.Context(0)
        finally:
            for k in env:
                del os.environ[k]
        try:
            return gpu_density(torch, css, c2, H, col, s, nc, flags=flags, **kw)
        finally:
            c2.close()

    ref = run({"CSS_SPMM_VARIANT": "0"})
    for v in range(4):
        got = run({"CSS_SPMM_DUP_VARIANT": str(v)})
        assert np.array_equal(got["P"], ref["P"]), v
        assert got["mu"] == ref["mu"] and got["trP"] == ref["trP"], v
    two_ref = run({"CSS_SPMM_VARIANT": "0"}, css.CSS_SYMMETRIZE | css.CSS_TWO_PASS)
    two = run({}, css.CSS_SYMMETRIZE | css.CSS_TWO_PASS)
    assert np.array_equal(two["P"], two_ref["P"])


@pytest.mark.parametrize("kind", ["minimal", "dzp"])
def test_exact_width_hv_in_a_batch_equals_the_padded_kernel_bitwise(torch, css, kind):
    """The same bitwise equality through css_density_batch, where the systems' Lanczos passes run
    concurrently on side streams and each system's H*V shape is tuned on its own stream."""
    import os
    sizes = [27, 64, 125, 216, 343, 100] if kind == "minimal" else [27, 64, 125]
    systems = []
    for i, n_i in enumerate(sizes):
        gi = synth.water_box(n_i, seed=1101 + i)
        systems.append((gi, synth.hamiltonian(gi, kind)))

    def run(env):
        os.environ.update(env)
        try:
            c2 = css.Context(0)
        finally:
            for k in env:
                del os.environ[k]
        try:
            Hs, cols, signs, ncs, fs = [], [], [], [], []
            for gi, Hi in systems:
                col, nc = oracle.color(gi.pos, gi.box, 8.0, 1004)
                Hs.append(css.DeviceBSR.from_host(Hi))
                cols.append(torch.as_tensor(col, device="cuda"))
                signs.append(torch.as_tensor(oracle.probes(col, Hi.b, 1005), device="cuda"))
                ncs.append(nc)
                fs.append({"kT": 0.05, "n_elec": synth.n_electrons(gi.n_mol), "solve_mu": True})
            P = [torch.empty((H.nnzb, H.b, H.b), dtype=torch.float64, device="cuda") for _, H in systems]
            c2.density_batch(Hs, cols, signs, ncs, P, fs, m=12, precision=css.CSS_MIXED_FP32)
            torch.cuda.synchronize()
            return P
        finally:
            c2.close()

    ref = run({"CSS_SPMM_VARIANT": "0"})
    got = run({})
    for i in range(len(systems)):
        assert torch.equal(got[i], ref[i]), i


# ------------------------------------------- energy-weighted density matrix (forces)
@pytest.mark.parametrize("n,kind,r_col,m,flags", [(64, "minimal", 8.0, 10, 1), (125, "minimal", 8.0, 12, 0),
                                                  (27, "dzp", 6.0, 6, 1), (64, "minimal", 8.0, 10, 1 | 2)])
def test_energy_weighted_fp64_matches_oracle(torch, css, ctx, n, kind, r_col, m, flags):
    """rho_E (Z built with lambda f(lambda), mu from f) against the oracle: FP64 to 1e-10 of
    its scale (entries carry energies of tens of eV); the two-pass path too."""
    g, H, col, s, nc = _system(n, kind, r_col)
    ne = synth.n_electrons(n)
    ew = css.CSS_ENERGY_WEIGHTED
    ref = oracle.density(H, col, s, nc, kT=0.05, n_elec=ne, m=m, flags=(flags & ~2) | oracle.ENERGY_WEIGHTED)
    got = gpu_density(torch, css, ctx, H, col, s, nc, kT=0.05, n_elec=ne, m=m, flags=flags | ew,
                      precision=css.CSS_FP64)
    scale = max(1.0, float(np.abs(ref["P"]).max()))
    assert float(np.abs(got["P"] - ref["P"]).max()) < FP64_TOL * scale
    assert abs(got["trP"] - ref["trP"]) < 1e-8 * max(1.0, abs(ref["trP"]))
    assert got["mu"] == pytest.approx(ref["mu"], abs=1e-9)


def test_energy_weighted_mixed_within_tolerance(torch, css, ctx):
    g, H, col, s, nc = _system(125, "dzp", 10.0)
    ne = synth.n_electrons(125)
    ew = css.CSS_ENERGY_WEIGHTED
    ref = oracle.density(H, col, s, nc, kT=0.05, n_elec=ne, m=20, mu=-4.0, solve_mu=False,
                         flags=1 | oracle.ENERGY_WEIGHTED)
    got = gpu_density(torch, css, ctx, H, col, s, nc, kT=0.05, n_elec=ne, m=20, mu=-4.0, solve_mu=False,
                      flags=1 | ew, precision=css.CSS_MIXED_FP32)
    scale = max(1.0, float(np.abs(ref["P"]).max()))
    assert float(np.abs(got["P"] - ref["P"]).max()) < MIXED_P_TOL * scale


# ------------------------------------------------ S^(-1/2) of an overlap (Eq. 8-10)
@pytest.mark.parametrize("n,kind,r_col,m,flags", [(64, "minimal", 6.0, 10, 1), (125, "minimal", 9.0, 10, 0),
                                                  (27, "dzp", 6.0, 6, 1), (64, "minimal", 6.0, 10, 1 | 2)])
def test_inv_sqrt_fp64_matches_oracle(torch, css, ctx, n, kind, r_col, m, flags):
    g = synth.water_box(n)
    S = synth.overlap(g, kind)
    col, nc = oracle.color(g.pos, g.box, r_col, 1004)
    s = oracle.probes(col, S.b, 1005)
    ref = oracle.density(S, col, s, nc, m=m, flags=(flags & ~2) | oracle.INV_SQRT)
    got = gpu_density(torch, css, ctx, S, col, s, nc, m=m, flags=flags | css.CSS_INV_SQRT,
                      precision=css.CSS_FP64)
    assert float(np.abs(got["P"] - ref["P"]).max()) < FP64_TOL
    assert abs(got["trP"] - ref["trP"]) < 1e-9 * max(1.0, abs(ref["trP"]))


def test_inv_sqrt_mixed_within_tolerance(torch, css, ctx):
    g = synth.water_box(343)
    S = synth.overlap(g, "dzp")
    col, nc = oracle.color(g.pos, g.box, 9.0, 1004)
    s = oracle.probes(col, S.b, 1005)
    ref = oracle.density(S, col, s, nc, m=10, flags=1 | oracle.INV_SQRT)
    got = gpu_density(torch, css, ctx, S, col, s, nc, m=10, flags=1 | css.CSS_INV_SQRT,
                      precision=css.CSS_MIXED_FP32)
    assert float(np.abs(got["P"] - ref["P"]).max()) < MIXED_P_TOL


# ------------------------------------------- H' of a non-orthogonal basis (after Eq. 10)
@pytest.mark.parametrize("n,kind,r_col,m,flags,prec", [(64, "minimal", 6.0, 10, 1, "fp64"),
                                                        (125, "minimal", 9.0, 10, 0, "fp64"),
                                                        (27, "dzp", 6.0, 6, 1, "fp64"),
                                                        (125, "dzp", 9.0, 10, 1, "mixed")])
def test_hprime_matches_oracle(torch, css, ctx, n, kind, r_col, m, flags, prec):
    g = synth.water_box(n)
    S = synth.overlap(g, kind)
    H = synth.hamiltonian(g, kind)
    col, nc = oracle.color(g.pos, g.box, r_col, 1004)
    s = oracle.probes(col, S.b, 1005)
    ref = oracle.hprime(S, H, col, s, nc, m=m, flags=flags)
    Sd, Hd = css.DeviceBSR.from_host(S), css.DeviceBSR.from_host(H)
    Si = torch.full((S.nnzb, S.b, S.b), float("nan"), dtype=torch.float64, device="cuda")
    Hp = torch.full((H.nnzb, H.b, H.b), float("nan"), dtype=torch.float64, device="cuda")
    p = css.CSS_FP64 if prec == "fp64" else css.CSS_MIXED_FP32
    r = ctx.hprime(Sd, Hd, torch.as_tensor(col, device="cuda"), torch.as_tensor(s, device="cuda"), nc, Si, Hp,
                   m=m, precision=p, flags=flags)
    tol = FP64_TOL if prec == "fp64" else MIXED_P_TOL
    scale = max(1.0, float(np.abs(ref["Hp"]).max()))
    assert float(np.abs(Si.cpu().numpy() - ref["Sinv"]).max()) < tol
    # mixed: Y is accumulated over m steps and H Y, S~^(-1/2) (H Y) are FP32 products; rounding
    # of 2^-24 per operation grows as sqrt(m b (S and H neighbours)) ~ sqrt(10 * 23 * 50), i.e.
    # about 6e-6 relative to the entries of H'
    htol = FP64_TOL if prec == "fp64" else 5e-6
    assert float(np.abs(Hp.cpu().numpy() - ref["Hp"]).max()) < htol * scale
    assert abs(r["trHp"] - ref["trHp"]) < htol * scale * H.n_brow * H.b


# ------------------------------------------------------------------ batch / pbuild
def test_batch_equals_single(torch, css, ctx):
    systems = [_system(n, "minimal", 10.0) for n in (27, 64, 100)]
    Hs, cols, signs, ncs, Ps, fs, singles = [], [], [], [], [], [], []
    for g, H, col, s, nc in systems:
        Hs.append(css.DeviceBSR.from_host(H))
        cols.append(torch.as_tensor(col, device="cuda"))
        signs.append(torch.as_tensor(s, device="cuda"))
        ncs.append(nc)
        Ps.append(torch.empty((H.nnzb, H.b, H.b), dtype=torch.float64, device="cuda"))
        fs.append({"kT": 0.05, "n_elec": synth.n_electrons(g.n_mol), "solve_mu": True})
        singles.append(gpu_density(torch, css, ctx, H, col, s, nc, kT=0.05, n_elec=synth.n_electrons(g.n_mol), m=8))
    r = ctx.density_batch(Hs, cols, signs, ncs, Ps, fs, m=8)
    torch.cuda.synchronize()
    for i, one in enumerate(singles):
        assert np.abs(Ps[i].cpu().numpy() - one["P"]).max() < 1e-12
        assert abs(r["mu"][i] - one["mu"]) < 1e-9
        assert abs(r["trP"][i] - one["trP"]) < 1e-9


def test_pbuild_host_buffers_equal_device_path(torch, css, ctx):
    g = synth.water_box(125)
    H = synth.hamiltonian(g)
    P_host = np.zeros((H.nnzb, H.b, H.b))
    col_host = np.zeros(125, np.int32)
    r = ctx.pbuild(g.pos, g.box, H, P_host, r_col=8.0, kT=0.05, n_elec=1000.0, m=10,
                   flags=css.CSS_SYMMETRIZE | css.CSS_HOST_IO, colour_out=col_host)
    col, nc = oracle.color(g.pos, g.box, 8.0, 1004)
    assert np.array_equal(col_host, col) and r["n_colours"] == nc
    s = oracle.probes(col, H.b, 1005)
    ref = oracle.density(H, col, s, nc, kT=0.05, n_elec=1000.0, m=10)
    assert np.abs(P_host - ref["P"]).max() < FP64_TOL


# --------------------------------------------------------------------- errors
def test_invalid_arguments_are_reported(torch, css, ctx):
    g, H, col, s, nc = _system(27, "minimal", 6.0)
    with pytest.raises(css.CSSError) as e:
        gpu_density(torch, css, ctx, H, col, s, nc, m=0)
    assert e.value.status == css.CSS_ERR_INVALID_ARG
    bad = synth.BSR(H.n_brow, H.b, H.row_ptr.copy(), H.col_idx.copy(), H.val.copy())
    bad.col_idx[1] = (bad.col_idx[1] + 5) % H.n_brow  # breaks the symmetric pattern
    with pytest.raises(css.CSSError):
        gpu_density(torch, css, ctx, bad, col, s, nc, m=4)
    with pytest.raises(css.CSSError):
        gpu_density(torch, css, ctx, H, np.full_like(col, nc + 1), s, nc, m=4)
