"""Pins of the CPU oracle against things other than itself (no GPU needed).

Each test fixes part of the oracle with a published value, a closed form, LAPACK on a dense
matrix, brute force on a tiny input or an invariant of the method, chosen so that a dropped
term, a wrong sign or index, or a transposed operand in the oracle fails at least one.
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest

from paper_2605_20918_gb300 import synth
from tests.dense_truth import Dense, fermi, probe_matrix, symmetrize

GOLDEN = Path(__file__).resolve().parent / "golden"


@pytest.fixture(scope="module")
def O(oracle_lib):
    return oracle_lib


# ------------------------------------------------------------------ hash and probes
def test_splitmix64_published_outputs(O):
    g = json.loads((GOLDEN / "splitmix64.json").read_text())
    got = [O.hash64(g["seed"], i) for i in range(len(g["outputs"]))]
    assert got == [int(x) for x in g["outputs"]]


def test_probe_signs_and_structure(O):
    g = synth.water_box(64)
    col, nc = O.color(g.pos, g.box, 8.0, 1004)
    b = 6
    s = O.probes(col, b, 1005)
    assert set(np.unique(s)) == {-1, 1}
    frac = (s == -1).mean()
    assert abs(frac - 0.5) < 4 * math.sqrt(0.25 / s.size)
    R = probe_matrix(col, s, b, nc)
    counts = np.bincount(col, minlength=nc)
    # R_c^T R_c = |c| I and probe blocks of different colours are orthogonal
    assert np.array_equal(R.T @ R, np.diag(np.repeat(counts, b)).astype(float))
    # every orbital sits in exactly one probe column
    assert np.array_equal((R != 0).sum(axis=1), np.ones(64 * b))
    ones = O.probes(col, b, 1005, flags=O.SIGNS_ONES)
    assert np.all(ones == 1)
    assert np.array_equal(O.probes(col, b, 1005), s)
    assert not np.array_equal(O.probes(col, b, 1006), s)


# ------------------------------------------------------------------- colouring
def _min_image_dist(p, q, L):
    d = p - q
    d -= L * np.round(d / L)
    return float(np.sqrt((d * d).sum()))


def test_neighbours_match_float_distances(O):
    rng = np.random.default_rng(7)
    L, R = 20.0, 6.5
    x = rng.uniform(-3, 23, size=(120, 3))
    ptr, adj = O.neighbours(x, L, R)
    for i in range(len(x)):
        mine = set(adj[ptr[i]:ptr[i + 1]].tolist())
        for j in range(len(x)):
            if i == j:
                continue
            d = _min_image_dist(x[i], x[j], L)
            if abs(d - R) < 1e-5:
                continue
            assert (j in mine) == (d < R), (i, j, d)


def test_neighbours_strict_cutoff_fixed_point(O):
    # exactly R apart (representable in 2^-20 A) is NOT an edge; a hair closer is
    x = np.array([[1.0, 1.0, 1.0], [9.0, 1.0, 1.0], [1.0, 1.0, 8.999999]])
    ptr, adj = O.neighbours(x, 100.0, 8.0)
    assert adj[ptr[0]:ptr[1]].tolist() == [2]
    # minimum image across the boundary
    y = np.array([[0.5, 0.5, 0.5], [9.5, 0.5, 0.5]])
    ptr, adj = O.neighbours(y, 10.0, 1.5)
    assert adj.tolist() == [1, 0]


def _check_greedy(O, ptr, adj, col, seed):
    n = len(ptr) - 1
    deg = np.diff(ptr)
    key = [O.hash64(seed, i) for i in range(n)]
    prio = lambda v: (int(deg[v]), key[v], -v)  # larger = earlier
    for v in range(n):
        nb = adj[ptr[v]:ptr[v + 1]]
        assert all(col[u] != col[v] for u in nb), "monochromatic edge"
        higher = [u for u in nb if prio(u) > prio(v)]
        hc = {int(col[u]) for u in higher}
        # greedy in priority order <=> every smaller colour is taken by a higher-priority neighbour
        assert all(c in hc for c in range(int(col[v]))), (v, col[v], hc)


def _random_graph(n, p, rng):
    A = np.triu(rng.random((n, n)) < p, 1)
    A = A | A.T
    ptr = np.concatenate([[0], np.cumsum(A.sum(1))]).astype(np.int32)
    adj = np.concatenate([np.nonzero(A[i])[0] for i in range(n)]).astype(np.int32)
    return ptr, adj


@pytest.mark.parametrize("n,p", [(1, 0.0), (10, 0.0), (30, 0.2), (60, 0.5), (40, 1.0)])
def test_greedy_colouring_characterisation(O, n, p):
    rng = np.random.default_rng(n)
    ptr, adj = _random_graph(n, p, rng)
    col, nc = O.color_graph(ptr, adj, 1004)
    assert nc == (col.max() + 1 if n else 0)
    _check_greedy(O, ptr, adj, col, 1004)
    if p == 1.0:
        assert nc == n
    if p == 0.0:
        assert nc == 1


def test_hand_checked_graphs(O):
    # star K_{1,5}: hub (degree 5) first -> colour 0, leaves -> colour 1
    ptr = np.array([0, 5, 6, 7, 8, 9, 10], np.int32)
    adj = np.array([1, 2, 3, 4, 5, 0, 0, 0, 0, 0], np.int32)
    col, nc = O.color_graph(ptr, adj, 99)
    assert col.tolist() == [0, 1, 1, 1, 1, 1] and nc == 2
    # complete bipartite K_{3,5}: the degree-5 side is coloured first and takes colour 0
    A = np.zeros((8, 8), bool)
    A[:3, 3:] = True
    A = A | A.T
    ptr = np.concatenate([[0], np.cumsum(A.sum(1))]).astype(np.int32)
    adj = np.concatenate([np.nonzero(A[i])[0] for i in range(8)]).astype(np.int32)
    col, nc = O.color_graph(ptr, adj, 5)
    assert col.tolist() == [0, 0, 0, 1, 1, 1, 1, 1] and nc == 2


def test_lattice_colouring_valid_and_greedy(O):
    g = synth.water_box(216)
    ptr, adj = O.neighbours(g.pos, g.box, 8.0)
    col, nc = O.color(g.pos, g.box, 8.0, 1004)
    _check_greedy(O, ptr, adj, col, 1004)
    col2, _ = O.color(g.pos, g.box, 8.0, 1004)
    assert np.array_equal(col, col2)


# --------------------------------------------------- colouring kept across MD steps
def _pair_dists(x, L, pairs):
    d = x[pairs[:, 0]] - x[pairs[:, 1]]
    d -= L * np.round(d / L)
    return np.sqrt((d * d).sum(1))


def test_conflicts_match_periodic_kdtree(O):
    """Same-coloured pairs closer than R_col on displaced geometries, counted independently
    with scipy's periodic k-d tree on float distances (no pair lies within 1e-5 A of the
    cut-off in these geometries, so float and fixed point agree on every pair)."""
    spatial = pytest.importorskip("scipy.spatial")
    R = 8.0
    g0 = synth.water_box(400)
    col, nc = O.color(g0.pos, g0.box, R, 1004)
    counts = []
    for sigma, seed in [(0.0, 0), (0.05, 3001), (0.3, 3002), (1.0, 3006)]:
        g = synth.perturb(g0, seed, sigma=sigma) if sigma else g0
        x = np.mod(g.pos, g.box)
        pairs = spatial.cKDTree(x, boxsize=g.box).query_pairs(R + 1e-5, output_type="ndarray")
        d = _pair_dists(x, g.box, pairs)
        assert not np.any(np.abs(d - R) < 1e-5)
        want = int(((col[pairs[:, 0]] == col[pairs[:, 1]]) & (d < R)).sum())
        assert O.color_conflicts(g.pos, g.box, R, col) == want
        counts.append(want)
    # the colouring is valid on its own geometry and breaks as the displacements grow
    assert counts[0] == 0 and counts[-1] > counts[1]


def test_conflicts_brute_force_tiny(O):
    rng = np.random.default_rng(11)
    L, R, n = 15.0, 5.0, 40
    x = rng.uniform(-2.0, L + 2.0, size=(n, 3))
    d = np.array([[_min_image_dist(x[i], x[j], L) for j in range(n)] for i in range(n)])
    iu = np.triu_indices(n, 1)
    assert not np.any(np.abs(d[iu] - R) < 1e-5)
    col = rng.integers(0, 4, size=n).astype(np.int32)
    want = sum(1 for i in range(n) for j in range(i + 1, n) if col[i] == col[j] and d[i, j] < R)
    assert O.color_conflicts(x, L, R, col) == want
    # one colour: every edge of the colour graph is a conflict; all colours distinct: none
    assert O.color_conflicts(x, L, R, np.zeros(n, np.int32)) == int((d[iu] < R).sum())
    assert O.color_conflicts(x, L, R, np.arange(n, dtype=np.int32)) == 0
    # R = 0: no pair is closer than 0
    assert O.color_conflicts(x, L, 0.0, np.zeros(n, np.int32)) == 0


def test_conflicts_strict_cutoff_and_minimum_image(O):
    same = np.zeros(3, np.int32)
    x = np.array([[1.0, 1.0, 1.0], [9.0, 1.0, 1.0], [1.0, 1.0, 8.999999]])
    assert O.color_conflicts(x, 100.0, 8.0, same) == 1  # only (0, 2); (0, 1) is exactly R apart
    y = np.array([[0.5, 0.5, 0.5], [9.5, 0.5, 0.5]])
    assert O.color_conflicts(y, 10.0, 1.5, same[:2]) == 1  # 1 A apart across the boundary
    assert O.color_conflicts(y, 10.0, 1.5, np.array([0, 1], np.int32)) == 0


def test_color_update_keeps_valid_colourings(O):
    R = 8.0
    g0 = synth.water_box(216)
    col, nc = O.color(g0.pos, g0.box, R, 1004)
    # a small displacement that keeps the colouring valid: kept as it is
    g1 = synth.perturb(g0, 3100, sigma=0.001)
    assert O.color_conflicts(g1.pos, g1.box, R, col) == 0
    c1, n1, re1 = O.color_update(g1.pos, g1.box, R, 1004, col, nc)
    assert not re1 and n1 == nc and np.array_equal(c1, col)
    # a large one breaks it: recoloured from scratch, exactly as a fresh colouring
    g2 = synth.perturb(g0, 3101, sigma=1.0)
    assert O.color_conflicts(g2.pos, g2.box, R, col) > 0
    c2, n2, re2 = O.color_update(g2.pos, g2.box, R, 1004, col, nc)
    fresh, nf = O.color(g2.pos, g2.box, R, 1004)
    assert re2 and n2 == nf and np.array_equal(c2, fresh)
    # no colouring yet (n_colours = 0) or colours out of range: recoloured
    fresh1, nf1 = O.color(g1.pos, g1.box, R, 1004)
    for bad_col, bad_nc in [(col, 0), (col, int(col.max())), (col - 1, nc)]:
        c3, n3, re3 = O.color_update(g1.pos, g1.box, R, 1004, bad_col, bad_nc)
        assert re3 and n3 == nf1 and np.array_equal(c3, fresh1)


def test_color_update_with_a_skin(O):
    """Recolouring at R_col + skin leaves room to move: on an MD-like walk of 0.02 A steps the
    skinned colouring stays conflict-free at R_col for several steps, while a colouring at
    R_col itself has conflicts after the first step (greedy colourings pack same-coloured
    molecules just outside the cut-off)."""
    R, skin = 8.0, 0.3
    seq = list(synth.md_sequence(400, 6))
    tight, _ = O.color(seq[0].pos, seq[0].box, R, 1004)
    assert O.color_conflicts(seq[1].pos, seq[1].box, R, tight) > 0
    col, nc, re = O.color_update(seq[0].pos, seq[0].box, R, 1004, np.zeros(400, np.int32), 0, skin=skin)
    fresh, nf = O.color(seq[0].pos, seq[0].box, R + skin, 1004)
    assert re and nc == nf and np.array_equal(col, fresh)
    # a colouring at the larger radius is valid at the smaller one
    assert O.color_conflicts(seq[0].pos, seq[0].box, R + skin, col) == 0
    for g in seq[1:]:
        c2, n2, re2 = O.color_update(g.pos, g.box, R, 1004, col, nc, skin=skin)
        assert not re2 and n2 == nc and np.array_equal(c2, col)


# ------------------------------------------------------------------- eigensolver
@pytest.mark.parametrize("n", [1, 2, 3, 17, 120])
def test_eigh_against_lapack(O, n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    A = A + A.T
    w, U = O.eigh(A)
    ref = np.linalg.eigvalsh(A)
    scale = max(1.0, abs(ref).max())
    assert np.abs(w - ref).max() <= 1e-13 * scale * n
    assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-13 * n
    assert np.abs(U @ np.diag(w) @ U.T - A).max() <= 1e-13 * scale * n


def test_eigh_degenerate_and_banded(O):
    # repeated eigenvalues
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    lam = np.repeat([-3.0, 1.0, 2.5, 7.0], 10)
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    w, U = O.eigh(A)
    assert np.abs(w - np.sort(lam)).max() < 1e-12
    assert np.abs(U @ np.diag(w) @ U.T - A).max() < 1e-12
    # diagonal input (already reduced)
    d = np.array([3.0, -1.0, 2.0])
    w, U = O.eigh(np.diag(d))
    assert np.array_equal(w, np.sort(d))


# --------------------------------------------------------------------- Lanczos
def test_block_lanczos_definition(O):
    g = synth.water_box(27)
    H = synth.hamiltonian(g)
    col, nc = O.color(g.pos, g.box, 6.0, 1004)
    s = O.probes(col, H.b, 1005)
    c = int(col[0])
    m = 5
    T, Q = O.lanczos(H, col, s, c, m, want_q=True)
    D = H.dense()
    n = T.shape[0]
    assert n == m * H.b
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-12           # orthonormal basis
    assert np.abs(Q.T @ D @ Q - T).max() < 1e-11               # projected Hamiltonian
    R = probe_matrix(col, s, H.b, nc)[:, c * H.b:(c + 1) * H.b]
    cnt = (col == c).sum()
    assert np.abs(Q[:, :H.b] - R / math.sqrt(cnt)).max() < 1e-15
    b = H.b
    for j in range(m - 1):                                      # block tridiagonal, B_j upper, diag >= 0
        Bj = T[(j + 1) * b:(j + 2) * b, j * b:(j + 1) * b]
        assert np.abs(np.tril(Bj, -1)).max() == 0.0
        assert np.all(np.diag(Bj) > 0)
        if j + 2 < m:
            assert np.abs(T[(j + 2) * b:, j * b:(j + 1) * b]).max() == 0.0
    # span: the Krylov blocks [R, HR, H^2 R, ...] lie in range(Q)
    K = [R]
    for _ in range(m - 1):
        K.append(D @ K[-1])
    K = np.concatenate(K, axis=1)
    resid = K - Q @ (Q.T @ K)
    assert np.linalg.norm(resid) / np.linalg.norm(K) < 1e-9


def test_ritz_weights_sum_to_probe_norm(O):
    g = synth.water_box(64)
    H = synth.hamiltonian(g)
    col, nc = O.color(g.pos, g.box, 8.0, 1004)
    s = O.probes(col, H.b, 1005)
    rz = O.ritz(H, col, s, nc, m=6)
    cnt = np.bincount(col, minlength=nc)
    for c, (lam, w) in enumerate(rz):
        assert abs(w.sum() - H.b * cnt[c]) < 1e-11 * H.b * cnt[c]
        assert np.all(np.diff(lam) >= 0)


# --------------------------------------------------------------------- density
def _pattern_err(A, B):
    return float(np.abs(A - B).max())


def test_degenerate_colouring_full_krylov_is_f_of_H(O):
    """Every molecule its own colour and m b >= N: P equals f(H) on the pattern."""
    g = synth.water_box(8)
    H = synth.hamiltonian(g)
    col, nc = O.color(g.pos, g.box, 100.0, 1004)
    assert nc == 8
    s = O.probes(col, H.b, 1005)
    ne = synth.n_electrons(8)
    r = O.density(H, col, s, nc, kT=0.05, n_elec=ne, m=8)
    dn = Dense(H)
    mu = dn.mu_exact(ne, 0.05)
    assert _pattern_err(r["P"], dn.on_pattern(dn.f(mu, 0.05))) < 1e-10
    assert abs(r["trP"] - ne / 2) <= 1e-4 * ne / 2


def test_contaminated_projection_full_krylov(O):
    """Shared colours and a Krylov space that spans everything: P~ = extract(f(H) R) (Eq. 2)."""
    g = synth.water_box(12, box=9.0)
    H = synth.hamiltonian(g, r_cut=5.0)
    col, nc = O.color(g.pos, g.box, 4.0, 1004)
    assert nc < 12
    s = O.probes(col, H.b, 1005)
    ne = synth.n_electrons(12)
    dn = Dense(H)
    R = probe_matrix(col, s, H.b, nc)
    mu = dn.mu_projected(R, ne, 0.05, nc, H.b)
    Pt = dn.css_extract(mu, 0.05, col, s, nc)
    r = O.density(H, col, s, nc, kT=0.05, n_elec=ne, m=12, flags=0)
    assert _pattern_err(r["P"], Pt) < 1e-10
    r2 = O.density(H, col, s, nc, kT=0.05, n_elec=ne, m=12)
    assert _pattern_err(r2["P"], symmetrize(H, Pt)) < 1e-10
    # symmetrisation leaves the traces unchanged
    assert abs(r["trP"] - r2["trP"]) < 1e-10 and abs(r["trPH"] - r2["trPH"]) < 1e-9
    # the traces against the dense truth
    assert abs(r["trP"] - ne / 2) <= 1e-4 * ne / 2
    assert abs(r2["trPH"] - float((Pt * H.val).sum())) < 1e-9


def test_fixed_mu_matches_dense(O):
    g = synth.water_box(12, box=9.0)
    H = synth.hamiltonian(g, r_cut=5.0)
    col, nc = O.color(g.pos, g.box, 4.0, 1004)
    s = O.probes(col, H.b, 1005)
    dn = Dense(H)
    for mu, kT in [(-4.0, 0.05), (-10.5, 0.3), (1.7, 0.5)]:
        r = O.density(H, col, s, nc, mu=mu, kT=kT, solve_mu=False, m=12, flags=0)
        assert _pattern_err(r["P"], dn.css_extract(mu, kT, col, s, nc)) < 1e-10
        assert r["mu"] == mu


def test_zero_coupling_blocks(O):
    """Block-diagonal H: P_II = U f(D) U^T exactly and no off-diagonal density."""
    g = synth.water_box(27)
    H = synth.hamiltonian(g, coupling=0.0)
    col, nc = O.color(g.pos, g.box, 6.0, 1004)
    s = O.probes(col, H.b, 1005)
    ne = synth.n_electrons(27)
    r = O.density(H, col, s, nc, kT=0.05, n_elec=ne, m=10)
    assert r["n_breakdown"] > 0
    rows = H.rows()
    for k in range(H.nnzb):
        I, J = rows[k], H.col_idx[k]
        if I == J:
            w, V = np.linalg.eigh(H.val[k])
            ref = (V * fermi(w, r["mu"], 0.05)) @ V.T
            assert np.abs(r["P"][k] - ref).max() < 1e-11
        else:
            assert np.abs(r["P"][k]).max() < 1e-11
    assert abs(r["trP"] - ne / 2) <= 1e-4 * ne / 2


def test_single_molecule(O):
    g = synth.water_box(1)
    H = synth.hamiltonian(g, "dzp")
    col = np.zeros(1, np.int32)
    s = O.probes(col, H.b, 1005)
    r = O.density(H, col, s, 1, kT=0.05, n_elec=8.0, m=3)
    w, V = np.linalg.eigh(H.val[0])
    mu = r["mu"]
    assert np.abs(r["P"][0] - (V * fermi(w, mu, 0.05)) @ V.T).max() < 1e-11
    assert abs(r["trP"] - 4.0) <= 4e-6
    # the single molecule has a gap between levels 4 and 5: mu is its midpoint
    lv = np.sort(w)
    assert abs(mu - 0.5 * (lv[3] + lv[4])) < 0.3 * (lv[4] - lv[3])


def test_two_level_closed_form(O):
    """b = 1, two coupled sites: f(H) from the closed-form 2x2 eigen-decomposition."""
    a, d, t = -1.3, 0.4, 0.7
    H = synth.BSR(n_brow=2, b=1, row_ptr=np.array([0, 2, 4], np.int32), col_idx=np.array([0, 1, 0, 1], np.int32),
                  val=np.array([a, t, t, d], dtype=float).reshape(4, 1, 1))
    col = np.array([0, 1], np.int32)
    s = np.array([1, -1], np.int8)
    mu, kT = -0.2, 0.25
    r = O.density(H, col, s, 2, mu=mu, kT=kT, solve_mu=False, m=2)
    h = math.sqrt(((a - d) / 2) ** 2 + t * t)
    lp, lm = (a + d) / 2 + h, (a + d) / 2 - h
    vp = np.array([t, lp - a]); vp /= np.linalg.norm(vp)
    vm = np.array([t, lm - a]); vm /= np.linalg.norm(vm)
    fp = 1.0 / (1.0 + math.exp((lp - mu) / kT))
    fm = 1.0 / (1.0 + math.exp((lm - mu) / kT))
    F = fp * np.outer(vp, vp) + fm * np.outer(vm, vm)
    assert np.abs(r["P"].ravel() - F.ravel()).max() < 1e-14
    assert abs(r["trP"] - (fp + fm)) < 1e-14
    assert abs(r["trPH"] - (lp * fp + lm * fm)) < 1e-14


def test_trace_identity_and_bisection(O):
    """Tr of the unsymmetrised extraction equals the Ritz quadrature sum_j f w (Eq. 6-7)."""
    g = synth.water_box(64)
    H = synth.hamiltonian(g)
    col, nc = O.color(g.pos, g.box, 8.0, 1004)
    s = O.probes(col, H.b, 1005)
    ne = synth.n_electrons(64)
    r = O.density(H, col, s, nc, kT=0.05, n_elec=ne, m=6, flags=0)
    rz = O.ritz(H, col, s, nc, m=6)
    quad = sum(float((fermi(l, r["mu"], 0.05) * w).sum()) for l, w in rz)
    assert abs(r["trP"] - quad) < 1e-9
    assert abs(quad - ne / 2) <= 1e-4 * ne / 2 * (1 + 1e-9)


def test_idempotent_as_kT_vanishes(O):
    g = synth.water_box(8)
    H = synth.hamiltonian(g)
    col, nc = O.color(g.pos, g.box, 100.0, 1004)
    s = O.probes(col, H.b, 1005)
    r = O.density(H, col, s, nc, kT=1e-3, n_elec=64.0, m=8)
    dn = Dense(H)
    P = np.zeros_like(dn.D)
    b = H.b
    rows = H.rows()
    for k in range(H.nnzb):
        P[rows[k] * b:(rows[k] + 1) * b, H.col_idx[k] * b:(H.col_idx[k] + 1) * b] = r["P"][k]
    assert H.nnzb == 64  # the tiny box couples every pair: P is the full matrix
    assert np.abs(P @ P - P).max() < 1e-10
    assert np.abs(P - P.T).max() == 0.0


def test_convergence_in_krylov_depth(O):
    g = synth.water_box(64)
    H = synth.hamiltonian(g)
    col, nc = O.color(g.pos, g.box, 8.0, 1004)
    s = O.probes(col, H.b, 1005)
    dn = Dense(H)
    mu = -4.0
    ref = dn.css_extract(mu, 0.05, col, s, nc)
    errs = [_pattern_err(O.density(H, col, s, nc, mu=mu, kT=0.05, solve_mu=False, m=m, flags=0)["P"], ref)
            for m in (2, 4, 8, 16, 24, 40)]
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-9


def test_decay_with_distance(O):
    """|P_IJ| decays with the molecule distance (nearsightedness behind Eq. 2)."""
    g = synth.water_box(216)
    H = synth.hamiltonian(g)
    rows = H.rows()
    dist = np.array([_min_image_dist(g.pos[rows[k]], g.pos[H.col_idx[k]], g.box) for k in range(H.nnzb)])
    bins = [(2.0, 3.0), (3.0, 4.0), (4.0, 5.0), (5.0, 6.1)]
    for r_col, stat in [(8.0, np.median), (12.0, np.max)]:
        # at R_col = 8 A < 2 x 6 A same-colour contamination lifts single far blocks, so the
        # envelope is taken on the median; at 12 A the maximum itself decays
        col, nc = O.color(g.pos, g.box, r_col, 1004)
        s = O.probes(col, H.b, 1005)
        r = O.density(H, col, s, nc, kT=0.05, n_elec=synth.n_electrons(216), m=10)
        amax = np.abs(r["P"]).max(axis=(1, 2))
        env = [stat(amax[(dist >= lo) & (dist < hi)]) for lo, hi in bins]
        assert all(a > b for a, b in zip(env, env[1:])), (r_col, env)


def test_local_reorth_agrees(O):
    g = synth.water_box(64)
    H = synth.hamiltonian(g)
    col, nc = O.color(g.pos, g.box, 8.0, 1004)
    s = O.probes(col, H.b, 1005)
    a = O.density(H, col, s, nc, mu=-4.0, solve_mu=False, m=10, flags=0)
    b = O.density(H, col, s, nc, mu=-4.0, solve_mu=False, m=10, flags=O.REORTH_LOCAL)
    assert _pattern_err(a["P"], b["P"]) < 1e-9


def test_colour_subset_equals_full_columns(O):
    g = synth.water_box(64)
    H = synth.hamiltonian(g)
    col, nc = O.color(g.pos, g.box, 8.0, 1004)
    s = O.probes(col, H.b, 1005)
    full = O.density(H, col, s, nc, mu=-4.0, solve_mu=False, m=6, flags=0)
    sub = [1, 3]
    part = O.density(H, col, s, nc, mu=-4.0, solve_mu=False, m=6, flags=0, colour_subset=sub,
                     P_init=np.full((H.nnzb, H.b, H.b), np.nan))
    sel = np.isin(col[H.col_idx], sub)
    assert np.array_equal(part["P"][sel], full["P"][sel])
    assert np.all(np.isnan(part["P"][~sel]))


# -------------------------------------------- energy-weighted density matrix (paper, forces)
def test_energy_weighted_degenerate_colouring_is_f_of_H_times_H(O):
    """Every molecule its own colour and a full Krylov space: rho_E = f(H) H on the pattern,
    with mu fixed by f exactly as for P."""
    g = synth.water_box(8)
    H = synth.hamiltonian(g)
    col, nc = O.color(g.pos, g.box, 100.0, 1004)
    s = O.probes(col, H.b, 1005)
    ne = synth.n_electrons(8)
    r = O.density(H, col, s, nc, kT=0.05, n_elec=ne, m=8)
    re = O.density(H, col, s, nc, kT=0.05, n_elec=ne, m=8, flags=O.SYMMETRIZE | O.ENERGY_WEIGHTED)
    dn = Dense(H)
    mu = dn.mu_exact(ne, 0.05)
    assert re["mu"] == r["mu"]
    ref = dn.on_pattern(dn.fe(mu, 0.05))
    assert _pattern_err(re["P"], ref) < 1e-9
    # Tr rho_E = sum_i f(e_i) e_i
    assert abs(re["trP"] - float((dn.w * fermi(dn.w, mu, 0.05)).sum())) < 1e-8


def test_energy_weighted_contaminated_full_krylov(O):
    """Shared colours, full Krylov space: rho~_E = extract(f(H) H R) (Eq. 2 with f(x) x)."""
    g = synth.water_box(12, box=9.0)
    H = synth.hamiltonian(g, r_cut=5.0)
    col, nc = O.color(g.pos, g.box, 4.0, 1004)
    s = O.probes(col, H.b, 1005)
    ne = synth.n_electrons(12)
    dn = Dense(H)
    R = probe_matrix(col, s, H.b, nc)
    mu = dn.mu_projected(R, ne, 0.05, nc, H.b)
    re = O.density(H, col, s, nc, kT=0.05, n_elec=ne, m=12, flags=O.ENERGY_WEIGHTED)
    assert _pattern_err(re["P"], dn.css_extract(mu, 0.05, col, s, nc, energy=True)) < 1e-9
    rs = O.density(H, col, s, nc, kT=0.05, n_elec=ne, m=12, flags=O.ENERGY_WEIGHTED | O.SYMMETRIZE)
    assert _pattern_err(rs["P"], symmetrize(H, dn.css_extract(mu, 0.05, col, s, nc, energy=True))) < 1e-9


def test_energy_weighted_trace_identity_truncated(O):
    """With a truncated Krylov space the unsymmetrised trace is still the Ritz quadrature
    sum_j lambda_j f(lambda_j) w_j (Eq. 6-7)."""
    g = synth.water_box(64)
    H = synth.hamiltonian(g)
    col, nc = O.color(g.pos, g.box, 8.0, 1004)
    s = O.probes(col, H.b, 1005)
    ne = synth.n_electrons(64)
    re = O.density(H, col, s, nc, kT=0.05, n_elec=ne, m=6, flags=O.ENERGY_WEIGHTED)
    rz = O.ritz(H, col, s, nc, m=6)
    quad = sum(float((l * fermi(l, re["mu"], 0.05) * w).sum()) for l, w in rz)
    assert abs(re["trP"] - quad) < 1e-8 * max(1.0, abs(quad))


def test_energy_weighted_zero_coupling_blocks(O):
    """Block-diagonal H: (rho_E)_II = H_II f(H_II) and nothing off the diagonal."""
    g = synth.water_box(27)
    H = synth.hamiltonian(g, coupling=0.0)
    col, nc = O.color(g.pos, g.box, 6.0, 1004)
    s = O.probes(col, H.b, 1005)
    ne = synth.n_electrons(27)
    re = O.density(H, col, s, nc, kT=0.05, n_elec=ne, m=10, flags=O.SYMMETRIZE | O.ENERGY_WEIGHTED)
    rows = H.rows()
    for k in range(H.nnzb):
        I, J = rows[k], H.col_idx[k]
        if I == J:
            w, V = np.linalg.eigh(H.val[k])
            ref = (V * (w * fermi(w, re["mu"], 0.05))) @ V.T
            assert np.abs(re["P"][k] - ref).max() < 1e-10
        else:
            assert np.abs(re["P"][k]).max() < 1e-11


# ------------------------------------------- S^(-1/2) of an overlap matrix (paper, Eq. 8-10)
def test_inv_sqrt_degenerate_colouring_is_exact(O):
    """Every molecule its own colour and a full Krylov space: S~^(-1/2) = S^(-1/2) on the pattern."""
    g = synth.water_box(8)
    S = synth.overlap(g)
    col, nc = O.color(g.pos, g.box, 100.0, 1004)
    s = O.probes(col, S.b, 1005)
    r = O.density(S, col, s, nc, m=8, flags=O.SYMMETRIZE | O.INV_SQRT)
    dn = Dense(S)
    assert _pattern_err(r["P"], dn.on_pattern(dn.inv_sqrt())) < 1e-11
    assert abs(r["trP"] - float((1.0 / np.sqrt(dn.w)).sum())) < 1e-10


def test_inv_sqrt_contaminated_full_krylov(O):
    """Shared colours, full Krylov space: S~^(-1/2) = extract(S^(-1/2) o) (Eq. 8-9 taken literally)."""
    g = synth.water_box(12, box=9.0)
    S = synth.overlap(g)
    col, nc = O.color(g.pos, g.box, 4.0, 1004)
    assert nc < 12
    s = O.probes(col, S.b, 1005)
    dn = Dense(S)
    ref = dn.extract(dn.inv_sqrt(), col, s, nc)
    r = O.density(S, col, s, nc, m=12, flags=O.INV_SQRT)
    assert _pattern_err(r["P"], ref) < 1e-11
    r2 = O.density(S, col, s, nc, m=12, flags=O.INV_SQRT | O.SYMMETRIZE)
    assert _pattern_err(r2["P"], symmetrize(S, ref)) < 1e-11


def test_inv_sqrt_trace_identity_and_convergence(O):
    """Truncated Krylov space: Tr of the extraction is the Ritz quadrature sum_j lambda_j^(-1/2)
    w_j, and with a colouring radius beyond the overlap range the error against the dense
    S^(-1/2) falls with the Krylov depth (the paper uses 10)."""
    g = synth.water_box(64)
    S = synth.overlap(g)
    col, nc = O.color(g.pos, g.box, 9.0, 1004)
    s = O.probes(col, S.b, 1005)
    rz = O.ritz(S, col, s, nc, m=4)
    r = O.density(S, col, s, nc, m=4, flags=O.INV_SQRT)
    quad = sum(float((w / np.sqrt(l)).sum()) for l, w in rz)
    assert abs(r["trP"] - quad) < 1e-9
    dn = Dense(S)
    contaminated = symmetrize(S, dn.extract(dn.inv_sqrt(), col, s, nc))
    got = {m: O.density(S, col, s, nc, m=m, flags=O.INV_SQRT | O.SYMMETRIZE)["P"] for m in (2, 4, 8)}
    errs = [_pattern_err(got[m], contaminated) for m in (2, 4, 8)]   # Krylov truncation only
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] < 1e-8, errs
    # what is left against the true S^(-1/2) is the same-colour contamination (Eq. 2)
    assert _pattern_err(got[8], dn.on_pattern(dn.inv_sqrt())) < 1e-3


# ------------------------------------- H' of a non-orthogonal basis (paper, after Eq. 10)
def _block_mask(M):
    """Dense 0/1 mask of a BSR pattern."""
    b = M.b
    mask = np.zeros((M.n_brow * b, M.n_brow * b))
    rows = M.rows()
    for k in range(M.nnzb):
        I, J = rows[k], M.col_idx[k]
        mask[I * b:(I + 1) * b, J * b:(J + 1) * b] = 1.0
    return mask


def test_hprime_full_pattern_is_the_orthogonalised_H(O):
    """An overlap whose pattern covers every pair and molecules in their own colours: H' is
    S^(-1/2) H S^(-1/2) exactly, and its spectrum is the generalised spectrum of (H, S)."""
    g = synth.water_box(6, box=6.0)
    S = synth.overlap(g, r_cut=20.0)
    H = synth.hamiltonian(g, r_cut=20.0)
    col, nc = O.color(g.pos, g.box, 100.0, 1004)
    s = O.probes(col, S.b, 1005)
    r = O.hprime(S, H, col, s, nc, m=6)
    ds = Dense(S)
    Si = ds.inv_sqrt()
    ref = Si @ H.dense() @ Si
    assert _pattern_err(r["Sinv"], ds.on_pattern(Si)) < 1e-11
    assert _pattern_err(r["Hp"], Dense(H).on_pattern(ref)) < 1e-9
    import scipy.linalg as sl
    w = sl.eigh(H.dense(), S.dense(), eigvals_only=True)
    assert np.abs(np.linalg.eigvalsh(ref) - w).max() < 1e-9
    assert abs(r["trHp"] - np.trace(ref)) < 1e-9


def test_hprime_truncated_and_contaminated(O):
    """Shared colours, a truncated overlap pattern and a full Krylov space: H'~ is the literal
    extraction of trunc(S^(-1/2)) H (S^(-1/2) R) (the left factor is the sparse S~^(-1/2))."""
    g = synth.water_box(12, box=9.0)
    S = synth.overlap(g)
    H = synth.hamiltonian(g, r_cut=5.0)
    col, nc = O.color(g.pos, g.box, 4.0, 1004)
    assert nc < 12
    s = O.probes(col, S.b, 1005)
    r = O.hprime(S, H, col, s, nc, m=12, flags=0)
    ds, dh = Dense(S), Dense(H)
    R = probe_matrix(col, s, S.b, nc)
    Si = ds.inv_sqrt()
    Y = Si @ R
    Sinv_t = ds.extract(Si, col, s, nc)             # S~^(-1/2) on S's pattern (unsymmetrised)
    assert _pattern_err(r["Sinv"], Sinv_t) < 1e-11
    # dense S~^(-1/2) from its pattern blocks
    St = np.zeros_like(Si)
    rows = S.rows()
    b = S.b
    for k in range(S.nnzb):
        I, J = rows[k], S.col_idx[k]
        St[I * b:(I + 1) * b, J * b:(J + 1) * b] = Sinv_t[k]
    hrows = H.rows()

    def extract_h(Left):
        X = Left @ H.dense() @ Y
        out = np.empty((H.nnzb, b, b))
        for k in range(H.nnzb):
            I, J = hrows[k], H.col_idx[k]
            c = col[J]
            out[k] = X[I * b:(I + 1) * b, c * b:(c + 1) * b] * s[J * b:(J + 1) * b][None, :]
        return out

    assert _pattern_err(r["Hp"], extract_h(St)) < 1e-10
    # symmetrised: both S~^(-1/2) and H'~ are symmetrised on their patterns
    rs = O.hprime(S, H, col, s, nc, m=12)
    Sinv_s = symmetrize(S, Sinv_t)
    Ss = np.zeros_like(Si)
    for k in range(S.nnzb):
        I, J = rows[k], S.col_idx[k]
        Ss[I * b:(I + 1) * b, J * b:(J + 1) * b] = Sinv_s[k]
    assert _pattern_err(rs["Sinv"], Sinv_s) < 1e-11
    assert _pattern_err(rs["Hp"], symmetrize(H, extract_h(Ss))) < 1e-10


# ------------------------------------------ density matrix of a non-orthogonal basis
def _dense_from_blocks(M, vals):
    b = M.b
    out = np.zeros((M.n, M.n))
    rows = M.rows()
    for k in range(M.nnzb):
        I, J = rows[k], M.col_idx[k]
        out[I * b:(I + 1) * b, J * b:(J + 1) * b] = vals[k]
    return out


def _mid_tolerance_set(g, lo, hi, tol):
    import scipy.optimize as so
    a = so.brentq(lambda m: g(m) + tol, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    z = so.brentq(lambda m: g(m) - tol, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    return 0.5 * (a + z)


def test_nonorth_full_is_the_generalised_density(O):
    """Full overlap and Hamiltonian patterns, every molecule its own colour and full Krylov
    spaces: rho~ is the density matrix of the generalised problem H C = S C E, C^T S C = I,
    i.e. C f(E) C^T from scipy's generalised eigensolver; mu makes Tr(rho S) = sum f(e) equal
    N_e/2; Tr(rho H) = sum e f(e)."""
    import scipy.linalg as sl
    g = synth.water_box(6, box=6.0)
    S = synth.overlap(g, r_cut=20.0)
    H = synth.hamiltonian(g, r_cut=20.0)
    col, nc = O.color(g.pos, g.box, 100.0, 1004)
    s = O.probes(col, S.b, 1005)
    hp = O.hprime(S, H, col, s, nc, m=6)
    e, C = sl.eigh(H.dense(), S.dense())
    dh = Dense(H)
    kT, mu = 0.05, -5.0
    r = O.density_nonorth(S, hp["Sinv"], H, hp["Hp"], col, s, nc, mu=mu, kT=kT, solve_mu=False, m=6)
    rho = (C * fermi(e, mu, kT)) @ C.T
    assert _pattern_err(r["P"], dh.on_pattern(rho)) < 1e-9
    assert abs(r["trPS"] - fermi(e, mu, kT).sum()) < 1e-9
    assert abs(r["trPH"] - (e * fermi(e, mu, kT)).sum()) < 1e-8
    # mu solved on the electron count: the generalised spectrum's own mu (tolerance-set midpoint)
    ne = synth.n_electrons(6)
    tol = 1e-4 * 0.5 * ne
    mu_ref = _mid_tolerance_set(lambda m: fermi(e, m, kT).sum() - 0.5 * ne, e.min() - 5, e.max() + 5, tol)
    rs = O.density_nonorth(S, hp["Sinv"], H, hp["Hp"], col, s, nc, kT=kT, n_elec=ne, m=6)
    assert abs(rs["mu"] - mu_ref) < 1e-7
    assert _pattern_err(rs["P"], dh.on_pattern((C * fermi(e, rs["mu"], kT)) @ C.T)) < 1e-9
    assert abs(rs["trPS"] - 0.5 * ne) <= tol


def test_nonorth_contaminated_full_krylov(O):
    """Shared colours for the density probes, truncated overlap and Hamiltonian patterns and a
    full Krylov space of H': rho~ is the literal extraction of S~^(-1/2) f(H'~) S~^(-1/2) R, with
    S~^(-1/2) and H'~ the sparse matrices given as inputs.  (The overlap probes are one molecule
    per colour so that S~^(-1/2) stays well conditioned: with a heavily contaminated S~^(-1/2)
    the plain block-Lanczos loses orthogonality before the Krylov space is full.)"""
    g = synth.water_box(12, box=9.0)
    S = synth.overlap(g)
    H = synth.hamiltonian(g, r_cut=5.0)
    colS, ncS = O.color(g.pos, g.box, 100.0, 1004)
    sS = O.probes(colS, S.b, 1005)
    hp = O.hprime(S, H, colS, sS, ncS, m=12)
    col, nc = O.color(g.pos, g.box, 3.5, 2004)
    assert nc < 12
    s = O.probes(col, H.b, 2005)
    kT, mu = 0.05, -5.0
    r = O.density_nonorth(S, hp["Sinv"], H, hp["Hp"], col, s, nc, mu=mu, kT=kT, solve_mu=False, m=12, flags=0)
    Si = _dense_from_blocks(S, hp["Sinv"])
    Hp = _dense_from_blocks(H, hp["Hp"])
    w, V = np.linalg.eigh(Hp)
    R = probe_matrix(col, s, H.b, nc)
    X = Si @ ((V * fermi(w, mu, kT)) @ V.T) @ (Si @ R)
    b, rows = H.b, H.rows()
    want = np.empty((H.nnzb, b, b))
    for k in range(H.nnzb):
        I, J = rows[k], H.col_idx[k]
        c = col[J]
        want[k] = X[I * b:(I + 1) * b, c * b:(c + 1) * b] * s[J * b:(J + 1) * b][None, :]
    assert _pattern_err(r["P"], want) < 1e-10
    rsym = O.density_nonorth(S, hp["Sinv"], H, hp["Hp"], col, s, nc, mu=mu, kT=kT, solve_mu=False, m=12)
    assert _pattern_err(rsym["P"], symmetrize(H, want)) < 1e-10
    assert abs(r["trPH"] - float((want * H.val).sum())) < 1e-9


@pytest.mark.parametrize("m,hp_flags", [(2, 1), (4, 1), (3, 0)])
def test_nonorth_electron_count_identity(O, m, hp_flags):
    """Truncated Krylov spaces and shared colours: the kappa quadrature the chemical potential
    is solved on equals the extracted Tr(rho~ S), so at the solved mu the density matrix
    (symmetrised or not) holds N_e/2 electrons in the Mulliken count sum_IJ <rho_IJ, S_IJ>,
    taken here from the returned blocks.  hp_flags = 0 gives an unsymmetrised S~^(-1/2), for
    which the weights need its transpose."""
    g = synth.water_box(27)
    S = synth.overlap(g)
    H = synth.hamiltonian(g)
    colS, ncS = O.color(g.pos, g.box, 6.0, 1004)
    sS = O.probes(colS, S.b, 1005)
    hp = O.hprime(S, H, colS, sS, ncS, m=6, flags=hp_flags)
    if hp_flags == 0:
        Si = _dense_from_blocks(S, hp["Sinv"])
        assert np.abs(Si - Si.T).max() > 1e-6
    col, nc = O.color(g.pos, g.box, 5.0, 2004)
    s = O.probes(col, H.b, 2005)
    ne = synth.n_electrons(27)
    hpos = {(int(I), int(J)): k for k, (I, J) in enumerate(zip(H.rows(), H.col_idx))}
    for flags in (0, O.SYMMETRIZE):
        r = O.density_nonorth(S, hp["Sinv"], H, hp["Hp"], col, s, nc, kT=0.05, n_elec=ne, m=m, flags=flags)
        mulliken = sum(float((r["P"][hpos[(int(I), int(J))]] * S.val[k]).sum())
                       for k, (I, J) in enumerate(zip(S.rows(), S.col_idx)))
        assert abs(mulliken - 0.5 * ne) <= 1e-4 * 0.5 * ne + 1e-9, (flags, mulliken)
        assert abs(r["trPS"] - mulliken) < 1e-9


def test_nonorth_identity_overlap_is_the_orthogonal_density(O):
    """S = I (so S~^(-1/2) = I and H' = H): the start blocks are the probe blocks themselves,
    the electron-count weights are the Ritz weights, and the result is the orthogonal CSS
    density matrix, mu included."""
    g = synth.water_box(27)
    H = synth.hamiltonian(g)
    n, b = H.n_brow, H.b
    eye = synth.BSR(n, b, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
                    np.broadcast_to(np.eye(b), (n, b, b)).copy())
    col, nc = O.color(g.pos, g.box, 5.0, 2004)
    s = O.probes(col, b, 2005)
    ne = synth.n_electrons(27)
    for kw in ({"mu": -5.0, "solve_mu": False}, {"n_elec": ne}):
        r = O.density_nonorth(eye, eye.val, H, H.val, col, s, nc, kT=0.05, m=5, **kw)
        ref = O.density(H, col, s, nc, kT=0.05, m=5, **kw)
        assert _pattern_err(r["P"], ref["P"]) < 1e-11
        assert abs(r["mu"] - ref["mu"]) < 1e-9 and abs(r["trPH"] - ref["trPH"]) < 1e-9
        assert abs(r["trPS"] - ref["trP"]) < 1e-9


# ------------------------------------------------ mu from Ritz lists gathered across ranks
def test_solve_mu_on_ritz_lists_is_the_density_rule(O):
    g = synth.water_box(64)
    H = synth.hamiltonian(g, "minimal")
    col, nc = O.color(g.pos, g.box, 8.0, 1004)
    s = O.probes(col, H.b, 1005)
    ne = synth.n_electrons(64)
    ref = O.density(H, col, s, nc, kT=0.05, n_elec=ne, m=10)
    full = O.ritz(H, col, s, nc, 10)
    assert O.solve_mu(full, 0.05, ne) == ref["mu"]
    # the colour mask returns exactly the chosen colours' lists
    sub = O.ritz(H, col, s, nc, 10, colours=[1, 3])
    for c in range(nc):
        if c in (1, 3):
            assert np.array_equal(sub[c][0], full[c][0]) and np.array_equal(sub[c][1], full[c][1])
        else:
            assert sub[c][0].size == 0


def test_nonorth_idempotent_in_the_overlap_metric(O):
    """Full patterns, one molecule per colour, full Krylov spaces and a small kT: the density
    matrix of the non-orthogonal basis is a projector in the S metric, rho S rho = rho, and
    holds N_e/2 electrons in Tr(rho S)."""
    g = synth.water_box(6, box=6.0)
    S = synth.overlap(g, r_cut=20.0)
    H = synth.hamiltonian(g, r_cut=20.0)
    col, nc = O.color(g.pos, g.box, 100.0, 1004)
    s = O.probes(col, S.b, 1005)
    hp = O.hprime(S, H, col, s, nc, m=6)
    ne = synth.n_electrons(6)
    r = O.density_nonorth(S, hp["Sinv"], H, hp["Hp"], col, s, nc, kT=1e-3, n_elec=ne, m=6)
    rho = _dense_from_blocks(H, r["P"])
    Sd = S.dense()
    assert np.abs(rho @ Sd @ rho - rho).max() < 1e-9
    assert abs(np.trace(rho @ Sd) - 0.5 * ne) < 1e-9
    assert abs(r["trPS"] - 0.5 * ne) < 1e-9


# ------------------------------------------------ mu of an insulator with spurious gap weight
def test_mu_is_mid_gap_between_band_edges_despite_spurious_gap_weight(O):
    """A truncated, contaminated Krylov quadrature leaves a thin spread of Ritz weight inside the
    gap (measured at 10,000 molecules, m = 40: 1,349 values carrying 0.18 electrons, about
    4.5e-6 N_e/2).  Closed form at kT = 0: with N_e/2 electrons' worth of weight below the band
    edge e_v, none between the edges except a spread of total weight below ne_tol, and a band
    starting at e_c, the set {mu : |N(mu) - N_e/2| <= ne_tol} is [e_v, e_c], so mu = (e_v + e_c)/2
    whatever the spread looks like.  The default ne_tol (1e-4 N_e/2) must exceed such a spread;
    with 1e-6 N_e/2 the ends fall inside it and mu moves with it."""
    rng = np.random.default_rng(7)
    half_ne = 4000.0
    e_v, e_c = -9.75, 1.5
    occ = np.concatenate([rng.uniform(-25.0, e_v, 999), [e_v]])
    virt = np.concatenate([[e_c], rng.uniform(e_c, 30.0, 2999)])
    w_occ = np.full(occ.size, half_ne / occ.size)
    w_virt = np.full(virt.size, 3.0 * half_ne / virt.size)
    for total in (0.0, 0.02, 0.2):
        ghosts = rng.uniform(e_v + 0.01, e_c - 0.01, 500)
        wg = np.full(ghosts.size, total / ghosts.size)
        lists = [(np.concatenate([occ, ghosts[:250], virt[:1500]]), np.concatenate([w_occ, wg[:250], w_virt[:1500]])),
                 (np.concatenate([ghosts[250:], virt[1500:]]), np.concatenate([wg[250:], w_virt[1500:]]))]
        mu = O.solve_mu(lists, 0.0, 2.0 * half_ne)
        assert abs(mu - 0.5 * (e_v + e_c)) < 1e-11, (total, mu)
        if total > 1e-6 * half_ne:  # the narrower set of the former default lands inside the spread
            mu6 = O.solve_mu(lists, 0.0, 2.0 * half_ne, ne_tol=1e-6 * half_ne)
            assert abs(mu6 - 0.5 * (e_v + e_c)) > 0.1, (total, mu6)
