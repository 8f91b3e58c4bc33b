"""Checks of the seeded workload generator (inputs only, no method arithmetic)."""
import numpy as np
import pytest

from paper_2605_20918_gb300 import synth


def test_box_sides_of_the_workloads():
    assert abs(synth.box_side(64) - 12.42) < 1e-12
    assert abs(synth.box_side(4096) - 49.68) < 0.01
    assert abs(synth.box_side(10000) - 66.9) < 0.05
    assert abs(synth.box_side(1_000_000) - 310.5) < 0.5


@pytest.mark.parametrize("n", [1, 8, 64, 100])
def test_lattice_and_jitter(n):
    g = synth.water_box(n)
    assert g.pos.shape == (n, 3)
    n_s = int(np.ceil(round(n ** (1 / 3), 9)))
    a = g.box / n_s
    site = np.round(g.pos / a - 0.5)
    assert np.abs(g.pos - (site + 0.5) * a).max() <= 0.4 + 1e-12
    assert len({tuple(s) for s in site.astype(int)}) == n
    assert np.allclose(np.linalg.norm(g.orient, axis=1), 1.0)
    assert np.array_equal(g.pos, synth.water_box(n).pos)


@pytest.mark.parametrize("kind,b", [("minimal", 6), ("dzp", 23)])
def test_hamiltonian_structure(kind, b):
    g = synth.water_box(64)
    H = synth.hamiltonian(g, kind)
    assert H.b == b and H.n_brow == 64
    rows = H.rows()
    for i in range(H.n_brow):
        cols = H.col_idx[H.row_ptr[i]:H.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0) and i in cols
    pos = {(int(r), int(c)): k for k, (r, c) in enumerate(zip(rows, H.col_idx))}
    for (r, c), k in pos.items():
        assert np.array_equal(H.val[k], H.val[pos[(c, r)]].T)
    lv = synth.onsite_levels(64, kind)
    for i in range(64):
        w = np.linalg.eigvalsh(H.val[pos[(i, i)]])
        assert np.abs(w - np.sort(lv[i])).max() < 1e-11
    if kind == "dzp":
        assert np.all((lv[:, :4] >= -25) & (lv[:, :4] < -10)) and np.all((lv[:, 4:] >= 2) & (lv[:, 4:] < 30))


def test_coupling_law_and_cutoff():
    g = synth.water_box(216)
    H = synth.hamiltonian(g)
    rows = H.rows()
    d = g.pos[rows] - g.pos[H.col_idx]
    d -= g.box * np.round(d / g.box)
    r = np.linalg.norm(d, axis=1)
    off = rows != H.col_idx
    assert r[off].max() <= 6.0 and r[off].min() > 1.0
    # the coupling blocks' RMS follows t(r) / sqrt(b) * sqrt(b) / b ... i.e. |G| entries ~ N(0, 1/b)
    t = 0.5 * np.exp(-(r[off] - 2.8) / 0.5)
    G = H.val[off] / t[:, None, None]
    assert abs(G.std() - 1 / np.sqrt(6)) < 0.01 and abs(G.mean()) < 0.01
    # every pair within 6 A (brute force) is present
    n = g.n_mol
    dd = g.pos[:, None, :] - g.pos[None, :, :]
    dd -= g.box * np.round(dd / g.box)
    rr = np.linalg.norm(dd, axis=2)
    want = int(((rr <= 6.0) & ~np.eye(n, dtype=bool)).sum())
    assert int(off.sum()) == want


def test_zero_coupling_is_block_diagonal():
    g = synth.water_box(27)
    H = synth.hamiltonian(g, coupling=0.0)
    rows = H.rows()
    assert np.abs(H.val[rows != H.col_idx]).max() == 0.0


def test_pair_keyed_couplings_survive_perturbation():
    seq = list(synth.md_sequence(64, 3))
    assert len(seq) == 3
    d = seq[1].pos - seq[0].pos
    assert 0.015 < d.std() < 0.025
    H0 = synth.hamiltonian(seq[0]); H1 = synth.hamiltonian(seq[1])
    r0 = H0.rows(); r1 = H1.rows()
    k0 = {(int(a), int(c)): k for k, (a, c) in enumerate(zip(r0, H0.col_idx)) if a < c}
    k1 = {(int(a), int(c)): k for k, (a, c) in enumerate(zip(r1, H1.col_idx)) if a < c}
    common = sorted(set(k0) & set(k1))
    assert len(common) > 0.9 * len(k0)
    for p in common[:50]:
        a, b = H0.val[k0[p]], H1.val[k1[p]]
        ratio = a / b
        assert np.allclose(ratio, ratio.flat[0], rtol=1e-10)  # same G, rescaled by t(r)


def test_cell_list_equals_brute_force():
    g = synth.water_box(729)
    i1, j1, r1 = synth._pairs_within(g.pos, g.box, 6.0)
    n = g.n_mol
    dd = g.pos[:, None, :] - g.pos[None, :, :]
    dd -= g.box * np.round(dd / g.box)
    rr = np.linalg.norm(dd, axis=2)
    ii, jj = np.nonzero((rr <= 6.0) & (np.arange(n)[:, None] < np.arange(n)[None, :]))
    assert np.array_equal(i1, ii) and np.array_equal(j1, jj)


def test_log_uniform_sizes():
    s = synth.log_uniform_sizes(32)
    assert s.shape == (32,) and s.min() >= 200 and s.max() <= 5000
    assert np.array_equal(s, synth.log_uniform_sizes(32))
