"""GPU exact-diagonalisation stage (paper, Eq. 7) against LAPACK (numpy.linalg.eigh).

The projected matrices are block tridiagonal with upper-triangular sub-diagonal blocks, the
structure block-Lanczos produces.  Eigenvalues are compared directly; the weights through
their cumulative sums (they are unique only up to rotations inside degenerate eigenspaces),
and Z = U f(Lambda) U^T E_1 sqrt|c|, which is basis-invariant, element by element.
"""
import numpy as np
import pytest

import oracle
from paper_2605_20918_gb300 import synth
from tests.dense_truth import fermi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    import paper_2605_20918_gb300 as css
    from paper_2605_20918_gb300 import build
    build.build()
    c = css.Context(0)
    yield c
    c.close()


def dense_T(A, B, nb):
    b = A.shape[-1]
    n = nb * b
    T = np.zeros((n, n))
    for j in range(nb):
        T[j * b:(j + 1) * b, j * b:(j + 1) * b] = A[j]
        if j + 1 < nb:
            T[(j + 1) * b:(j + 2) * b, j * b:(j + 1) * b] = B[j]
            T[j * b:(j + 1) * b, (j + 1) * b:(j + 2) * b] = B[j].T
    return T


def random_blocks(rng, n_col, m, b, scale=10.0):
    A = rng.standard_normal((n_col, m, b, b)) * scale
    A = 0.5 * (A + np.swapaxes(A, -1, -2))
    B = np.triu(rng.standard_normal((n_col, m, b, b)))
    d = np.abs(np.diagonal(B, axis1=-2, axis2=-1)) + 0.1
    idx = np.arange(b)
    B[..., idx, idx] = d
    return A, B


def check(torch, ctx, A, B, nblk, cnt, mu, kT, tol=1e-10):
    n_col, m, b, _ = A.shape
    dev = "cuda"
    lam, wgt, Z = ctx.eigen_blocks(torch.as_tensor(A, device=dev), torch.as_tensor(B, device=dev),
                                   torch.as_tensor(nblk.astype(np.int32), device=dev),
                                   torch.as_tensor(cnt.astype(np.int32), device=dev), mu=mu, kT=kT)
    lam, wgt, Z = lam.cpu().numpy(), wgt.cpu().numpy(), Z.cpu().numpy()
    for c in range(n_col):
        n = nblk[c] * b
        T = dense_T(A[c], B[c], nblk[c])
        w, V = np.linalg.eigh(T)
        scale = max(1.0, np.abs(w).max())
        got = np.sort(lam[c, :n])
        assert np.abs(got - w).max() <= tol * scale, (c, np.abs(got - w).max())
        wref = cnt[c] * (V[:b, :] ** 2).sum(axis=0)
        assert abs(wgt[c, :n].sum() - b * cnt[c]) <= 1e-10 * b * cnt[c]
        o = np.argsort(lam[c, :n])
        cum_got = np.cumsum(wgt[c, :n][o])
        cum_ref = np.cumsum(wref)
        # compare at gaps of the spectrum (where the cumulative weight is basis-invariant)
        gaps = np.nonzero(np.diff(w) > 1e-6 * scale)[0]
        assert np.abs(cum_got[gaps] - cum_ref[gaps]).max() <= 1e-9 * b * cnt[c]
        E = np.zeros((n, b))
        E[:b, :b] = np.sqrt(cnt[c]) * np.eye(b)
        Zref = (V * fermi(w, mu, kT)) @ (V.T @ E)
        assert np.abs(Z[c, :n] - Zref).max() <= tol * np.sqrt(cnt[c]) * 10, (c, np.abs(Z[c, :n] - Zref).max())
        if n < Z.shape[1]:
            assert np.abs(Z[c, n:]).max() == 0.0


@pytest.mark.parametrize("b,m", [(1, 8), (2, 5), (6, 30), (7, 13), (23, 8), (23, 40), (32, 4)])
def test_random_block_tridiagonal(torch, ctx, b, m):
    rng = np.random.default_rng(b * 100 + m)
    n_col = 5
    A, B = random_blocks(rng, n_col, m, b)
    nblk = np.full(n_col, m)
    nblk[1] = max(1, m // 2)            # a truncated (breakdown) colour
    cnt = rng.integers(1, 50, n_col)
    check(torch, ctx, A, B, nblk, cnt, mu=0.3, kT=0.5)


def test_exactly_degenerate_spectrum(torch, ctx):
    """B = 0 and equal diagonal blocks: every eigenvalue is m-fold degenerate."""
    rng = np.random.default_rng(3)
    b, m = 6, 10
    a = rng.standard_normal((b, b))
    a = a + a.T
    A = np.broadcast_to(a, (2, m, b, b)).copy()
    B = np.zeros((2, m, b, b))
    check(torch, ctx, A, B, np.array([m, m]), np.array([3, 4]), mu=0.0, kT=0.2)


def _oracle_blocks(n_mol, cols, m=40, b=23):
    g = synth.water_box(n_mol)
    H = synth.hamiltonian(g, "dzp")
    col, nc = oracle.color(g.pos, g.box, 10.0, 1004)
    s = oracle.probes(col, b, 1005)
    cols = [c % nc for c in cols]
    A = np.zeros((len(cols), m, b, b))
    B = np.zeros((len(cols), m, b, b))
    nblk = np.zeros(len(cols), np.int64)
    for i, c in enumerate(cols):
        T = oracle.lanczos(H, col, s, c, m)
        nb = T.shape[0] // b
        nblk[i] = nb
        for j in range(nb):
            A[i, j] = T[j * b:(j + 1) * b, j * b:(j + 1) * b]
            if j + 1 < nb:
                B[i, j] = T[(j + 1) * b:(j + 2) * b, j * b:(j + 1) * b]
    return A, B, nblk, np.bincount(col, minlength=nc)[cols]


def test_projected_matrices_from_the_oracle(torch, ctx):
    """Real projected matrices (23 orbitals, m = 40) from the oracle's block-Lanczos."""
    A, B, nblk, cnt = _oracle_blocks(343, [0, 30, 59])
    check(torch, ctx, A, B, nblk, cnt, mu=-4.0, kT=0.05)


def test_start_vector_robustness(torch, ctx):
    """The same projected matrices repeated over many colours: every copy starts its inverse
    iterations from different vectors and must still find every eigenpair."""
    A, B, nblk, cnt = _oracle_blocks(512, [0, 10, 38])
    rep = 40
    check(torch, ctx, np.tile(A, (rep, 1, 1, 1)), np.tile(B, (rep, 1, 1, 1)), np.tile(nblk, rep), np.tile(cnt, rep),
          mu=-4.0, kT=0.05)
