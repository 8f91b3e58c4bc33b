"""Dense ground truth for tiny systems, from LAPACK (numpy.linalg.eigh) and scipy's brentq.

Independent of both the oracle and the CUDA library: f(H) is formed from the full
eigen-decomposition of the dense H, and the CSS projection rho~ = f(H) |r><r| (paper,
Eq. 2) is taken literally with explicit dense probe vectors.
"""
from __future__ import annotations

import numpy as np
import scipy.optimize as so


def fermi(x, mu, kT):
    x = np.asarray(x, dtype=np.float64)
    if kT > 0:
        return 0.5 * (1.0 - np.tanh((x - mu) / (2.0 * kT)))
    return np.where(x < mu, 1.0, np.where(x > mu, 0.0, 0.5))


def probe_matrix(colour, sign, b, n_colours):
    """Dense probe vectors: column (c, k) = +-1 on orbital k of every molecule of colour c."""
    n_mol = len(colour)
    R = np.zeros((n_mol * b, n_colours * b))
    for J in range(n_mol):
        for k in range(b):
            R[J * b + k, colour[J] * b + k] = sign[J * b + k]
    return R


class Dense:
    def __init__(self, H):
        self.H = H
        self.D = H.dense()
        self.w, self.V = np.linalg.eigh(self.D)

    def f(self, mu, kT):
        return (self.V * fermi(self.w, mu, kT)) @ self.V.T

    def inv_sqrt(self):
        """S^(-1/2) of a symmetric positive definite matrix."""
        assert self.w.min() > 0
        return (self.V / np.sqrt(self.w)) @ self.V.T

    def extract(self, M, colour, sign, n_colours):
        """(M R)[I, colour(J) block] diag(s_J) on the pattern for a dense matrix function M."""
        H = self.H
        b = H.b
        R = probe_matrix(colour, sign, b, n_colours)
        X = M @ R
        rows = H.rows()
        out = np.empty((H.nnzb, b, b))
        for k in range(H.nnzb):
            I, J = rows[k], H.col_idx[k]
            c = colour[J]
            out[k] = X[I * b:(I + 1) * b, c * b:(c + 1) * b] * sign[J * b:(J + 1) * b][None, :]
        return out

    def fe(self, mu, kT):
        """Energy-weighted density matrix sum_i f(e_i) e_i |psi_i><psi_i| = f(H) H."""
        return (self.V * (self.w * fermi(self.w, mu, kT))) @ self.V.T

    @staticmethod
    def _mid_of_tolerance_set(g, lo, hi, ne_tol):
        """Midpoint of {mu : |g(mu)| <= ne_tol} for increasing g (both ends by brentq)."""
        a = so.brentq(lambda m: g(m) + ne_tol, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
        z = so.brentq(lambda m: g(m) - ne_tol, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
        return 0.5 * (a + z)

    def mu_exact(self, n_elec, kT, ne_tol=None):
        """mu with Tr f(H) = N_e / 2 (midpoint of the set matching it within ne_tol)."""
        tol = 1e-4 * max(1.0, 0.5 * n_elec) if ne_tol is None else ne_tol
        return self._mid_of_tolerance_set(lambda m: fermi(self.w, m, kT).sum() - 0.5 * n_elec,
                                          self.w.min() - 5, self.w.max() + 5, tol)

    def mu_projected(self, R, n_elec, kT, n_colours, b, ne_tol=None):
        """mu for the quadrature sum_c tr(R_c^T f(H) R_c) = N_e / 2 the CSS method solves."""
        A = self.V.T @ R                         # eigenbasis components of every probe column
        wts = (A * A).sum(axis=1)                # sum over all probe columns
        tol = 1e-4 * max(1.0, 0.5 * n_elec) if ne_tol is None else ne_tol
        return self._mid_of_tolerance_set(lambda m: (fermi(self.w, m, kT) * wts).sum() - 0.5 * n_elec,
                                          self.w.min() - 5, self.w.max() + 5, tol)

    def on_pattern(self, M):
        """Blocks of a dense N x N matrix on H's pattern, (nnzb, b, b)."""
        H = self.H
        b = H.b
        rows = H.rows()
        out = np.empty((H.nnzb, b, b))
        for k in range(H.nnzb):
            I, J = rows[k], H.col_idx[k]
            out[k] = M[I * b:(I + 1) * b, J * b:(J + 1) * b]
        return out

    def css_extract(self, mu, kT, colour, sign, n_colours, energy=False):
        """P~_IJ = (f(H) R)[I, colour(J) block] diag(s_J) on the pattern (Eq. 2); with energy,
        the same extraction of f(H) H R."""
        H = self.H
        b = H.b
        R = probe_matrix(colour, sign, b, n_colours)
        X = (self.fe(mu, kT) if energy else self.f(mu, kT)) @ R
        rows = H.rows()
        out = np.empty((H.nnzb, b, b))
        for k in range(H.nnzb):
            I, J = rows[k], H.col_idx[k]
            c = colour[J]
            out[k] = X[I * b:(I + 1) * b, c * b:(c + 1) * b] * sign[J * b:(J + 1) * b][None, :]
        return out


def symmetrize(H, Pt):
    """(P~ + P~^T) / 2 on a structurally symmetric pattern."""
    rows = H.rows()
    pos = {(int(rows[k]), int(H.col_idx[k])): k for k in range(H.nnzb)}
    out = np.empty_like(Pt)
    for k in range(H.nnzb):
        q = pos[(int(H.col_idx[k]), int(rows[k]))]
        out[k] = 0.5 * (Pt[k] + Pt[q].T)
    return out
