"""Seeded synthetic water-like workloads for the CSS density-matrix path.

This module makes inputs only.  It holds no step of the CSS method: no colouring, no probe,
no Lanczos, no matrix function.  Both the CUDA library and the CPU oracle receive what it
produces, so it is the one piece of code the two sides share.

Workload recipe (orthogonal tight-binding stand-in for the paper's DFTB water, where a
molecule carries b orbitals and the basis is orthogonal, S = I):

* Positions: a jittered simple-cubic lattice in a periodic cubic box of side
  L = 12.42 A * (n_mol / 64)^(1/3).  With n_s = ceil(n_mol^(1/3)) sites per edge at
  (i + 1/2) * L / n_s; when n_s^3 > n_mol a seeded subset of n_mol sites is kept (in
  lattice order).  Every coordinate gets a uniform jitter in [-0.4, +0.4) A.  Orientations
  (unit quaternions) are drawn too, as the workload names them, though H does not use them.
* On-site blocks: H_II = U_I diag(levels_I) U_I^T with U_I Haar-orthogonal (QR of a
  Gaussian matrix with the sign of diag(R) folded in).  "minimal" (b = 6) levels are
  (-20, -15, -13, -11, +2, +5) eV; "dzp" (b = 23) levels are 4 occupied uniform in
  [-25, -10] eV and 19 virtual uniform in [+2, +30] eV, drawn per molecule.
* Couplings: every pair with minimum-image O-O distance r <= r_cut (6 A) gets
  H_IJ = t(r) G_IJ with t(r) = 0.5 eV * exp(-(r - 2.8) / 0.5) for I < J and H_JI = H_IJ^T.
  G_IJ has N(0, 1) / sqrt(b) entries drawn from a counter keyed by the unordered pair,
  so a pair keeps its G across a molecular-dynamics-like sequence of geometries.
* MD-like sequence: geometry t >= 1 is geometry t-1 plus Gaussian displacements of
  sigma = 0.02 A per coordinate, keyed by seed 2000 + t.

Random numbers come from a counter-based hash (the MurmurHash3 64-bit finaliser of Appleby,
used as a mixing function) so that any element can be drawn on its own and results do
not depend on chunking.  Seeds default to positions 1001, on-site 1002, couplings 1003.

H is returned in block-sparse-row (BSR) form: row_ptr[n_mol + 1], col_idx[nnzb] (sorted
within a row, diagonal present, pattern symmetric), val[nnzb, b, b] row-major, float64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Geometry", "BSR", "water_box", "perturb", "md_sequence", "hamiltonian", "onsite_levels",
    "system", "n_electrons", "box_side", "log_uniform_sizes",
]

_U64 = np.uint64
_MASK = (1 << 64) - 1

# purposes: independent streams under one seed
_P_SITES, _P_JITTER, _P_ORIENT, _P_LEVELS, _P_UMAT, _P_COUPLING, _P_DISPLACE, _P_SIZES = range(1, 9)


def _fmix64(x: np.ndarray) -> np.ndarray:
    """MurmurHash3 fmix64 finaliser on a uint64 array (wrapping arithmetic)."""
    x = x ^ (x >> _U64(33))
    x = x * _U64(0xFF51AFD7ED558CCD)
    x = x ^ (x >> _U64(33))
    x = x * _U64(0xC4CEB9FE1A85EC53)
    x = x ^ (x >> _U64(33))
    return x


def _key(seed: int, purpose: int) -> np.uint64:
    k = _fmix64(np.array([(seed * 0x9E3779B97F4A7C15 + purpose * 0x632BE59BD9B4E019) & _MASK],
                         dtype=_U64))
    return k[0]


def _bits(seed: int, purpose: int, idx: np.ndarray) -> np.ndarray:
    idx = np.asarray(idx, dtype=_U64)
    return _fmix64(idx * _U64(0xD1B54A32D192ED03) + _key(seed, purpose))


def _uniform(seed: int, purpose: int, idx: np.ndarray) -> np.ndarray:
    """Uniform in [0, 1) with 53 random bits."""
    return (_bits(seed, purpose, idx) >> _U64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _normal(seed: int, purpose: int, idx: np.ndarray) -> np.ndarray:
    """Standard normal per counter via Box-Muller on two hashed uniforms."""
    idx = np.asarray(idx, dtype=_U64)
    u1 = 1.0 - _uniform(seed, purpose, idx * _U64(2))          # (0, 1]
    u2 = _uniform(seed, purpose, idx * _U64(2) + _U64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


@dataclass
class Geometry:
    """Molecule centres (O positions) in a periodic cubic box, in Angstrom."""
    pos: np.ndarray            # (n_mol, 3) float64
    box: float                 # cubic box side L
    orient: np.ndarray | None = None  # (n_mol, 4) unit quaternions (not used by H)

    @property
    def n_mol(self) -> int:
        return int(self.pos.shape[0])


@dataclass
class BSR:
    """Block-sparse-row symmetric matrix with b x b float64 blocks."""
    n_brow: int
    b: int
    row_ptr: np.ndarray        # int32 [n_brow + 1]
    col_idx: np.ndarray        # int32 [nnzb]
    val: np.ndarray            # float64 [nnzb, b, b]
    meta: dict = field(default_factory=dict)

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def n(self) -> int:
        return self.n_brow * self.b

    def dense(self) -> np.ndarray:
        """Dense copy (for tiny test systems only)."""
        n, b = self.n, self.b
        out = np.zeros((n, n))
        for i in range(self.n_brow):
            for k in range(self.row_ptr[i], self.row_ptr[i + 1]):
                j = self.col_idx[k]
                out[i * b:(i + 1) * b, j * b:(j + 1) * b] = self.val[k]
        return out

    def rows(self) -> np.ndarray:
        """Block-row index of every stored block."""
        return np.repeat(np.arange(self.n_brow, dtype=np.int32), np.diff(self.row_ptr))


def box_side(n_mol: int) -> float:
    """Box side for n_mol water-like molecules at the 64-molecule density (12.42 A)."""
    return 12.42 * (n_mol / 64.0) ** (1.0 / 3.0)


def n_electrons(n_mol: int) -> float:
    """Valence electrons: 8 per water molecule."""
    return 8.0 * n_mol


def water_box(n_mol: int, seed: int = 1001, jitter: float = 0.4, box: float | None = None) -> Geometry:
    """Jittered cubic lattice of n_mol molecule centres in a periodic box."""
    if n_mol < 1:
        raise ValueError("n_mol must be >= 1")
    L = box_side(n_mol) if box is None else float(box)
    n_s = 1
    while n_s ** 3 < n_mol:
        n_s += 1
    a = L / n_s
    sites = np.arange(n_s ** 3, dtype=np.int64)
    if n_s ** 3 > n_mol:
        keys = _bits(seed, _P_SITES, sites)
        keep = np.sort(np.argsort(keys, kind="stable")[:n_mol])
        sites = sites[keep]
    ijk = np.stack([sites // (n_s * n_s), (sites // n_s) % n_s, sites % n_s], axis=1).astype(np.float64)
    pos = (ijk + 0.5) * a
    mol = np.arange(n_mol, dtype=np.int64)
    ctr = (mol[:, None] * 3 + np.arange(3)[None, :]).ravel()
    pos = pos + ((2.0 * _uniform(seed, _P_JITTER, ctr) - 1.0) * jitter).reshape(n_mol, 3)
    q = _normal(seed, _P_ORIENT, (mol[:, None] * 4 + np.arange(4)[None, :]).ravel()).reshape(n_mol, 4)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return Geometry(pos=pos, box=L, orient=q)


def perturb(geom: Geometry, seed: int, sigma: float = 0.02) -> Geometry:
    """Next geometry of an MD-like sequence: Gaussian displacements of width sigma."""
    n = geom.n_mol
    ctr = (np.arange(n, dtype=np.int64)[:, None] * 3 + np.arange(3)[None, :]).ravel()
    d = _normal(seed, _P_DISPLACE, ctr).reshape(n, 3) * sigma
    return Geometry(pos=geom.pos + d, box=geom.box, orient=geom.orient)


def md_sequence(n_mol: int, n_steps: int, seed: int = 1001, sigma: float = 0.02, first_seed: int = 2000):
    """Yield n_steps geometries; geometry t >= 1 is geometry t-1 displaced with seed first_seed + t."""
    g = water_box(n_mol, seed=seed)
    yield g
    for t in range(1, n_steps):
        g = perturb(g, seed=first_seed + t, sigma=sigma)
        yield g


def onsite_levels(n_mol: int, kind: str, seed: int = 1002) -> np.ndarray:
    """Per-molecule on-site spectra, (n_mol, b)."""
    if kind == "minimal":
        lv = np.array([-20.0, -15.0, -13.0, -11.0, 2.0, 5.0])
        return np.broadcast_to(lv, (n_mol, 6)).copy()
    if kind == "dzp":
        mol = np.arange(n_mol, dtype=np.int64)
        ctr = (mol[:, None] * 23 + np.arange(23)[None, :]).ravel()
        u = _uniform(seed, _P_LEVELS, ctr).reshape(n_mol, 23)
        occ = -25.0 + 15.0 * u[:, :4]
        virt = 2.0 + 28.0 * u[:, 4:]
        return np.concatenate([occ, virt], axis=1)
    raise ValueError(f"unknown level kind {kind!r}")


def _haar_orthogonal(n_mol: int, b: int, seed: int) -> np.ndarray:
    mol = np.arange(n_mol, dtype=np.int64)
    ctr = (mol[:, None] * (b * b) + np.arange(b * b)[None, :]).ravel()
    z = _normal(seed, _P_UMAT, ctr).reshape(n_mol, b, b)
    q, r = np.linalg.qr(z)
    s = np.sign(np.diagonal(r, axis1=1, axis2=2))
    s[s == 0] = 1.0
    return q * s[:, None, :]


def _min_image(d: np.ndarray, L: float) -> np.ndarray:
    return d - L * np.round(d / L)


def _pairs_within(pos: np.ndarray, L: float, rc: float):
    """All unordered pairs i < j with minimum-image distance <= rc; returns (i, j, r)."""
    n = pos.shape[0]
    nc = int(math.floor(L / rc))
    out_i, out_j, out_r = [], [], []
    if nc < 3 or n < 64:
        chunk = max(1, int(2_000_000 // max(n, 1)))
        for s in range(0, n, chunk):
            ii = np.arange(s, min(n, s + chunk))
            d = _min_image(pos[ii, None, :] - pos[None, :, :], L)
            r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
            a, bb = np.nonzero((r <= rc) & (ii[:, None] < np.arange(n)[None, :]))
            out_i.append(ii[a]); out_j.append(bb); out_r.append(r[a, bb])
    else:
        w = L / nc
        wrapped = pos - L * np.floor(pos / L)
        c = np.minimum((wrapped / w).astype(np.int64), nc - 1)
        cid = (c[:, 0] * nc + c[:, 1]) * nc + c[:, 2]
        order = np.argsort(cid, kind="stable")
        counts = np.bincount(cid, minlength=nc ** 3)
        start = np.concatenate([[0], np.cumsum(counts)])
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    nb = (((c[:, 0] + dx) % nc) * nc + (c[:, 1] + dy) % nc) * nc + (c[:, 2] + dz) % nc
                    cnt = counts[nb]
                    tot = int(cnt.sum())
                    if tot == 0:
                        continue
                    ii = np.repeat(np.arange(n), cnt)
                    off = np.arange(tot) - np.repeat(np.cumsum(cnt) - cnt, cnt)
                    jj = order[start[nb][ii] + off]
                    keep = ii < jj
                    ii, jj = ii[keep], jj[keep]
                    d = _min_image(pos[ii] - pos[jj], L)
                    r = np.sqrt(np.einsum("ij,ij->i", d, d))
                    m = r <= rc
                    out_i.append(ii[m]); out_j.append(jj[m]); out_r.append(r[m])
    if not out_i:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0)
    i = np.concatenate(out_i); j = np.concatenate(out_j); r = np.concatenate(out_r)
    o = np.lexsort((j, i))
    return i[o].astype(np.int64), j[o].astype(np.int64), r[o]


def _coupling_G(pi, pj, n, b, coupling_seed, pair_chunk):
    """Unscaled coupling blocks G of the pairs (pi < pj), keyed by the unordered pair."""
    bb = b * b
    out = np.empty((pi.shape[0], b, b))
    for s in range(0, pi.shape[0], pair_chunk):
        e = min(pi.shape[0], s + pair_chunk)
        key = pi[s:e].astype(np.uint64) * _U64(n) + pj[s:e].astype(np.uint64)
        ctr = (key[:, None] * _U64(bb) + np.arange(bb, dtype=np.uint64)[None, :]).ravel()
        out[s:e] = _normal(coupling_seed, _P_COUPLING, ctr).reshape(e - s, b, b) / math.sqrt(b)
    return out


def overlap(geom: Geometry, kind: str = "minimal", *, r_cut: float = 4.5, coupling: float = 0.05,
            overlap_seed: int = 1007, cache: dict | None = None) -> BSR:
    """Synthetic overlap S of a non-orthogonal basis (symmetric positive definite, BSR): unit
    on-site blocks and couplings coupling * exp(-(r - 2.8)/0.5) * G for O-O distance r <= r_cut,
    G drawn per unordered pair (seed `overlap_seed`) with N(0,1)/sqrt(b) entries.  With the
    defaults the off-diagonal row sums stay well below 1 at water density, so S is positive
    definite with a condition number of about 2."""
    b = 6 if kind == "minimal" else 23 if kind == "dzp" else None
    if b is None:
        raise ValueError(f"unknown level kind {kind!r}")
    return hamiltonian(geom, kind, r_cut=r_cut, coupling=coupling, levels=np.ones((geom.n_mol, b)),
                       coupling_seed=overlap_seed, cache=cache)


def hamiltonian(geom: Geometry, kind: str = "minimal", *, r_cut: float = 6.0, coupling: float = 0.5,
                levels: np.ndarray | None = None, onsite_seed: int = 1002, coupling_seed: int = 1003,
                pair_chunk: int = 200_000, cache: dict | None = None) -> BSR:
    """Orthogonal water-like tight-binding H in BSR form.

    kind: "minimal" (b = 6) or "dzp" (b = 23); `levels` (n_mol, b) overrides the spectra and
    then fixes b.  coupling = 0 gives a block-diagonal H.  `cache` (a dict kept by the caller
    across the geometries of one sequence) keeps the on-site blocks and the pair-keyed G
    blocks, which do not depend on the positions, so only new pairs are drawn.
    """
    n = geom.n_mol
    lv = onsite_levels(n, kind, onsite_seed) if levels is None else np.asarray(levels, dtype=np.float64)
    if lv.shape[0] != n:
        raise ValueError("levels must have one row per molecule")
    b = lv.shape[1]
    ckey = (n, b, kind, onsite_seed, coupling_seed, None if levels is None else lv.tobytes())
    if cache is not None and cache.get("key") != ckey:
        cache.clear()
        cache["key"] = ckey
    if cache is not None and "diag" in cache:
        diag = cache["diag"]
    else:
        U = _haar_orthogonal(n, b, onsite_seed)
        diag = np.einsum("nik,nk,njk->nij", U, lv, U)
        diag = 0.5 * (diag + np.transpose(diag, (0, 2, 1)))
        if cache is not None:
            cache["diag"] = diag

    pi, pj, pr = _pairs_within(geom.pos, geom.box, r_cut)
    npair = pi.shape[0]
    rows = np.concatenate([pi, pj, np.arange(n)])
    cols = np.concatenate([pj, pi, np.arange(n)])
    order = np.lexsort((cols, rows))
    nnzb = rows.shape[0]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    val = np.empty((nnzb, b, b), dtype=np.float64)
    inv = np.empty(nnzb, dtype=np.int64)
    inv[order] = np.arange(nnzb)
    # diagonal blocks
    val[inv[2 * npair:]] = diag
    # coupling blocks t(r) G, G drawn per unordered pair (or taken from the cache)
    t = coupling * np.exp(-(pr - 2.8) / 0.5)
    if cache is None:
        G = _coupling_G(pi, pj, n, b, coupling_seed, pair_chunk)
    else:
        keys = pi.astype(np.uint64) * _U64(n) + pj.astype(np.uint64)
        ck = cache.get("gkeys", np.zeros(0, np.uint64))
        cv = cache.get("gvals", np.zeros((0, b, b)))
        pos = np.searchsorted(ck, keys)
        hit = (pos < ck.shape[0]) & (ck[np.minimum(pos, max(ck.shape[0] - 1, 0))] == keys) if ck.shape[0] else \
            np.zeros(keys.shape[0], bool)
        G = np.empty((npair, b, b))
        G[hit] = cv[pos[hit]]
        miss = ~hit
        if miss.any():
            G[miss] = _coupling_G(pi[miss], pj[miss], n, b, coupling_seed, pair_chunk)
            allk = np.concatenate([ck, keys[miss]])
            allv = np.concatenate([cv, G[miss]])
            o = np.argsort(allk, kind="stable")
            cache["gkeys"], cache["gvals"] = allk[o], allv[o]
    blk = G * t[:, None, None]
    val[inv[:npair]] = blk
    val[inv[npair:2 * npair]] = np.transpose(blk, (0, 2, 1))
    col_idx = cols[order].astype(np.int32)
    return BSR(n_brow=n, b=b, row_ptr=row_ptr.astype(np.int32), col_idx=col_idx, val=val,
               meta={"n_pairs": int(npair), "r_cut": r_cut, "box": geom.box, "kind": kind})


def system(n_mol: int, kind: str = "minimal", seed: int = 1001, **kw):
    """Geometry and H of one workload system."""
    g = water_box(n_mol, seed=seed)
    return g, hamiltonian(g, kind, **kw)


def log_uniform_sizes(n_sys: int, lo: int = 200, hi: int = 5000, seed: int = 1006) -> np.ndarray:
    """Seeded log-uniform molecule counts for a batch of uneven systems."""
    u = _uniform(seed, _P_SIZES, np.arange(n_sys, dtype=np.int64))
    return np.floor(np.exp(np.log(lo) + u * (np.log(hi + 1) - np.log(lo)))).astype(np.int64).clip(lo, hi)
