"""ctypes front end of the CSS ORACLE (plain FP64 C in css_oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's CPU-baseline
leg may import this package; the library's product path never does.  It shares no code with
the CUDA library.  Every function takes and returns host numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "css_oracle.c"
_LIB = _HERE / "libcss_oracle.so"

SYMMETRIZE = 1
REORTH_LOCAL = 4
ENERGY_WEIGHTED = 16  # write the energy-weighted density matrix (Z built with lambda f(lambda))
INV_SQRT = 32  # the matrix is an overlap S: write S^(-1/2) (function x^(-1/2), no mu)
SIGNS_ONES = 1

_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with the host C compiler (gcc, OpenMP, no fp contraction)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".{os.getpid()}.tmp.so")
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", str(tmp), str(_SRC), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(str(_LIB))
        p = C.c_void_p
        i32, i64, u64, f64 = C.c_int32, C.c_int64, C.c_uint64, C.c_double
        lib.css_ref_hash.restype = u64
        lib.css_ref_hash.argtypes = [u64, u64]
        lib.css_ref_fermi.restype = f64
        lib.css_ref_fermi.argtypes = [f64, f64, f64]
        lib.css_ref_neighbours.argtypes = [i32, p, f64, f64, p, C.POINTER(C.c_void_p)]
        lib.css_ref_free.argtypes = [p]
        lib.css_ref_color_graph.argtypes = [i32, p, p, u64, p, p]
        lib.css_ref_color.argtypes = [i32, p, f64, f64, u64, p, p]
        lib.css_ref_color_conflicts.argtypes = [i32, p, f64, f64, p, p]
        lib.css_ref_probes.argtypes = [p, i32, i32, u64, C.c_int, p]
        lib.css_ref_eigh.argtypes = [i32, p, p]
        lib.css_ref_lanczos.argtypes = [i32, i32, p, p, p, p, p, i32, i32, C.c_int, p, p, p]
        lib.css_ref_density.argtypes = [i32, i32, i32, p, p, p, p, p, i32, f64, f64, f64, f64, C.c_int, i32,
                                        C.c_int, p, i32, p, p, p, p, p]
        lib.css_ref_ritz.argtypes = [i32, i32, p, p, p, p, p, i32, i32, C.c_int, p, p, p, p]
        lib.css_ref_hprime.argtypes = [i32, i32, i32, p, p, p, i32, p, p, p, p, p, i32, i32, C.c_int, p, p, p]
        lib.css_ref_density_nonorth.argtypes = [i32, i32, i32, p, p, p, p, i32, p, p, p, p, p, p, i32, f64, f64,
                                                f64, f64, C.c_int, i32, C.c_int, p, p, p, p, p]
        lib.css_ref_solve_mu.argtypes = [i32, p, i32, p, p, f64, f64, f64, p]
        lib.css_ref_num_threads.restype = C.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _chk(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def hash64(seed: int, x: int) -> int:
    return int(_load().css_ref_hash(seed, x))


def fermi(x: float, mu: float, kT: float) -> float:
    return float(_load().css_ref_fermi(x, mu, kT))


def neighbours(xyz, box: float, r_col: float):
    """Colour-graph adjacency (CSR) by brute force in int64 fixed point."""
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    ptr = np.zeros(n + 1, dtype=np.int32)
    adj = C.c_void_p()
    _chk(lib.css_ref_neighbours(n, _ptr(xyz), box, r_col, _ptr(ptr), C.byref(adj)), "neighbours")
    m = int(ptr[-1])
    out = np.ctypeslib.as_array(C.cast(adj, C.POINTER(C.c_int32)), shape=(max(m, 1),))[:m].copy()
    lib.css_ref_free(adj)
    return ptr, out


def color_graph(adj_ptr, adj, seed: int):
    lib = _load()
    adj_ptr = np.ascontiguousarray(adj_ptr, dtype=np.int32)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    n = adj_ptr.shape[0] - 1
    col = np.empty(n, dtype=np.int32)
    nc = np.zeros(1, dtype=np.int32)
    _chk(lib.css_ref_color_graph(n, _ptr(adj_ptr), _ptr(adj), seed, _ptr(col), _ptr(nc)), "color_graph")
    return col, int(nc[0])


def color(xyz, box: float, r_col: float, seed: int):
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    col = np.empty(n, dtype=np.int32)
    nc = np.zeros(1, dtype=np.int32)
    _chk(lib.css_ref_color(n, _ptr(xyz), box, r_col, seed, _ptr(col), _ptr(nc)), "color")
    return col, int(nc[0])


def color_conflicts(xyz, box: float, r_col: float, colour) -> int:
    """Same-coloured pairs closer than r_col (the colour-graph rule, brute force)."""
    lib = _load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    if colour.shape[0] != xyz.shape[0]:
        raise ValueError("one colour per molecule")
    k = np.zeros(1, dtype=np.int64)
    _chk(lib.css_ref_color_conflicts(xyz.shape[0], _ptr(xyz), box, r_col, _ptr(colour), _ptr(k)), "color_conflicts")
    return int(k[0])


def color_update(xyz, box: float, r_col: float, seed: int, colour, n_colours: int, skin: float = 0.0):
    """Keep (colour, n_colours) when it has no conflict at r_col on this geometry, else
    recolour from scratch at r_col + skin: returns (colour, n_colours, recoloured)."""
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    ok = (n_colours >= 1 and colour.size == len(xyz) and colour.min(initial=0) >= 0
          and colour.max(initial=0) < n_colours and color_conflicts(xyz, box, r_col, colour) == 0)
    if ok:
        return colour.copy(), int(n_colours), False
    col, nc = color(xyz, box, r_col + skin, seed)
    return col, nc, True


def probes(colour, b: int, sign_seed: int, flags: int = 0):
    lib = _load()
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    n = colour.shape[0]
    s = np.empty(n * b, dtype=np.int8)
    _chk(lib.css_ref_probes(_ptr(colour), n, b, sign_seed, flags, _ptr(s)), "probes")
    return s


def eigh(A):
    """Eigen-decomposition of a symmetric matrix: (w ascending, U columns)."""
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    n = A.shape[0]
    w = np.empty(n)
    _chk(_load().css_ref_eigh(n, _ptr(A), _ptr(w)), "eigh")
    return w, A


def _h(H):
    return (H.n_brow, H.b, _ptr(np.ascontiguousarray(H.row_ptr, dtype=np.int32)),
            _ptr(np.ascontiguousarray(H.col_idx, dtype=np.int32)),
            _ptr(np.ascontiguousarray(H.val, dtype=np.float64)))


def lanczos(H, colour, sign, c: int, m: int, flags: int = 0, want_q: bool = False):
    """Projected block-tridiagonal matrix T (n_used x n_used) of colour c, and Q if asked."""
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    sign = np.ascontiguousarray(sign, dtype=np.int8)
    nmax = m * H.b
    T = np.zeros((nmax, nmax))
    Q = np.zeros((H.n, nmax)) if want_q else None
    nb = np.zeros(1, dtype=np.int32)
    refs = (np.ascontiguousarray(H.row_ptr, dtype=np.int32), np.ascontiguousarray(H.col_idx, dtype=np.int32),
            np.ascontiguousarray(H.val, dtype=np.float64))
    _chk(_load().css_ref_lanczos(H.n_brow, H.b, _ptr(refs[0]), _ptr(refs[1]), _ptr(refs[2]), _ptr(colour),
                                 _ptr(sign), c, m, flags, _ptr(T), _ptr(Q), _ptr(nb)), "lanczos")
    n = int(nb[0]) * H.b
    T = T[:n, :n].copy()
    return (T, Q[:, :n].copy()) if want_q else T


def ritz(H, colour, sign, n_colours: int, m: int, flags: int = 0, colours=None):
    """Per-colour Ritz values and weights: list of (lam, w) arrays (empty for colours not in
    `colours` when that is given)."""
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    sign = np.ascontiguousarray(sign, dtype=np.int8)
    want = None
    if colours is not None:
        want = np.zeros(n_colours, dtype=np.int8)
        want[np.asarray(colours, dtype=np.int64)] = 1
    nmax = m * H.b
    lam = np.zeros((n_colours, nmax)); wgt = np.zeros((n_colours, nmax))
    nper = np.zeros(n_colours, dtype=np.int32)
    rp = np.ascontiguousarray(H.row_ptr, dtype=np.int32); ci = np.ascontiguousarray(H.col_idx, dtype=np.int32)
    vv = np.ascontiguousarray(H.val, dtype=np.float64)
    _chk(_load().css_ref_ritz(H.n_brow, H.b, _ptr(rp), _ptr(ci), _ptr(vv), _ptr(colour), _ptr(sign),
                              n_colours, m, flags, _ptr(want), _ptr(lam), _ptr(wgt), _ptr(nper)), "ritz")
    return [(lam[c, :nper[c]].copy(), wgt[c, :nper[c]].copy()) for c in range(n_colours)]


def solve_mu(ritz_lists, kT: float, n_elec: float, ne_tol: float = 0.0) -> float:
    """mu from per-colour Ritz lists [(lam, w), ...] (the rule of `density`, lists summed in the
    order given)."""
    n = len(ritz_lists)
    nmax = max(1, max(len(l) for l, _ in ritz_lists))
    lam = np.zeros((n, nmax)); wgt = np.zeros((n, nmax))
    nper = np.zeros(n, dtype=np.int32)
    for t, (l, w) in enumerate(ritz_lists):
        nper[t] = len(l)
        lam[t, :len(l)] = l
        wgt[t, :len(w)] = w
    mu = np.zeros(1)
    _chk(_load().css_ref_solve_mu(n, _ptr(nper), nmax, _ptr(lam), _ptr(wgt), kT, n_elec, ne_tol, _ptr(mu)),
         "solve_mu")
    return float(mu[0])


def density(H, colour, sign, n_colours: int, *, mu: float = 0.0, kT: float = 0.05, n_elec: float = 0.0,
            solve_mu: bool = True, m: int = 30, flags: int = SYMMETRIZE, colour_subset=None, P_init=None,
            ne_tol: float = 0.0):
    """CSS density matrix on H's pattern.

    ne_tol: electron-count tolerance of the mu rule (<= 0: 1e-4 N_e/2).
    Returns dict(P=(nnzb, b, b), trP, trPH, mu, n_breakdown)."""
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    sign = np.ascontiguousarray(sign, dtype=np.int8)
    P = np.zeros((H.nnzb, H.b, H.b)) if P_init is None else np.array(P_init, dtype=np.float64, order="C")
    sub = None if colour_subset is None else np.ascontiguousarray(colour_subset, dtype=np.int32)
    out = np.zeros(3)
    nb = np.zeros(1, dtype=np.int32)
    rp = np.ascontiguousarray(H.row_ptr, dtype=np.int32); ci = np.ascontiguousarray(H.col_idx, dtype=np.int32)
    vv = np.ascontiguousarray(H.val, dtype=np.float64)
    st = _load().css_ref_density(
        H.n_brow, H.b, H.nnzb, _ptr(rp), _ptr(ci), _ptr(vv), _ptr(colour), _ptr(sign), n_colours,
        mu, kT, n_elec, ne_tol, int(bool(solve_mu)), m, flags, _ptr(sub), 0 if sub is None else sub.shape[0],
        _ptr(P), _ptr(out[0:1]), _ptr(out[1:2]), _ptr(out[2:3]), _ptr(nb))
    _chk(st, "density")
    return {"P": P, "trP": float(out[0]), "trPH": float(out[1]), "mu": float(out[2]),
            "n_breakdown": int(nb[0])}


def hprime(S, H, colour, sign, n_colours: int, *, m: int = 10, flags: int = SYMMETRIZE):
    """H' of a non-orthogonal basis: S~^(-1/2) by CSS on S (probes from colour/sign), then
    H' extracted from S~^(-1/2) H Y <o|.  Returns dict(Sinv=(nnzb_S, b, b), Hp=(nnzb_H, b, b), trHp)."""
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    sign = np.ascontiguousarray(sign, dtype=np.int8)
    Si = np.zeros((S.nnzb, S.b, S.b)); Hp = np.zeros((H.nnzb, H.b, H.b)); tr = np.zeros(1)
    arrs = []
    for M in (S, H):
        arrs.append((np.ascontiguousarray(M.row_ptr, dtype=np.int32), np.ascontiguousarray(M.col_idx, dtype=np.int32),
                     np.ascontiguousarray(M.val, dtype=np.float64)))
    (sr, sc, sv), (hr, hc, hv) = arrs
    st = _load().css_ref_hprime(S.n_brow, S.b, S.nnzb, _ptr(sr), _ptr(sc), _ptr(sv), H.nnzb, _ptr(hr), _ptr(hc),
                                _ptr(hv), _ptr(colour), _ptr(sign), n_colours, m, flags, _ptr(Si), _ptr(Hp), _ptr(tr))
    _chk(st, "hprime")
    return {"Sinv": Si, "Hp": Hp, "trHp": float(tr[0])}


def density_nonorth(S, Sinv, H, Hp, colour, sign, n_colours: int, *, mu: float = 0.0, kT: float = 0.05,
                    n_elec: float = 0.0, solve_mu: bool = True, m: int = 30, flags: int = SYMMETRIZE,
                    ne_tol: float = 0.0):
    """Density matrix of a non-orthogonal basis from S~^(-1/2) (values Sinv on S's pattern) and
    H' (values Hp on H's pattern), with Krylov spaces of H' started at S~^(-1/2) r_c; mu from the
    electron count Tr(rho S).  Returns dict(P=(nnzb_H, b, b), trPS, trPH, mu, n_breakdown)."""
    colour = np.ascontiguousarray(colour, dtype=np.int32)
    sign = np.ascontiguousarray(sign, dtype=np.int8)
    P = np.zeros((H.nnzb, H.b, H.b))
    out = np.zeros(3)
    nb = np.zeros(1, dtype=np.int32)
    sr, sc, sv = (np.ascontiguousarray(S.row_ptr, dtype=np.int32), np.ascontiguousarray(S.col_idx, dtype=np.int32),
                  np.ascontiguousarray(S.val, dtype=np.float64))
    hr, hc, hv = (np.ascontiguousarray(H.row_ptr, dtype=np.int32), np.ascontiguousarray(H.col_idx, dtype=np.int32),
                  np.ascontiguousarray(H.val, dtype=np.float64))
    si = np.ascontiguousarray(Sinv, dtype=np.float64).reshape(S.nnzb, S.b, S.b)
    hp = np.ascontiguousarray(Hp, dtype=np.float64).reshape(H.nnzb, H.b, H.b)
    st = _load().css_ref_density_nonorth(
        H.n_brow, H.b, S.nnzb, _ptr(sr), _ptr(sc), _ptr(sv), _ptr(si), H.nnzb, _ptr(hr), _ptr(hc), _ptr(hv),
        _ptr(hp), _ptr(colour), _ptr(sign), n_colours, mu, kT, n_elec, ne_tol, int(bool(solve_mu)), m, flags,
        _ptr(P), _ptr(out[0:1]), _ptr(out[1:2]), _ptr(out[2:3]), _ptr(nb))
    _chk(st, "density_nonorth")
    return {"P": P, "trPS": float(out[0]), "trPH": float(out[1]), "mu": float(out[2]), "n_breakdown": int(nb[0])}


def num_threads() -> int:
    return int(_load().css_ref_num_threads())
