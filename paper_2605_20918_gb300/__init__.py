"""GB300 (sm_103a) CSS density-matrix library: Python binding of the C-ABI in include/css.h.

Argument marshalling only: every step of the method runs in the CUDA kernels of libcss.so.
Device arrays are passed as torch CUDA tensors (torch supplies device memory and streams);
there is no CPU fallback, and loading fails loudly when the library is missing.

Names follow the C entry points: css_create, css_color, css_color_graph, css_probes,
css_density, css_density_batch, css_pbuild, css_get_info.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from pathlib import Path

import numpy as np

__all__ = [
    "CSSError", "Context", "DeviceBSR", "load_library", "library_path", "css_create", "css_destroy", "css_color",
    "css_color_graph", "css_color_check", "css_color_update", "css_probes", "css_density", "css_density_nonorth", "css_density_batch", "css_pbuild", "css_get_info", "css_ritz", "css_projected", "css_eigen_blocks",
    "CSS_OK", "CSS_WARN_BREAKDOWN", "CSS_FP64", "CSS_MIXED_FP32", "CSS_MIXED_3XTF32", "CSS_FP64_SPLIT", "CSS_SYMMETRIZE", "CSS_TWO_PASS",
    "CSS_REORTH_LOCAL", "CSS_HOST_IO", "CSS_SIGNS_ONES", "CSS_ENERGY_WEIGHTED", "CSS_INV_SQRT", "CSS_RITZ_ONLY",
    "css_density_colours", "css_solve_mu",
]

CSS_OK, CSS_ERR_INVALID_ARG, CSS_ERR_NOMEM, CSS_ERR_CUDA, CSS_ERR_TIMEOUT, CSS_ERR_NUMERIC = 0, 1, 2, 3, 4, 5
CSS_WARN_BREAKDOWN, CSS_ERR_UNSUPPORTED = 6, 7
CSS_FP64, CSS_MIXED_FP32, CSS_MIXED_3XTF32, CSS_FP64_SPLIT = 0, 1, 2, 3
CSS_SYMMETRIZE, CSS_TWO_PASS, CSS_REORTH_LOCAL, CSS_HOST_IO, CSS_ENERGY_WEIGHTED, CSS_INV_SQRT = 1, 2, 4, 8, 16, 32
CSS_RITZ_ONLY = 64
CSS_SIGNS_ONES = 1

_PKG = Path(__file__).resolve().parent


def library_path() -> Path:
    return _PKG / "libcss.so"


class _Geom(C.Structure):
    _fields_ = [("n_mol", C.c_int32), ("xyz", C.c_void_p), ("box", C.c_double)]


class _BSR(C.Structure):
    _fields_ = [("n_brow", C.c_int32), ("b", C.c_int32), ("nnzb", C.c_int32), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("val", C.c_void_p)]


class _Fermi(C.Structure):
    _fields_ = [("mu", C.c_double), ("kT", C.c_double), ("n_elec", C.c_double), ("ne_tol", C.c_double),
                ("solve_mu", C.c_int32)]


class _Info(C.Structure):
    _fields_ = [("n_colours", C.c_int32), ("n_pairs", C.c_int32), ("n_breakdown", C.c_int32), ("m", C.c_int32),
                ("workspace_bytes", C.c_int64)] + \
               [(k, C.c_double) for k in ("ms_color", "ms_probes", "ms_setup", "ms_lanczos", "ms_spmm", "ms_eigen",
                                          "ms_mu", "ms_extract", "ms_total")] + \
               [("spmm_launches", C.c_int64), ("spmm_flops", C.c_double), ("spmm_bytes", C.c_double),
                ("kernel_launches", C.c_int64), ("ms_rows", C.c_double), ("graph_launches", C.c_int64),
                ("graph_instantiations", C.c_int64)]


_lib = None


def load_library(path: str | Path | None = None):
    """Load libcss.so (no fallback: raises if it is missing or does not load)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = Path(path) if path else library_path()
    if not p.exists():
        raise RuntimeError(f"CSS CUDA library not found at {p}; build it with "
                           f"`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(str(p))
    v, i32, u32, u64, f64 = C.c_void_p, C.c_int32, C.c_uint32, C.c_uint64, C.c_double
    st = C.c_int
    lib.css_create.argtypes = [C.POINTER(C.c_void_p), C.c_int]
    lib.css_create.restype = st
    lib.css_destroy.argtypes = [v]
    lib.css_destroy.restype = None
    lib.css_status_str.argtypes = [st]
    lib.css_status_str.restype = C.c_char_p
    lib.css_last_error.argtypes = [v]
    lib.css_last_error.restype = C.c_char_p
    lib.css_get_info.argtypes = [v, C.POINTER(_Info)]
    lib.css_get_info.restype = st
    lib.css_color.argtypes = [v, C.POINTER(_Geom), f64, u64, v, C.POINTER(C.c_int32), v]
    lib.css_color.restype = st
    lib.css_color_graph.argtypes = [v, i32, v, v, u64, v, C.POINTER(C.c_int32), v]
    lib.css_color_graph.restype = st
    lib.css_color_check.argtypes = [v, C.POINTER(_Geom), f64, v, i32, C.POINTER(C.c_int64), v]
    lib.css_color_check.restype = st
    lib.css_color_update.argtypes = [v, C.POINTER(_Geom), f64, f64, u64, v, C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int32), v]
    lib.css_color_update.restype = st
    lib.css_probes.argtypes = [v, v, i32, i32, u64, u32, v, v]
    lib.css_probes.restype = st
    lib.css_density.argtypes = [v, C.POINTER(_BSR), v, v, i32, C.POINTER(_Fermi), i32, st, u32, v,
                                C.POINTER(f64), C.POINTER(f64), C.POINTER(f64), v]
    lib.css_density.restype = st
    lib.css_density_batch.argtypes = [v, i32, C.POINTER(_BSR), C.POINTER(v), C.POINTER(v), C.POINTER(i32),
                                      C.POINTER(_Fermi), i32, st, u32, C.POINTER(v), C.POINTER(f64), C.POINTER(f64),
                                      C.POINTER(f64), v]
    lib.css_density_batch.restype = st
    lib.css_pbuild.argtypes = [v, C.POINTER(_Geom), C.POINTER(_BSR), f64, u64, u64, C.POINTER(_Fermi), i32, st, u32,
                               v, v, C.POINTER(C.c_int32), C.POINTER(f64), C.POINTER(f64), C.POINTER(f64), v]
    lib.css_pbuild.restype = st
    lib.css_ritz.argtypes = [v, v, v, v, C.c_int64, C.POINTER(C.c_int32)]
    lib.css_projected.argtypes = [v, v, v, v, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_int32)]
    lib.css_projected.restype = st
    lib.css_eigen_blocks.argtypes = [v, i32, i32, i32, v, v, v, v, f64, f64, v, v, v, v]
    lib.css_eigen_blocks.restype = st
    lib.css_hprime.argtypes = [v, C.POINTER(_BSR), C.POINTER(_BSR), v, v, i32, i32, st, u32, v, v,
                               C.POINTER(C.c_double), v]
    lib.css_hprime.restype = st
    lib.css_density_nonorth.argtypes = [v, C.POINTER(_BSR), v, C.POINTER(_BSR), v, v, v, i32, C.POINTER(_Fermi), i32,
                                        st, u32, v, C.POINTER(f64), C.POINTER(f64), C.POINTER(f64), v]
    lib.css_density_nonorth.restype = st
    lib.css_density_colours.argtypes = [v, C.POINTER(_BSR), v, v, i32, v, C.POINTER(_Fermi), i32, st, u32, v,
                                        C.POINTER(f64), C.POINTER(f64), v]
    lib.css_density_colours.restype = st
    lib.css_solve_mu.argtypes = [v, i32, v, v, v, f64, f64, f64, C.POINTER(f64), v]
    lib.css_solve_mu.restype = st
    lib.css_ritz.restype = st
    _lib = lib
    return lib


class CSSError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


def _check(lib, ctx, status: int, what: str) -> int:
    if status in (CSS_OK, CSS_WARN_BREAKDOWN):
        return status
    msg = lib.css_last_error(ctx).decode() if ctx else ""
    raise CSSError(status, f"{what}: {lib.css_status_str(status).decode()} {msg}")


def _torch():
    import torch
    return torch


def _dev(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return C.c_void_p(t.data_ptr())


def _need(t, n: int, name: str) -> None:
    """Refuse a buffer of the wrong size before any pointer reaches the library (the C-ABI
    takes raw pointers and cannot check lengths)."""
    k = int(t.numel()) if hasattr(t, "numel") else int(np.asarray(t).size)
    if k != int(n):
        raise ValueError(f"{name} has {k} elements, expected {int(n)}")


def _stream(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


@dataclass
class DeviceBSR:
    """Block-sparse-row H on the device (torch tensors)."""
    n_brow: int
    b: int
    row_ptr: "object"   # int32 [n_brow+1]
    col_idx: "object"   # int32 [nnzb]
    val: "object"       # float64 [nnzb, b, b]

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.numel())

    @classmethod
    def from_host(cls, H, device="cuda"):
        """Upload a host BSR (synth.BSR-like) after checking its pattern arrays."""
        torch = _torch()
        rp = np.asarray(H.row_ptr)
        ci = np.asarray(H.col_idx)
        if rp.shape != (H.n_brow + 1,) or rp[0] != 0 or np.any(np.diff(rp) < 0) or rp[-1] != ci.size:
            raise ValueError("row_ptr must have n_brow + 1 non-decreasing entries from 0 to nnzb")
        if ci.size and (ci.min() < 0 or ci.max() >= H.n_brow):
            raise ValueError("col_idx outside [0, n_brow)")
        _need(H.val, ci.size * H.b * H.b, "val")
        return cls(H.n_brow, H.b, torch.as_tensor(np.ascontiguousarray(H.row_ptr, np.int32), device=device),
                   torch.as_tensor(np.ascontiguousarray(H.col_idx, np.int32), device=device),
                   torch.as_tensor(np.ascontiguousarray(H.val, np.float64), device=device))

    def _c(self) -> _BSR:
        torch = _torch()
        _need(self.row_ptr, self.n_brow + 1, "row_ptr")
        _need(self.val, self.nnzb * self.b * self.b, "val")
        return _BSR(self.n_brow, self.b, self.nnzb, _dev(self.row_ptr, torch.int32, "row_ptr"),
                    _dev(self.col_idx, torch.int32, "col_idx"), _dev(self.val, torch.float64, "val"))


def css_create(device: int = 0) -> C.c_void_p:
    lib = load_library()
    h = C.c_void_p()
    _check(lib, None, lib.css_create(C.byref(h), device), "css_create")
    return h


def css_destroy(ctx) -> None:
    load_library().css_destroy(ctx)


def css_get_info(ctx) -> dict:
    lib = load_library()
    info = _Info()
    _check(lib, ctx, lib.css_get_info(ctx, C.byref(info)), "css_get_info")
    return {k: getattr(info, k) for k, _ in _Info._fields_}


def css_color(ctx, xyz, box: float, r_col: float, seed: int, colour, stream=None) -> int:
    """Colour molecules (device xyz float64 [n,3] -> device colour int32 [n]); returns n_colours."""
    torch = _torch()
    lib = load_library()
    n = int(xyz.shape[0])
    _need(xyz, 3 * n, "xyz")
    _need(colour, n, "colour")
    g = _Geom(n, _dev(xyz, torch.float64, "xyz"), float(box))
    nc = C.c_int32()
    _check(lib, ctx, lib.css_color(ctx, C.byref(g), float(r_col), C.c_uint64(seed), _dev(colour, torch.int32, "colour"),
                                   C.byref(nc), _stream(stream)), "css_color")
    return int(nc.value)


def css_color_graph(ctx, adj_ptr, adj, seed: int, colour, stream=None) -> int:
    torch = _torch()
    lib = load_library()
    nc = C.c_int32()
    n = int(adj_ptr.numel()) - 1
    _need(colour, n, "colour")
    _check(lib, ctx, lib.css_color_graph(ctx, n, _dev(adj_ptr, torch.int32, "adj_ptr"),
                                         _dev(adj, torch.int32, "adj") if adj.numel() else C.c_void_p(0),
                                         C.c_uint64(seed), _dev(colour, torch.int32, "colour"), C.byref(nc),
                                         _stream(stream)), "css_color_graph")
    return int(nc.value)


def css_color_check(ctx, xyz, box: float, r_col: float, colour, n_colours: int, stream=None) -> int:
    """Same-coloured molecule pairs closer than r_col on the geometry xyz (0: still valid)."""
    torch = _torch()
    lib = load_library()
    n = int(xyz.shape[0])
    _need(xyz, 3 * n, "xyz")
    _need(colour, n, "colour")
    g = _Geom(n, _dev(xyz, torch.float64, "xyz"), float(box))
    k = C.c_int64()
    _check(lib, ctx, lib.css_color_check(ctx, C.byref(g), float(r_col), _dev(colour, torch.int32, "colour"),
                                         int(n_colours), C.byref(k), _stream(stream)), "css_color_check")
    return int(k.value)


def css_color_update(ctx, xyz, box: float, r_col: float, seed: int, colour, n_colours: int, *, skin: float = 0.0,
                     stream=None):
    """Keep `colour` (device int32 [n]) when it has no conflict at r_col on xyz, else recolour
    it in place at r_col + skin; n_colours = 0 means no colouring yet.  Returns
    (n_colours, recoloured)."""
    torch = _torch()
    lib = load_library()
    n = int(xyz.shape[0])
    _need(xyz, 3 * n, "xyz")
    _need(colour, n, "colour")
    g = _Geom(n, _dev(xyz, torch.float64, "xyz"), float(box))
    nc = C.c_int32(int(n_colours))
    re = C.c_int32(0)
    _check(lib, ctx, lib.css_color_update(ctx, C.byref(g), float(r_col), float(skin), C.c_uint64(seed),
                                          _dev(colour, torch.int32, "colour"), C.byref(nc), C.byref(re),
                                          _stream(stream)), "css_color_update")
    return int(nc.value), bool(re.value)


def css_probes(ctx, colour, b: int, sign_seed: int, sign, flags: int = 0, stream=None) -> None:
    torch = _torch()
    lib = load_library()
    _need(sign, int(colour.numel()) * int(b), "sign")
    _check(lib, ctx, lib.css_probes(ctx, _dev(colour, torch.int32, "colour"), int(colour.numel()), int(b),
                                    C.c_uint64(sign_seed), flags, _dev(sign, torch.int8, "sign"), _stream(stream)),
           "css_probes")


def _fermi(mu, kT, n_elec, solve_mu, ne_tol=0.0):
    return _Fermi(float(mu), float(kT), float(n_elec), float(ne_tol), 1 if solve_mu else 0)


def css_density(ctx, H: DeviceBSR, colour, sign, n_colours: int, P, *, mu=0.0, kT=0.05, n_elec=0.0,
                solve_mu=True, ne_tol=0.0, m=30, precision=CSS_FP64, flags=CSS_SYMMETRIZE, stream=None) -> dict:
    """CSS density matrix on H's pattern into P (device float64 [nnzb, b, b])."""
    torch = _torch()
    lib = load_library()
    _need(colour, H.n_brow, "colour")
    _need(sign, H.n_brow * H.b, "sign")
    _need(P, H.nnzb * H.b * H.b, "P")
    hb = H._c()
    f = _fermi(mu, kT, n_elec, solve_mu, ne_tol)
    tp, tph, mo = C.c_double(), C.c_double(), C.c_double()
    st = _check(lib, ctx, lib.css_density(ctx, C.byref(hb), _dev(colour, torch.int32, "colour"),
                                          _dev(sign, torch.int8, "sign"), int(n_colours), C.byref(f), int(m),
                                          int(precision), int(flags), _dev(P, torch.float64, "P"), C.byref(tp),
                                          C.byref(tph), C.byref(mo), _stream(stream)), "css_density")
    return {"trP": tp.value, "trPH": tph.value, "mu": mo.value, "status": st}


def css_hprime(ctx, S: DeviceBSR, H: DeviceBSR, colour, sign, n_colours: int, Sinv, Hp, *, m=10,
               precision=CSS_FP64, flags=CSS_SYMMETRIZE, stream=None) -> dict:
    """S~^(-1/2) (into Sinv, S's pattern) and H' (into Hp, H's pattern) of a non-orthogonal basis."""
    torch = _torch()
    lib = load_library()
    _need(colour, S.n_brow, "colour")
    _need(sign, S.n_brow * S.b, "sign")
    _need(Sinv, S.nnzb * S.b * S.b, "Sinv")
    _need(Hp, H.nnzb * H.b * H.b, "Hp")
    sb, hb = S._c(), H._c()
    tr = C.c_double()
    st = _check(lib, ctx, lib.css_hprime(ctx, C.byref(sb), C.byref(hb), _dev(colour, torch.int32, "colour"),
                                         _dev(sign, torch.int8, "sign"), int(n_colours), int(m), int(precision),
                                         int(flags), _dev(Sinv, torch.float64, "Sinv"), _dev(Hp, torch.float64, "Hp"),
                                         C.byref(tr), _stream(stream)), "css_hprime")
    return {"trHp": tr.value, "status": st}


def css_density_nonorth(ctx, S: DeviceBSR, Sinv, Hp: DeviceBSR, H_val, colour, sign, n_colours: int, P, *, mu=0.0,
                        kT=0.05, n_elec=0.0, solve_mu=True, ne_tol=0.0, m=30, precision=CSS_FP64,
                        flags=CSS_SYMMETRIZE, stream=None) -> dict:
    """Density matrix of a non-orthogonal basis into P (H's pattern) from S, S~^(-1/2) (Sinv, S's
    pattern), H' (Hp: values of H' on H's pattern) and H's own values (H_val)."""
    torch = _torch()
    lib = load_library()
    _need(Sinv, S.nnzb * S.b * S.b, "Sinv")
    _need(H_val, Hp.nnzb * Hp.b * Hp.b, "H_val")
    _need(colour, Hp.n_brow, "colour")
    _need(sign, Hp.n_brow * Hp.b, "sign")
    _need(P, Hp.nnzb * Hp.b * Hp.b, "P")
    sb, hb = S._c(), Hp._c()
    f = _fermi(mu, kT, n_elec, solve_mu, ne_tol)
    tps, tph, mo = C.c_double(), C.c_double(), C.c_double()
    st = _check(lib, ctx, lib.css_density_nonorth(ctx, C.byref(sb), _dev(Sinv, torch.float64, "Sinv"), C.byref(hb),
                                                  _dev(H_val, torch.float64, "H_val"),
                                                  _dev(colour, torch.int32, "colour"), _dev(sign, torch.int8, "sign"),
                                                  int(n_colours), C.byref(f), int(m), int(precision), int(flags),
                                                  _dev(P, torch.float64, "P"), C.byref(tps), C.byref(tph),
                                                  C.byref(mo), _stream(stream)), "css_density_nonorth")
    return {"trPS": tps.value, "trPH": tph.value, "mu": mo.value, "status": st}


def css_density_colours(ctx, H: DeviceBSR, colour, sign, n_colours: int, owned, P, *, mu, kT=0.05, m=30,
                        precision=CSS_FP64, flags=0, stream=None) -> dict:
    """Colours with owned[c] != 0 only (host sequence of n_colours flags): unsymmetrised columns
    of P at the given mu into P (other blocks zero), or with CSS_RITZ_ONLY their Ritz data only."""
    torch = _torch()
    lib = load_library()
    _need(colour, H.n_brow, "colour")
    _need(sign, H.n_brow * H.b, "sign")
    _need(P, H.nnzb * H.b * H.b, "P")
    ow = np.ascontiguousarray(np.asarray(owned, dtype=np.uint8))
    _need(ow, n_colours, "owned")
    hb = H._c()
    f = _fermi(mu, kT, 0.0, False)
    tp, tph = C.c_double(), C.c_double()
    st = _check(lib, ctx, lib.css_density_colours(ctx, C.byref(hb), _dev(colour, torch.int32, "colour"),
                                                  _dev(sign, torch.int8, "sign"), int(n_colours),
                                                  ow.ctypes.data_as(C.c_void_p), C.byref(f), int(m), int(precision),
                                                  int(flags), _dev(P, torch.float64, "P"), C.byref(tp), C.byref(tph),
                                                  _stream(stream)), "css_density_colours")
    return {"trP": tp.value, "trPH": tph.value, "status": st}


def css_solve_mu(ctx, ritz_lists, *, kT=0.05, n_elec=0.0, ne_tol=0.0, stream=None) -> float:
    """mu from gathered Ritz lists [(lam, w), ...] (host arrays) with the rule of css_density."""
    lib = load_library()
    n = len(ritz_lists)
    n_per = np.array([len(l) for l, _ in ritz_lists], dtype=np.int32)
    lam = np.ascontiguousarray(np.concatenate([np.asarray(l, np.float64) for l, _ in ritz_lists] + [np.zeros(1)]))
    wgt = np.ascontiguousarray(np.concatenate([np.asarray(w, np.float64) for _, w in ritz_lists] + [np.zeros(1)]))
    mu = C.c_double()
    _check(lib, ctx, lib.css_solve_mu(ctx, n, n_per.ctypes.data_as(C.c_void_p), lam.ctypes.data_as(C.c_void_p),
                                      wgt.ctypes.data_as(C.c_void_p), float(kT), float(n_elec), float(ne_tol),
                                      C.byref(mu), _stream(stream)), "css_solve_mu")
    return mu.value


def css_density_batch(ctx, Hs, colours, signs, n_colours, Ps, fermis, *, m=30, precision=CSS_FP64,
                      flags=CSS_SYMMETRIZE, stream=None) -> dict:
    """Several systems in one call.  fermis: list of dicts(mu, kT, n_elec, solve_mu)."""
    torch = _torch()
    lib = load_library()
    n = len(Hs)
    if not (len(colours) == len(signs) == len(n_colours) == len(Ps) == len(fermis) == n):
        raise ValueError("css_density_batch: one colour, sign, n_colours, P and fermi entry per system")
    for h, c, s_, p in zip(Hs, colours, signs, Ps):
        _need(c, h.n_brow, "colour")
        _need(s_, h.n_brow * h.b, "sign")
        _need(p, h.nnzb * h.b * h.b, "P")
    hb = (_BSR * n)(*[h._c() for h in Hs])
    cp = (C.c_void_p * n)(*[_dev(c, torch.int32, "colour") for c in colours])
    sp = (C.c_void_p * n)(*[_dev(s, torch.int8, "sign") for s in signs])
    nc = (C.c_int32 * n)(*[int(x) for x in n_colours])
    fr = (_Fermi * n)(*[_fermi(f.get("mu", 0.0), f.get("kT", 0.05), f.get("n_elec", 0.0), f.get("solve_mu", True),
                               f.get("ne_tol", 0.0)) for f in fermis])
    pp = (C.c_void_p * n)(*[_dev(p, torch.float64, "P") for p in Ps])
    tp, tph, mo = (C.c_double * n)(), (C.c_double * n)(), (C.c_double * n)()
    st = _check(lib, ctx, lib.css_density_batch(ctx, n, hb, cp, sp, nc, fr, int(m), int(precision), int(flags), pp,
                                                tp, tph, mo, _stream(stream)), "css_density_batch")
    return {"trP": list(tp), "trPH": list(tph), "mu": list(mo), "status": st}


def css_pbuild(ctx, xyz, box, H, P, *, r_col, colour_seed=1004, sign_seed=1005, mu=0.0, kT=0.05, n_elec=0.0,
               solve_mu=True, ne_tol=0.0, m=30, precision=CSS_FP64, flags=CSS_SYMMETRIZE, colour_out=None, stream=None) -> dict:
    """Whole P build.  With CSS_HOST_IO in flags, xyz / H (synth.BSR) / P / colour_out are host
    numpy arrays and the copies happen inside the call; otherwise torch CUDA tensors."""
    lib = load_library()
    host = bool(flags & CSS_HOST_IO)
    n_mol = int(xyz.shape[0])
    _need(xyz, 3 * n_mol, "xyz")
    _need(P, H.nnzb * H.b * H.b, "P")
    if colour_out is not None:
        _need(colour_out, n_mol, "colour_out")
    if host:
        xyz = np.ascontiguousarray(xyz, np.float64)
        rp = np.ascontiguousarray(H.row_ptr, np.int32)
        ci = np.ascontiguousarray(H.col_idx, np.int32)
        vv = np.ascontiguousarray(H.val, np.float64)
        if not (isinstance(P, np.ndarray) and P.flags.c_contiguous and P.dtype == np.float64):
            raise TypeError("P must be a C-contiguous float64 numpy array with CSS_HOST_IO")
        if colour_out is not None and not (isinstance(colour_out, np.ndarray) and colour_out.dtype == np.int32
                                           and colour_out.flags.c_contiguous):
            raise TypeError("colour_out must be a C-contiguous int32 numpy array with CSS_HOST_IO")
        g = _Geom(xyz.shape[0], xyz.ctypes.data_as(C.c_void_p), float(box))
        hb = _BSR(H.n_brow, H.b, int(ci.shape[0]), rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                  vv.ctypes.data_as(C.c_void_p))
        pp = P.ctypes.data_as(C.c_void_p)
        cop = colour_out.ctypes.data_as(C.c_void_p) if colour_out is not None else C.c_void_p(0)
        keep = (xyz, rp, ci, vv)
    else:
        torch = _torch()
        g = _Geom(int(xyz.shape[0]), _dev(xyz, torch.float64, "xyz"), float(box))
        hb = H._c()
        pp = _dev(P, torch.float64, "P")
        cop = _dev(colour_out, torch.int32, "colour_out") if colour_out is not None else C.c_void_p(0)
        keep = ()
    f = _fermi(mu, kT, n_elec, solve_mu, ne_tol)
    nc = C.c_int32()
    tp, tph, mo = C.c_double(), C.c_double(), C.c_double()
    st = _check(lib, ctx, lib.css_pbuild(ctx, C.byref(g), C.byref(hb), float(r_col), C.c_uint64(colour_seed),
                                         C.c_uint64(sign_seed), C.byref(f), int(m), int(precision), int(flags), pp,
                                         cop, C.byref(nc), C.byref(tp), C.byref(tph), C.byref(mo), _stream(stream)),
                "css_pbuild")
    del keep
    return {"n_colours": nc.value, "trP": tp.value, "trPH": tph.value, "mu": mo.value, "status": st}


def css_ritz(ctx):
    """Ritz values and weights of the last density call: list of (lam, w) per colour."""
    lib = load_library()
    nc = C.c_int32()
    _check(lib, ctx, lib.css_ritz(ctx, None, None, None, 0, C.byref(nc)), "css_ritz")
    n_per = np.zeros(nc.value, np.int32)
    # sizes first: with capacity 0 the call fills n_per and reports INVALID_ARG
    lib.css_ritz(ctx, None, None, n_per.ctypes.data_as(C.c_void_p), 0, C.byref(nc))
    total = int(n_per.sum())
    lam = np.zeros(max(total, 1)); wgt = np.zeros(max(total, 1))
    _check(lib, ctx, lib.css_ritz(ctx, lam.ctypes.data_as(C.c_void_p), wgt.ctypes.data_as(C.c_void_p),
                                  n_per.ctypes.data_as(C.c_void_p), total, C.byref(nc)), "css_ritz")
    out, o = [], 0
    for k in n_per:
        out.append((lam[o:o + k].copy(), wgt[o:o + k].copy()))
        o += k
    return out


def css_projected(ctx):
    """Projected block-tridiagonal matrices of the last density call: (A, B, nblk) with A, B of
    shape [n_colours, m, b, b]."""
    lib = load_library()
    nc, m, b = C.c_int32(), C.c_int32(), C.c_int32()
    lib.css_projected(ctx, None, None, None, 0, C.byref(nc), C.byref(m), C.byref(b))
    shape = (nc.value, m.value, b.value, b.value)
    A = np.zeros(shape); B = np.zeros(shape); nb = np.zeros(nc.value, np.int32)
    _check(lib, ctx, lib.css_projected(ctx, A.ctypes.data_as(C.c_void_p), B.ctypes.data_as(C.c_void_p),
                                       nb.ctypes.data_as(C.c_void_p), A.size, C.byref(nc), C.byref(m), C.byref(b)),
           "css_projected")
    return A, B, nb


def css_eigen_blocks(ctx, A, B, nblk, cnt, *, mu=0.0, kT=0.05, want_z=True, stream=None):
    """Eigen stage alone.  A, B: float64 CUDA tensors [n_col, m, b, b]; nblk, cnt: int32 CUDA
    tensors [n_col].  Returns (lam [n_col, m b], wgt [n_col, m b], Z [n_col, m b, b] or None)."""
    torch = _torch()
    lib = load_library()
    n_col, m, b = int(A.shape[0]), int(A.shape[1]), int(A.shape[2])
    _need(A, n_col * m * b * b, "A")
    _need(B, n_col * m * b * b, "B")
    _need(nblk, n_col, "nblk")
    _need(cnt, n_col, "cnt")
    lam = torch.zeros((n_col, m * b), dtype=torch.float64, device=A.device)
    wgt = torch.zeros_like(lam)
    Z = torch.zeros((n_col, m * b, b), dtype=torch.float64, device=A.device) if want_z else None
    _check(lib, ctx, lib.css_eigen_blocks(ctx, n_col, b, m, _dev(A, torch.float64, "A"), _dev(B, torch.float64, "B"),
                                          _dev(nblk, torch.int32, "nblk"), _dev(cnt, torch.int32, "cnt"), float(mu),
                                          float(kT), _dev(lam, torch.float64, "lam"), _dev(wgt, torch.float64, "wgt"),
                                          _dev(Z, torch.float64, "Z") if want_z else C.c_void_p(0), _stream(stream)),
           "css_eigen_blocks")
    return lam, wgt, Z


class Context:
    """Owns a css_ctx (device workspace) for one GPU."""

    def __init__(self, device: int = 0):
        self.handle = css_create(device)

    def close(self):
        if self.handle:
            css_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def color(self, *a, **k):
        return css_color(self.handle, *a, **k)

    def color_graph(self, *a, **k):
        return css_color_graph(self.handle, *a, **k)

    def color_check(self, *a, **k):
        return css_color_check(self.handle, *a, **k)

    def color_update(self, *a, **k):
        return css_color_update(self.handle, *a, **k)

    def probes(self, *a, **k):
        return css_probes(self.handle, *a, **k)

    def density(self, *a, **k):
        return css_density(self.handle, *a, **k)

    def hprime(self, *a, **k):
        return css_hprime(self.handle, *a, **k)

    def density_nonorth(self, *a, **k):
        return css_density_nonorth(self.handle, *a, **k)

    def density_batch(self, *a, **k):
        return css_density_batch(self.handle, *a, **k)

    def density_colours(self, *a, **k):
        return css_density_colours(self.handle, *a, **k)

    def solve_mu(self, *a, **k):
        return css_solve_mu(self.handle, *a, **k)

    def pbuild(self, *a, **k):
        return css_pbuild(self.handle, *a, **k)

    def info(self):
        return css_get_info(self.handle)

    def ritz(self):
        return css_ritz(self.handle)

    def projected(self):
        return css_projected(self.handle)

    def eigen_blocks(self, *a, **k):
        return css_eigen_blocks(self.handle, *a, **k)
