"""ctypes binding of the C ABI in ``include/tpcf.h`` (argument marshalling only).

Every function of the C library is exposed here under the same name
(``tpcf_create``, ``tpcf_catalog_create``, ``tpcf_count_auto``, ...); they
raise :class:`TpcfError` on a non-zero status instead of returning it.  All
computation happens inside ``libtpcf.so`` (CUDA kernels and the native host
runtime); this module only converts numpy arrays / torch tensors to pointers.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA).
Streams are ``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers or
``None`` (the legacy default stream).

The library must have been built (``paper_1204_6630_gb300.build.build()``);
importing this module does not build it, and a missing library raises
``ImportError``: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

TPCF_OK, TPCF_EINVAL, TPCF_ENOMEM, TPCF_EBUDGET, TPCF_ECUDA = 0, 1, 2, 3, 4
TPCF_EAGAIN, TPCF_ETIMEOUT, TPCF_EOVERFLOW, TPCF_ECANCELED, TPCF_ENOTFOUND, TPCF_ESTATE = 5, 6, 7, 8, 9, 10
TPCF_HOST, TPCF_DEVICE = 0, 1
TPCF_SCREEN_RECHECK, TPCF_PLAIN_FP64 = 0, 1
TPCF_LS_EXACT, TPCF_LS_PAPER = 0, 1
TPCF_F_NO_SORT = 0x1
TPCF_F_PACKED_FMA = 0x4
TPCF_F_AUTOTUNE = 0x8
TPCF_F_PRUNE = 0x10
TPCF_F_CHECK_OVERFLOW = 0x20
TPCF_F_TEST_WAIT_TIMEOUT = 0x100
TPCF_F_TEST_BAD_TOTAL = 0x200
TPCF_MAX_EDGES = 321
TPCF_GRAPH_AUTO, TPCF_GRAPH_CROSS, TPCF_GRAPH_ALL, TPCF_GRAPH_PATCHES = 0, 1, 2, 3


class TpcfError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {strerror(status)} ({status})"
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


class tpcf_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("precision", ctypes.c_int), ("guard_band", ctypes.c_double),
                ("hbm_budget_bytes", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("threads", ctypes.c_int), ("ipt", ctypes.c_int), ("jtile", ctypes.c_int), ("stages", ctypes.c_int),
                ("shard_index", ctypes.c_uint32), ("shard_count", ctypes.c_uint32),
                ("wait_timeout_us", ctypes.c_uint32), ("server_workers", ctypes.c_int)]


class tpcf_stats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_uint64), ("band_pairs", ctypes.c_uint64),
                ("band_mismatch", ctypes.c_uint64), ("device_error", ctypes.c_uint32),
                ("launches", ctypes.c_uint32), ("kernel_ms", ctypes.c_double),
                ("pruned_pairs", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class tpcf_job(ctypes.Structure):
    _fields_ = [("d_xyz", ctypes.c_void_p), ("nd", ctypes.c_uint64), ("r_xyz", ctypes.c_void_p),
                ("nr", ctypes.c_uint64), ("edges_rad", ctypes.c_void_p), ("nedges", ctypes.c_int),
                ("estimator", ctypes.c_int)]


class tpcf_result(ctypes.Structure):
    _fields_ = [("dd", ctypes.c_void_p), ("dr", ctypes.c_void_p), ("rr", ctypes.c_void_p),
                ("w", ctypes.c_void_p), ("status", ctypes.c_int), ("nedges", ctypes.c_int),
                ("submit_ms", ctypes.c_double), ("queued_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("pairs", ctypes.c_uint64)]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_dp = ctypes.POINTER(ctypes.c_double)
_u64p = ctypes.POINTER(ctypes.c_uint64)

# name -> (restype, argtypes); the list matches include/tpcf.h
_SIGS = {
    "tpcf_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "tpcf_last_error": (ctypes.c_char_p, [_vp]),
    "tpcf_config_default": (None, [ctypes.POINTER(tpcf_config)]),
    "tpcf_version": (ctypes.c_int, []),
    "tpcf_kernel_launches": (_u64, [_vp]),
    "tpcf_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(tpcf_config)]),
    "tpcf_destroy": (ctypes.c_int, [_vp]),
    "tpcf_catalog_create": (ctypes.c_int, [_vp, _vp, _u64, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    "tpcf_catalog_create_segmented": (ctypes.c_int, [_vp, _vp, _u64, ctypes.c_int, _u64p, ctypes.c_int,
                                                     _vp, ctypes.POINTER(_vp)]),
    "tpcf_catalog_destroy": (ctypes.c_int, [_vp]),
    "tpcf_catalog_size": (_u64, [_vp]),
    "tpcf_bins_create": (ctypes.c_int, [_vp, _dp, ctypes.c_int, ctypes.POINTER(_vp)]),
    "tpcf_catalog_create_3d": (ctypes.c_int, [_vp, _vp, _u64, ctypes.c_int, _u64p, ctypes.c_int, _vp,
                                              ctypes.POINTER(_vp)]),
    "tpcf_bins_create_3d": (ctypes.c_int, [_vp, _dp, ctypes.c_int, ctypes.POINTER(_vp)]),
    "tpcf_bins_thresholds_3d": (ctypes.c_int, [_dp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_int)]),
    "tpcf_bins_destroy": (ctypes.c_int, [_vp]),
    "tpcf_bins_thresholds": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.c_double, _dp,
                                            ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                            ctypes.POINTER(ctypes.c_int)]),
    "tpcf_count_auto": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(tpcf_stats)]),
    "tpcf_count_cross": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int,
                                        ctypes.POINTER(tpcf_stats)]),
    "tpcf_count_all": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int,
                                      ctypes.POINTER(tpcf_stats)]),
    "tpcf_count_patches": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int,
                                          ctypes.POINTER(tpcf_stats)]),
    "tpcf_estimate": (ctypes.c_int, [_u64p, _u64p, _u64p, ctypes.c_int, _u64, _u64, ctypes.c_int, _dp]),
    "tpcf_correlate": (ctypes.c_int, [_vp, _vp, _u64, _vp, _u64, _dp, ctypes.c_int, ctypes.c_int, _vp,
                                      _u64p, _u64p, _u64p, _dp, ctypes.POINTER(tpcf_stats)]),
    "tpcf_plan_coverage": (ctypes.c_int64, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int, ctypes.c_uint32,
                                            ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.POINTER(ctypes.c_uint32), _u64p]),
    "tpcf_debug_fail_alloc_after": (None, [ctypes.c_int]),
    "tpcf_debug_noalloc_grid": (None, [ctypes.c_int]),
    "tpcf_fp32_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp]),
    "tpcf_count_auto_noalloc": (ctypes.c_int, [_vp, _u64, _dp, ctypes.c_int, _vp, _vp]),
    "tpcf_jackknife": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, _u64p, _dp, _dp,
                                      ctypes.POINTER(tpcf_stats)]),
    "tpcf_submit": (ctypes.c_int, [_vp, ctypes.POINTER(tpcf_job), _u64p]),
    "tpcf_poll": (ctypes.c_int, [_vp, _u64, ctypes.c_int, ctypes.POINTER(tpcf_result)]),
    "tpcf_cancel": (ctypes.c_int, [_vp, _u64]),
    "tpcf_graph_create": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "tpcf_graph_launch": (ctypes.c_int, [_vp, _vp]),
    "tpcf_graph_stats": (ctypes.c_int, [_vp, ctypes.POINTER(tpcf_stats)]),
    "tpcf_graph_destroy": (ctypes.c_int, [_vp]),
}


def library_path() -> str:
    return _build.LIB


def load():
    """Load libtpcf.so (built beforehand); raises ImportError if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise ImportError(f"{path} is missing: build the CUDA library first "
                                  "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def tpcf_strerror(status: int) -> str:
    return load().tpcf_strerror(status).decode()


def strerror(status: int) -> str:
    try:
        return tpcf_strerror(status)
    except ImportError:
        return "status"


def tpcf_last_error(ctx: int) -> str:
    return load().tpcf_last_error(ctx).decode()


def _check(rc: int, where: str, ctx=None):
    if rc != TPCF_OK:
        detail = load().tpcf_last_error(ctx).decode() if ctx else ""
        raise TpcfError(rc, where, detail)


# ------------------------------------------------------------------ marshalling
def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _where_ptr(x, dtype):
    """(where, pointer, keepalive) for a numpy array or torch tensor of `dtype`."""
    if _is_torch(x):
        import torch
        tdt = {np.float64: torch.float64, np.uint64: torch.int64}[dtype]
        t = x if x.dtype == tdt else x.to(tdt)
        t = t.contiguous()
        return (TPCF_DEVICE if t.is_cuda else TPCF_HOST), t.data_ptr(), t
    a = np.ascontiguousarray(x, dtype=dtype)
    return TPCF_HOST, a.ctypes.data, a


# ------------------------------------------------------------------ C ABI, same names
def tpcf_config_default() -> tpcf_config:
    cfg = tpcf_config()
    load().tpcf_config_default(ctypes.byref(cfg))
    return cfg


def tpcf_version() -> int:
    return load().tpcf_version()


def tpcf_kernel_launches(ctx: int) -> int:
    return int(load().tpcf_kernel_launches(ctx))


def tpcf_create(cfg: tpcf_config | None = None) -> int:
    h = _vp()
    rc = load().tpcf_create(ctypes.byref(h), ctypes.byref(cfg) if cfg is not None else None)
    _check(rc, "tpcf_create")
    return h.value


def tpcf_destroy(ctx: int) -> None:
    _check(load().tpcf_destroy(ctx), "tpcf_destroy")


def tpcf_catalog_create(ctx: int, xyz, stream=None, offsets=None) -> int:
    """Catalog from an (n, 3) float64 array of unit vectors (numpy or torch)."""
    where, ptr, keep = _where_ptr(xyz, np.float64)
    shape = tuple(keep.shape)
    if len(shape) != 2 or (shape[0] and shape[1] != 3):
        raise ValueError("xyz must be an (n, 3) array")
    n = shape[0]
    h = _vp()
    if offsets is None:
        rc = load().tpcf_catalog_create(ctx, ptr, n, where, _stream_ptr(stream), ctypes.byref(h))
        _check(rc, "tpcf_catalog_create", ctx)
    else:
        off = np.ascontiguousarray(offsets, dtype=np.uint64)
        rc = load().tpcf_catalog_create_segmented(ctx, ptr, n, where,
                                                  off.ctypes.data_as(_u64p), len(off) - 1,
                                                  _stream_ptr(stream), ctypes.byref(h))
        _check(rc, "tpcf_catalog_create_segmented", ctx)
    return h.value


def tpcf_catalog_create_segmented(ctx: int, xyz, offsets, stream=None) -> int:
    return tpcf_catalog_create(ctx, xyz, stream, offsets)


def tpcf_catalog_create_3d(ctx: int, xyz, stream=None, offsets=None) -> int:
    """3-D catalog from an (n, 3) float64 array of points (numpy or torch)."""
    where, ptr, keep = _where_ptr(xyz, np.float64)
    shape = tuple(keep.shape)
    if len(shape) != 2 or (shape[0] and shape[1] != 3):
        raise ValueError("xyz must be an (n, 3) array")
    h = _vp()
    off = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.uint64)
    rc = load().tpcf_catalog_create_3d(ctx, ptr, shape[0], where,
                                       off.ctypes.data_as(_u64p) if off is not None else None,
                                       len(off) - 1 if off is not None else 0, _stream_ptr(stream), ctypes.byref(h))
    _check(rc, "tpcf_catalog_create_3d", ctx)
    return h.value


def tpcf_catalog_destroy(cat: int) -> None:
    _check(load().tpcf_catalog_destroy(cat), "tpcf_catalog_destroy")


def tpcf_catalog_size(cat: int) -> int:
    return int(load().tpcf_catalog_size(cat))


def tpcf_bins_create(ctx: int, edges_rad) -> int:
    e = np.ascontiguousarray(edges_rad, dtype=np.float64)
    h = _vp()
    rc = load().tpcf_bins_create(ctx, e.ctypes.data_as(_dp), len(e), ctypes.byref(h))
    _check(rc, "tpcf_bins_create", ctx)
    return h.value


def tpcf_bins_create_3d(ctx: int, edges) -> int:
    """3-D bins from distance edges."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    h = _vp()
    _check(load().tpcf_bins_create_3d(ctx, e.ctypes.data_as(_dp), len(e), ctypes.byref(h)), "tpcf_bins_create_3d", ctx)
    return h.value


def tpcf_bins_thresholds_3d(edges):
    """(S, verified) for 3-D distance edges; host-only, no GPU needed."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    sq = np.empty(len(e), np.float64)
    ver = np.empty(len(e), np.int32)
    _check(load().tpcf_bins_thresholds_3d(e.ctypes.data_as(_dp), len(e), sq.ctypes.data_as(_dp),
                                          ver.ctypes.data_as(ctypes.POINTER(ctypes.c_int))), "tpcf_bins_thresholds_3d")
    return sq, ver


def tpcf_bins_destroy(bins: int) -> None:
    _check(load().tpcf_bins_destroy(bins), "tpcf_bins_destroy")


def tpcf_bins_thresholds(edges_rad, guard_band: float = 0.0):
    """(C, lo, hi, verified) for the edges; host-only, no GPU needed."""
    e = np.ascontiguousarray(edges_rad, dtype=np.float64)
    n = len(e)
    c = np.empty(n, np.float64)
    lo = np.empty(n, np.float32)
    hi = np.empty(n, np.float32)
    ver = np.empty(n, np.int32)
    rc = load().tpcf_bins_thresholds(e.ctypes.data_as(_dp), n, guard_band, c.ctypes.data_as(_dp),
                                     lo.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                     hi.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                     ver.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    _check(rc, "tpcf_bins_thresholds")
    return c, lo, hi, ver


def _out(nbins_plus2: int, out, like_device: bool):
    if out is None:
        if like_device:
            import torch
            return torch.empty(nbins_plus2, dtype=torch.int64, device="cuda")
        return np.empty(nbins_plus2, dtype=np.uint64)
    return out


def _hist_args(outs):
    wheres, ptrs = set(), []
    for o in outs:
        w, p, _ = _where_ptr(o, np.uint64)
        if _is_torch(o) and not o.is_contiguous():
            raise ValueError("output tensors must be contiguous")
        if not _is_torch(o) and not (isinstance(o, np.ndarray) and o.dtype == np.uint64
                                     and o.flags.c_contiguous):
            raise ValueError("output arrays must be contiguous uint64 numpy arrays")
        wheres.add(w)
        ptrs.append(p)
    if len(wheres) != 1:
        raise ValueError("all outputs must live on the same side (host or device)")
    return wheres.pop(), ptrs


def tpcf_count_auto(ctx: int, cat: int, bins: int, nedges: int, stream=None, out=None,
                    device_out: bool = False, stats: bool = False):
    out = _out(nedges + 1, out, device_out)
    where, (p,) = _hist_args([out])
    st = tpcf_stats() if (stats and where == TPCF_HOST) else None
    rc = load().tpcf_count_auto(ctx, cat, bins, _stream_ptr(stream), p, where,
                                ctypes.byref(st) if st is not None else None)
    _check(rc, "tpcf_count_auto", ctx)
    return (out, st.as_dict()) if st is not None else out


def tpcf_count_cross(ctx: int, d: int, r: int, bins: int, nedges: int, stream=None, out=None,
                     device_out: bool = False, stats: bool = False):
    out = _out(nedges + 1, out, device_out)
    where, (p,) = _hist_args([out])
    st = tpcf_stats() if (stats and where == TPCF_HOST) else None
    rc = load().tpcf_count_cross(ctx, d, r, bins, _stream_ptr(stream), p, where,
                                 ctypes.byref(st) if st is not None else None)
    _check(rc, "tpcf_count_cross", ctx)
    return (out, st.as_dict()) if st is not None else out


def tpcf_count_all(ctx: int, d: int, r: int, bins: int, nedges: int, stream=None, outs=None,
                   device_out: bool = False, stats: bool = False):
    """(dd, dr, rr) histograms in one launch."""
    outs = outs or tuple(_out(nedges + 1, None, device_out) for _ in range(3))
    where, (pdd, pdr, prr) = _hist_args(list(outs))
    st = tpcf_stats() if (stats and where == TPCF_HOST) else None
    rc = load().tpcf_count_all(ctx, d, r, bins, _stream_ptr(stream), pdd, pdr, prr, where,
                               ctypes.byref(st) if st is not None else None)
    _check(rc, "tpcf_count_all", ctx)
    return (tuple(outs), st.as_dict()) if st is not None else tuple(outs)


def tpcf_count_patches(ctx: int, d: int, r: int, bins: int, nedges: int, npatch: int, stream=None,
                       out=None, device_out: bool = False, stats: bool = False):
    """Per-patch (DD, DR, RR) of segmented catalogs: array (npatch, 3, nedges + 1)."""
    if out is None:
        if device_out:
            import torch
            out = torch.empty((npatch, 3, nedges + 1), dtype=torch.int64, device="cuda")
        else:
            out = np.empty((npatch, 3, nedges + 1), dtype=np.uint64)
    where, (p,) = _hist_args([out])
    st = tpcf_stats() if (stats and where == TPCF_HOST) else None
    rc = load().tpcf_count_patches(ctx, d, r, bins, _stream_ptr(stream), p, where,
                                   ctypes.byref(st) if st is not None else None)
    _check(rc, "tpcf_count_patches", ctx)
    return (out, st.as_dict()) if st is not None else out


def tpcf_estimate(dd, dr, rr, nd: int, nr: int, estimator: int = TPCF_LS_EXACT) -> np.ndarray:
    """w(theta) from per-bin counts (no underflow/overflow entries)."""
    a = [np.ascontiguousarray(x, dtype=np.uint64) for x in (dd, dr, rr)]
    nb = len(a[0])
    w = np.empty(nb, np.float64)
    rc = load().tpcf_estimate(*(x.ctypes.data_as(_u64p) for x in a), nb, nd, nr, estimator,
                              w.ctypes.data_as(_dp))
    _check(rc, "tpcf_estimate")
    return w


def tpcf_correlate(ctx: int, d_xyz, r_xyz, edges_rad, estimator: int = TPCF_LS_EXACT, stream=None,
                   stats: bool = False):
    """Host arrays in, (dd, dr, rr, w) out, in one call."""
    d = np.ascontiguousarray(d_xyz, dtype=np.float64)
    r = np.ascontiguousarray(r_xyz, dtype=np.float64)
    e = np.ascontiguousarray(edges_rad, dtype=np.float64)
    ne = len(e)
    dd, dr, rr = (np.empty(ne + 1, np.uint64) for _ in range(3))
    w = np.empty(ne - 1, np.float64)
    st = tpcf_stats() if stats else None
    rc = load().tpcf_correlate(ctx, d.ctypes.data, len(d), r.ctypes.data, len(r), e.ctypes.data_as(_dp),
                               ne, estimator, _stream_ptr(stream), dd.ctypes.data_as(_u64p),
                               dr.ctypes.data_as(_u64p), rr.ctypes.data_as(_u64p), w.ctypes.data_as(_dp),
                               ctypes.byref(st) if st is not None else None)
    _check(rc, "tpcf_correlate", ctx)
    return (dd, dr, rr, w, st.as_dict()) if st is not None else (dd, dr, rr, w)


def tpcf_plan_coverage(na: int, nb: int, auto_mode: bool, I: int, Jc: int, J: int, with_counts=True,
                       shard_index: int = 0, shard_count: int = 0):
    counts = np.zeros(na * nb, np.uint32) if with_counts else None
    pairs = ctypes.c_uint64(0)
    items = load().tpcf_plan_coverage(na, nb, int(auto_mode), I, Jc, J, shard_index, shard_count,
                                      counts.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
                                      if counts is not None else None, ctypes.byref(pairs))
    if items < 0:
        raise ValueError("bad plan sizes")
    return items, int(pairs.value), (counts.reshape(na, nb) if counts is not None else None)


def tpcf_count_auto_noalloc(xyz_dev, edges_rad, out_dev, stream=None) -> None:
    """Auto-count histogram without any allocation (see include/tpcf.h).

    ``xyz_dev``: CUDA tensor (n, 3) float64; ``out_dev``: CUDA tensor of
    len(edges) + 1 int64 (uint64 bit patterns), written in stream order.
    """
    if not (_is_torch(xyz_dev) and xyz_dev.is_cuda and _is_torch(out_dev) and out_dev.is_cuda):
        raise ValueError("xyz_dev and out_dev must be CUDA tensors")
    import torch
    if xyz_dev.dtype != torch.float64 or not xyz_dev.is_contiguous() or xyz_dev.dim() != 2 \
            or xyz_dev.shape[1] != 3:
        raise ValueError("xyz_dev must be a contiguous (n, 3) float64 tensor")
    e = np.ascontiguousarray(edges_rad, dtype=np.float64)
    if out_dev.dtype != torch.int64 or not out_dev.is_contiguous() or out_dev.numel() != len(e) + 1:
        raise ValueError("out_dev must be a contiguous int64 tensor of len(edges) + 1")
    rc = load().tpcf_count_auto_noalloc(xyz_dev.data_ptr(), xyz_dev.shape[0], e.ctypes.data_as(_dp), len(e),
                                        _stream_ptr(stream), out_dev.data_ptr())
    _check(rc, "tpcf_count_auto_noalloc")


def tpcf_jackknife(ctx: int, d: int, r: int, bins: int, nedges: int, npatch: int, stream=None,
                   estimator: int = TPCF_LS_EXACT, stats: bool = False):
    """Leave-one-out histograms (npatch, 3, nedges + 1), w of each resampling
    (npatch, nedges - 1) and their covariance (nedges - 1, nedges - 1)."""
    nb = nedges - 1
    loo = np.empty((npatch, 3, nedges + 1), np.uint64)
    w = np.empty((npatch, nb), np.float64)
    cov = np.empty((nb, nb), np.float64) if npatch >= 2 else None
    st = tpcf_stats() if stats else None
    rc = load().tpcf_jackknife(ctx, d, r, bins, _stream_ptr(stream), estimator, loo.ctypes.data_as(_u64p),
                               w.ctypes.data_as(_dp), cov.ctypes.data_as(_dp) if cov is not None else None,
                               ctypes.byref(st) if st is not None else None)
    _check(rc, "tpcf_jackknife", ctx)
    out = (loo, w, cov)
    return out + (st.as_dict(),) if st is not None else out


def tpcf_submit(ctx: int, d_xyz, r_xyz, edges_rad, estimator: int = TPCF_LS_EXACT) -> int:
    """Queue a correlation job (host arrays, copied by the call); returns its id."""
    d = np.ascontiguousarray(d_xyz, dtype=np.float64).reshape(-1, 3)
    r = np.ascontiguousarray(r_xyz, dtype=np.float64).reshape(-1, 3)
    e = np.ascontiguousarray(edges_rad, dtype=np.float64)
    job = tpcf_job(d.ctypes.data, len(d), r.ctypes.data, len(r), e.ctypes.data, len(e), estimator)
    jid = ctypes.c_uint64(0)
    _check(load().tpcf_submit(ctx, ctypes.byref(job), ctypes.byref(jid)), "tpcf_submit", ctx)
    return int(jid.value)


class JobResult(dict):
    """Result of a finished job: dd, dr, rr, w and the timings of tpcf_result."""


def tpcf_poll(ctx: int, job_id: int, nedges: int, timeout_ms: int = -1, raise_on_error: bool = True):
    """The job's JobResult, or None while it is not finished (TPCF_EAGAIN).

    A finished job that failed raises TpcfError (or, with raise_on_error=False,
    comes back with its status and no histograms)."""
    dd, dr, rr = (np.zeros(nedges + 1, np.uint64) for _ in range(3))
    w = np.full(max(nedges - 1, 0), np.nan)
    res = tpcf_result(dd.ctypes.data, dr.ctypes.data, rr.ctypes.data, w.ctypes.data)
    rc = load().tpcf_poll(ctx, job_id, timeout_ms, ctypes.byref(res))
    if rc == TPCF_EAGAIN:
        return None
    if rc == TPCF_ENOTFOUND or (rc != TPCF_OK and raise_on_error):
        _check(rc, "tpcf_poll", ctx)
    out = JobResult(status=rc, submit_ms=res.submit_ms, queued_ms=res.queued_ms, run_ms=res.run_ms,
                    latency_ms=res.latency_ms,
                    kernel_ms=res.kernel_ms, pairs=int(res.pairs))
    if rc == TPCF_OK:
        out.update(dd=dd, dr=dr, rr=rr, w=w)
    return out


def tpcf_cancel(ctx: int, job_id: int) -> None:
    _check(load().tpcf_cancel(ctx, job_id), "tpcf_cancel", ctx)


def tpcf_graph_create(ctx: int, kind: int, d: int, r: int | None, bins: int, out_dev) -> int:
    """Capture a counting call into a CUDA graph writing the CUDA tensor out_dev."""
    if not (_is_torch(out_dev) and out_dev.is_cuda and out_dev.is_contiguous()):
        raise ValueError("out_dev must be a contiguous CUDA tensor")
    h = _vp()
    _check(load().tpcf_graph_create(ctx, kind, d, r, bins, out_dev.data_ptr(), ctypes.byref(h)),
           "tpcf_graph_create", ctx)
    return h.value


def tpcf_graph_launch(graph: int, stream=None, ctx: int | None = None) -> None:
    _check(load().tpcf_graph_launch(graph, _stream_ptr(stream)), "tpcf_graph_launch", ctx)


def tpcf_graph_stats(graph: int, ctx: int | None = None) -> dict:
    st = tpcf_stats()
    _check(load().tpcf_graph_stats(graph, ctypes.byref(st)), "tpcf_graph_stats", ctx)
    return st.as_dict()


def tpcf_graph_destroy(graph: int) -> None:
    _check(load().tpcf_graph_destroy(graph), "tpcf_graph_destroy")


def tpcf_debug_fail_alloc_after(n: int) -> None:
    load().tpcf_debug_fail_alloc_after(n)


def tpcf_debug_noalloc_grid(blocks: int) -> None:
    load().tpcf_debug_noalloc_grid(blocks)


def tpcf_fp32_peak(device: int = 0, packed: bool = False) -> float:
    """Measured FP32 FMA throughput of the device in TFLOP/s (see include/tpcf.h)."""
    v = ctypes.c_double(0.0)
    _check(load().tpcf_fp32_peak(device, 1 if packed else 0, ctypes.byref(v)), "tpcf_fp32_peak")
    return v.value


# ------------------------------------------------------------------ object layer
class Context:
    """Owns a tpcf_ctx; catalogs and bins created through it are freed with it."""

    def __init__(self, device: int = 0, precision: int = TPCF_SCREEN_RECHECK, **overrides):
        cfg = tpcf_config_default()
        cfg.device = device
        cfg.precision = precision
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.config = cfg
        self.handle = tpcf_create(cfg)
        self._owned: list[tuple[str, int]] = []

    def catalog(self, xyz, stream=None, offsets=None) -> "Catalog":
        """tpcf_catalog_create[_segmented]: (n, 3) float64 unit vectors, host array or CUDA tensor;
        offsets (P + 1 ascending, from 0 to n) make a segmented catalog for patches and the jackknife."""
        h = tpcf_catalog_create(self.handle, xyz, stream, offsets)
        c = Catalog(self, h, tpcf_catalog_size(h), 0 if offsets is None else len(offsets) - 1)
        self._owned.append(("cat", h))
        return c

    def catalog3d(self, xyz, stream=None, offsets=None) -> "Catalog":
        """tpcf_catalog_create_3d: (n, 3) float64 points of the 3-D variant (finite, |x| <= 1e28)."""
        h = tpcf_catalog_create_3d(self.handle, xyz, stream, offsets)
        c = Catalog(self, h, tpcf_catalog_size(h), 0 if offsets is None else len(offsets) - 1)
        self._owned.append(("cat", h))
        return c

    def bins3d(self, edges) -> "Bins":
        """tpcf_bins_create_3d: distance edges (B + 1 increasing, finite, the last in (0, 1e18])."""
        h = tpcf_bins_create_3d(self.handle, edges)
        self._owned.append(("bins", h))
        return Bins(self, h, len(edges))

    def bins(self, edges_rad) -> "Bins":
        """tpcf_bins_create: angular edges in radians (B + 1 strictly increasing, in [0, pi])."""
        h = tpcf_bins_create(self.handle, edges_rad)
        self._owned.append(("bins", h))
        return Bins(self, h, len(edges_rad))

    def count_auto(self, cat: "Catalog", bins: "Bins", stream=None, out=None, device_out=False, stats=False):
        """tpcf_count_auto: DD or RR over pairs i < j; B + 2 uint64 [underflow, bins, overflow]."""
        return tpcf_count_auto(self.handle, cat.handle, bins.handle, bins.nedges, stream, out, device_out, stats)

    def count_cross(self, d: "Catalog", r: "Catalog", bins: "Bins", stream=None, out=None, device_out=False,
                    stats=False):
        """tpcf_count_cross: DR over all ordered pairs (i in d, j in r)."""
        return tpcf_count_cross(self.handle, d.handle, r.handle, bins.handle, bins.nedges, stream, out,
                                device_out, stats)

    def count_all(self, d: "Catalog", r: "Catalog", bins: "Bins", stream=None, outs=None, device_out=False,
                  stats=False):
        """tpcf_count_all: (DD, DR, RR) in one fused launch."""
        return tpcf_count_all(self.handle, d.handle, r.handle, bins.handle, bins.nedges, stream, outs,
                              device_out, stats)

    def count_patches(self, d: "Catalog", r: "Catalog", bins: "Bins", stream=None, out=None, device_out=False,
                      stats=False):
        """tpcf_count_patches: (P, 3, B + 2) per-patch DD, DR, RR of two segmented catalogs, one launch."""
        return tpcf_count_patches(self.handle, d.handle, r.handle, bins.handle, bins.nedges, d.npatch, stream, out,
                                  device_out, stats)

    def jackknife(self, d: "Catalog", r: "Catalog", bins: "Bins", stream=None, estimator=TPCF_LS_EXACT, stats=False):
        """tpcf_jackknife: leave-one-out histograms (P, 3, B + 2), w (P, B) and its covariance (B, B)."""
        return tpcf_jackknife(self.handle, d.handle, r.handle, bins.handle, bins.nedges, d.npatch, stream, estimator,
                              stats)

    def correlate(self, d_xyz, r_xyz, edges_rad, estimator=TPCF_LS_EXACT, stream=None, stats=False):
        """tpcf_correlate: host arrays in, (DD, DR, RR, w) out."""
        return tpcf_correlate(self.handle, d_xyz, r_xyz, edges_rad, estimator, stream, stats)

    def submit(self, d_xyz, r_xyz, edges_rad, estimator=TPCF_LS_EXACT) -> int:
        """tpcf_submit: queue a correlation job on the context's job server; returns its id."""
        return tpcf_submit(self.handle, d_xyz, r_xyz, edges_rad, estimator)

    def poll(self, job_id: int, nedges: int, timeout_ms: int = -1, raise_on_error: bool = True):
        """tpcf_poll: wait up to timeout_ms (0: do not wait, < 0: no limit) for a job; its histograms, w, timings."""
        return tpcf_poll(self.handle, job_id, nedges, timeout_ms, raise_on_error)

    def cancel(self, job_id: int) -> None:
        """tpcf_cancel: cancel a queued job."""
        tpcf_cancel(self.handle, job_id)

    def graph(self, kind: int, d: "Catalog", r: "Catalog | None", bins: "Bins", out_dev=None) -> "Graph":
        """A captured counting graph (see include/tpcf.h); out_dev is allocated when None."""
        hs = bins.nedges + 1
        if out_dev is None:
            import torch
            shape = {TPCF_GRAPH_AUTO: (hs,), TPCF_GRAPH_CROSS: (hs,), TPCF_GRAPH_ALL: (3, hs),
                     TPCF_GRAPH_PATCHES: (d.npatch, 3, hs)}[kind]
            out_dev = torch.empty(shape, dtype=torch.int64, device="cuda")
        h = tpcf_graph_create(self.handle, kind, d.handle, r.handle if r is not None else None, bins.handle, out_dev)
        g = Graph(self, h, out_dev)
        self._owned.append(("graph", h))
        return g

    _DESTROY = {"cat": "tpcf_catalog_destroy", "bins": "tpcf_bins_destroy", "graph": "tpcf_graph_destroy"}

    def free(self, obj) -> None:
        """Destroy a catalog, bins or graph made by this context before the context closes."""
        kind = "cat" if isinstance(obj, Catalog) else ("graph" if isinstance(obj, Graph) else "bins")
        if (kind, obj.handle) in self._owned:
            self._owned.remove((kind, obj.handle))
            globals()[self._DESTROY[kind]](obj.handle)

    def close(self) -> None:
        """Destroy everything this context made, then the context."""
        if self.handle:
            for kind, h in reversed(self._owned):
                globals()[self._DESTROY[kind]](h)
            self._owned.clear()
            tpcf_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Catalog:
    def __init__(self, ctx: Context, handle: int, n: int, npatch: int = 0):
        self.ctx, self.handle, self.n, self.npatch = ctx, handle, n, npatch


class Bins:
    def __init__(self, ctx: Context, handle: int, nedges: int):
        self.ctx, self.handle, self.nedges = ctx, handle, nedges


class Graph:
    def __init__(self, ctx: Context, handle: int, out):
        self.ctx, self.handle, self.out = ctx, handle, out

    def launch(self, stream=None) -> None:
        tpcf_graph_launch(self.handle, stream, self.ctx.handle)

    def stats(self) -> dict:
        return tpcf_graph_stats(self.handle, self.ctx.handle)
