"""Python access to the plain CPU oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  The CUDA library never imports it.

The C source is compiled on first use with ``gcc -O2 -ffp-contract=off
-fno-fast-math`` so that every binary64 operation is rounded exactly as
written (no fused multiply-add, no reassociation).

Functions follow the paper's definitions (Section 1, Eq. 1; Section 3):
``count_auto`` (DD or RR, unordered pairs i < j), ``count_cross`` (DR, all
ordered pairs) and ``estimate`` (Landy-Szalay w(theta)).  Histograms have
``len(edges) + 1`` entries: [underflow, bin 0 .. bin B-1, overflow].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fno-builtin", "-fPIC", "-shared"]

LS_EXACT = 0
LS_PAPER = 1


def build(src: str = _SRC, out: str = _LIB, force: bool = False) -> str:
    """Compile ``src`` into the shared library ``out`` (if stale) and return its path."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(out), exist_ok=True)
        tmp = f"{out}.{os.getpid()}.tmp"
        subprocess.run(["gcc", *CFLAGS, src, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, out)
    return out


def _bind(lib):
    u64p = ctypes.POINTER(ctypes.c_uint64)
    dp = ctypes.POINTER(ctypes.c_double)
    u64 = ctypes.c_uint64
    lib.oracle_count_auto_rows.argtypes = [dp, u64, dp, ctypes.c_int, u64, u64, u64p]
    lib.oracle_count_cross_rows.argtypes = [dp, u64, dp, u64, dp, ctypes.c_int, u64, u64, u64p]
    lib.oracle_estimate.argtypes = [u64p, u64p, u64p, ctypes.c_int, u64, u64, ctypes.c_int, dp]
    lib.oracle_count_auto3_rows.argtypes = [dp, u64, dp, ctypes.c_int, u64, u64, u64p]
    lib.oracle_count_cross3_rows.argtypes = [dp, u64, dp, u64, dp, ctypes.c_int, u64, u64, u64p]
    lib.oracle_near_edge_rows.argtypes = [dp, u64, dp, u64, ctypes.c_int, dp, ctypes.c_int, ctypes.c_double,
                                          u64, u64, u64, u64p, dp, u64p]
    for f in (lib.oracle_count_auto_rows, lib.oracle_count_cross_rows, lib.oracle_estimate,
              lib.oracle_count_auto3_rows, lib.oracle_count_cross3_rows, lib.oracle_near_edge_rows):
        f.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load (building if needed) the oracle library; ``path`` loads another build."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _uptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _as_xyz(x) -> np.ndarray:
    a = np.ascontiguousarray(x, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("catalog must be an (n, 3) array")
    return a


def _row_splits(n_rows: int, weights, parts: int) -> list[tuple[int, int]]:
    """Cut [0, n_rows) into ``parts`` contiguous ranges of about equal work."""
    if parts <= 1 or n_rows == 0:
        return [(0, n_rows)]
    cum = np.concatenate([[0.0], np.cumsum(weights)])
    cuts = np.searchsorted(cum, np.linspace(0.0, cum[-1], parts + 1))
    cuts[0], cuts[-1] = 0, n_rows
    cuts = np.maximum.accumulate(cuts)
    return [(int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]


def count_auto(xyz, edges, threads: int = 1, lib=None, euclid: bool = False) -> np.ndarray:
    """DD or RR histogram over unordered pairs i < j (B + 2 uint64 entries).

    ``threads > 1`` splits the rows of the triangle across host threads (the
    C call releases the GIL) and sums the per-range histograms.  ``euclid``:
    the 3-D variant (Euclidean distances between arbitrary points, edges in
    the same length unit) instead of angles between unit vectors.
    """
    lib = lib or load()
    a = _as_xyz(xyz)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    n = a.shape[0]
    fn = lib.oracle_count_auto3_rows if euclid else lib.oracle_count_auto_rows

    def run(r):
        h = np.zeros(len(e) + 1, dtype=np.uint64)
        rc = fn(_dptr(a), n, _dptr(e), len(e), r[0], r[1], _uptr(h))
        if rc != 0:
            raise ValueError("oracle_count_auto: invalid arguments")
        return h

    ranges = _row_splits(n, n - 1 - np.arange(n, dtype=np.float64), threads)
    if len(ranges) == 1:
        return run(ranges[0])
    with ThreadPoolExecutor(len(ranges)) as ex:
        return np.sum(list(ex.map(run, ranges)), axis=0, dtype=np.uint64)


def count_cross(xyz_d, xyz_r, edges, threads: int = 1, lib=None, euclid: bool = False) -> np.ndarray:
    """DR histogram over all ordered pairs (i in D, j in R) (B + 2 uint64 entries); ``euclid`` as above."""
    lib = lib or load()
    d = _as_xyz(xyz_d)
    r_ = _as_xyz(xyz_r)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    nd, nr = d.shape[0], r_.shape[0]
    fn = lib.oracle_count_cross3_rows if euclid else lib.oracle_count_cross_rows

    def run(rg):
        h = np.zeros(len(e) + 1, dtype=np.uint64)
        rc = fn(_dptr(d), nd, _dptr(r_), nr, _dptr(e), len(e), rg[0], rg[1], _uptr(h))
        if rc != 0:
            raise ValueError("oracle_count_cross: invalid arguments")
        return h

    ranges = _row_splits(nd, np.ones(nd), threads)
    if len(ranges) == 1:
        return run(ranges[0])
    with ThreadPoolExecutor(len(ranges)) as ex:
        return np.sum(list(ex.map(run, ranges)), axis=0, dtype=np.uint64)


def near_edge_pairs(a, b, edges, auto: bool, tol: float = 1e-12, threads: int = 1, max_out: int = 1000,
                    lib=None):
    """Pairs whose angle lies within ``tol`` radians of a bin edge.

    ``auto``: unordered pairs i < j of catalog ``a`` (``b`` ignored); else every
    pair (i in a, j in b).  These are the pairs a different (correctly behaved)
    arc-cosine could put in a neighbouring bin.  Returns ``(count, pairs)`` with
    ``pairs`` a list of up to ``max_out`` ``(i, j, theta - t_m)`` tuples.
    """
    lib = lib or load()
    a = _as_xyz(a)
    b = a if auto else _as_xyz(b)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    na, nb = a.shape[0], b.shape[0]

    def run(rg):
        ij = np.zeros(2 * max(1, max_out), dtype=np.uint64)
        gap = np.zeros(max(1, max_out), dtype=np.float64)
        c = np.zeros(1, dtype=np.uint64)
        rc = lib.oracle_near_edge_rows(_dptr(a), na, _dptr(b), nb, 1 if auto else 0, _dptr(e), len(e), float(tol),
                                       rg[0], rg[1], max_out, _uptr(ij), _dptr(gap), _uptr(c))
        if rc != 0:
            raise ValueError("oracle_near_edge_rows: invalid arguments")
        k = int(min(int(c[0]), max_out))
        return int(c[0]), [(int(ij[2 * q]), int(ij[2 * q + 1]), float(gap[q])) for q in range(k)]

    weights = (na - 1 - np.arange(na, dtype=np.float64)) if auto else np.ones(na)
    ranges = _row_splits(na, weights, threads)
    if len(ranges) == 1:
        return run(ranges[0])
    with ThreadPoolExecutor(len(ranges)) as ex:
        parts = list(ex.map(run, ranges))
    pairs = [p for _, ps in parts for p in ps][:max_out]
    return sum(c for c, _ in parts), pairs


def estimate(dd, dr, rr, nd: int, nr: int, estimator: int = LS_EXACT, lib=None) -> np.ndarray:
    """Landy-Szalay w(theta) per bin (Eq. 1; see ``oracle_estimate`` for the two readings).

    ``dd``, ``dr``, ``rr`` are the per-bin counts without underflow/overflow.
    """
    lib = lib or load()
    dd = np.ascontiguousarray(dd, dtype=np.uint64)
    dr = np.ascontiguousarray(dr, dtype=np.uint64)
    rr = np.ascontiguousarray(rr, dtype=np.uint64)
    nb = len(dd)
    if len(dr) != nb or len(rr) != nb:
        raise ValueError("dd, dr and rr must have the same length")
    w = np.empty(nb, dtype=np.float64)
    rc = lib.oracle_estimate(_uptr(dd), _uptr(dr), _uptr(rr), nb, nd, nr, estimator, _dptr(w))
    if rc != 0:
        raise ValueError("oracle_estimate: invalid arguments")
    return w


def correlation(data, rand, edges, estimator: int = LS_EXACT, threads: int = 1):
    """DD, DR, RR histograms and w(theta) for one data/random catalog pair."""
    dd = count_auto(data, edges, threads)
    rr = count_auto(rand, edges, threads)
    dr = count_cross(data, rand, edges, threads)
    w = estimate(dd[1:-1], dr[1:-1], rr[1:-1], len(data), len(rand), estimator)
    return dd, dr, rr, w


def jackknife(data, rand, data_offsets, rand_offsets, edges, estimator: int = LS_EXACT, threads: int = 1,
              euclid: bool = False):
    """Delete-one jackknife of the three histograms over the patches of a segmented catalog pair.

    Patch p holds ``data[data_offsets[p]:data_offsets[p+1]]`` and likewise for
    the randoms.  For each p the patch is removed and DD, DR and RR are counted
    again from scratch on what remains (the definition of the resampling, no
    shortcut); w of each resampling follows from ``estimate`` with the remaining
    point counts (NaN when fewer than 2 points remain), and the covariance is
    C_ab = (P - 1)/P sum_p (w_pa - mean_a)(w_pb - mean_b), the sums taken in
    patch order.  ``euclid``: the 3-D variant (distances).

    Returns ``(loo, w, cov)``: loo (P, 3, B + 2) uint64, w (P, B), cov (B, B).
    """
    data, rand = _as_xyz(data), _as_xyz(rand)
    doff = [int(x) for x in data_offsets]
    roff = [int(x) for x in rand_offsets]
    P = len(doff) - 1
    nb = len(edges) - 1
    loo = np.zeros((P, 3, nb + 2), dtype=np.uint64)
    w = np.full((P, nb), np.nan)
    for p in range(P):
        d = np.concatenate([data[:doff[p]], data[doff[p + 1]:]])
        r = np.concatenate([rand[:roff[p]], rand[roff[p + 1]:]])
        loo[p, 0] = count_auto(d, edges, threads, euclid=euclid)
        loo[p, 1] = count_cross(d, r, edges, threads, euclid=euclid)
        loo[p, 2] = count_auto(r, edges, threads, euclid=euclid)
        if len(d) >= 2 and len(r) >= 2:
            w[p] = estimate(loo[p, 0, 1:-1], loo[p, 1, 1:-1], loo[p, 2, 1:-1], len(d), len(r), estimator)
    cov = None
    if P >= 2:
        mean = [0.0] * nb
        for a in range(nb):
            s = 0.0
            for p in range(P):
                s += float(w[p, a])
            mean[a] = s / P
        f = (P - 1) / P
        cov = np.empty((nb, nb))
        for a in range(nb):
            for b in range(nb):
                s = 0.0
                for p in range(P):
                    s += (float(w[p, a]) - mean[a]) * (float(w[p, b]) - mean[b])
                cov[a, b] = f * s
    return loo, w, cov
