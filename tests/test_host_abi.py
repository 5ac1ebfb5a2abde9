"""Host-side checks of the C-ABI library (no GPU): it loads, exports every
symbol ``include/tpcf.h`` declares, and its host logic (thresholds, work
plan, estimator, argument validation) is right."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_1204_6630_gb300 import build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tpcf():
    build.build()
    from paper_1204_6630_gb300 import tpcf as t
    t.load()
    return t


def header_functions():
    text = open(os.path.join(ROOT, "include", "tpcf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tpcf_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(tpcf):
    names = header_functions()
    assert len(names) >= 20
    lib = tpcf.load()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding wraps each one under the same name
    assert not [n for n in names if not hasattr(tpcf, n)]


def test_strerror_and_version(tpcf):
    assert tpcf.tpcf_version() >= 100
    assert tpcf.strerror(0) == "ok"
    assert "timed out" in tpcf.strerror(tpcf.TPCF_ETIMEOUT)


def test_context_creation_without_gpu_fails_cleanly(tpcf):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tpcf.TpcfError) as ei:
        tpcf.tpcf_create(None)
    assert ei.value.status == tpcf.TPCF_ECUDA


# ------------------------------------------------------------------ thresholds
@pytest.mark.parametrize("edges", [synth.log_edges(0.01, 10.0, 64), synth.linear_edges(0.0, 10.0, 40),
                                   synth.log_edges(0.005, 2.0, 80), np.linspace(0.0, math.pi, 19)])
def test_thresholds_define_the_oracle_predicate(tpcf, edges):
    # C_k is the largest double d with acos(d) >= t_k (host acos, same libm as
    # the oracle): the predicate holds at C_k and fails at the next double up.
    c, lo, hi, ver = tpcf.tpcf_bins_thresholds(edges)
    # The neighbour scan cannot cover 4 ulps of t when C_k is within ~1e-10 of
    # zero (t ~ pi/2): there the doubles are too dense; such edges are flagged.
    assert np.all(ver[np.abs(edges - math.pi / 2) > 1e-6] == 1)
    for t, ck in zip(edges, c):
        if t == 0.0:
            assert ck == math.inf
            continue
        assert math.acos(max(-1.0, min(1.0, ck))) >= t
        up = math.nextafter(ck, math.inf)
        if up <= 1.0:
            assert math.acos(up) < t
    assert np.all(np.diff(c) < 0)
    g = 9.0 * 2.0 ** -24
    fin = np.isfinite(c)
    assert np.all(lo[fin].astype(np.float64) <= c[fin] - g)
    assert np.all(hi[fin].astype(np.float64) >= c[fin] + g)


def test_thresholds_agree_with_exact_cosines(tpcf):
    # Independently of libm: the exact threshold is the largest double <= cos(t)
    # (mpmath, 40 digits).  The library follows the host acos, whose result is
    # rounded to a double: doubles whose exact angle is within about half an
    # ulp of t_k can land on either side.  So the two thresholds may differ,
    # but only by doubles whose exact angle is within 1e-12 rad of the edge.
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    edges = np.concatenate([synth.log_edges(0.01, 10.0, 64), synth.linear_edges(12.0, 170.0, 40)])
    c, _, _, _ = tpcf.tpcf_bins_thresholds(edges)
    differ = 0
    for t, ck in zip(edges, c):
        exact = mp.cos(mp.mpf(float(t)))
        d = float(exact)
        if mp.mpf(d) > exact:
            d = math.nextafter(d, -math.inf)
        if d != ck:
            differ += 1
            lo, hi = sorted([d, ck])
            assert abs(mp.acos(mp.mpf(lo)) - mp.mpf(float(t))) < 1e-12
            assert abs(mp.acos(mp.mpf(hi)) - mp.mpf(float(t))) < 1e-12
    print(f"{differ} of {len(edges)} libm thresholds differ from the exact ones (all within 1e-12 rad)")


def test_bad_edges_rejected(tpcf):
    for bad in ([0.1], [0.2, 0.1], [0.1, 0.1], [-0.1, 0.2], [0.1, 4.0], [0.1, float("nan")]):
        with pytest.raises(tpcf.TpcfError) as ei:
            tpcf.tpcf_bins_thresholds(np.array(bad))
        assert ei.value.status == tpcf.TPCF_EINVAL
    with pytest.raises(tpcf.TpcfError):
        tpcf.tpcf_bins_thresholds(np.linspace(0.0, 1.0, 2000))


# ------------------------------------------------------------------ work plan
@pytest.mark.parametrize("auto", [True, False])
@pytest.mark.parametrize("shape", [(32, 32, 8), (32, 16, 8), (16, 64, 16), (64, 64, 64), (64, 16, 16),
                                   (128, 512, 64)])
@pytest.mark.parametrize("n", [1, 2, 7, 31, 32, 33, 100, 257])
def test_plan_covers_every_pair_once(tpcf, auto, shape, n):
    I, Jc, J = shape
    na, nb = (n, n) if auto else (n, n + 13)
    items, pairs, cnt = tpcf.tpcf_plan_coverage(na, nb, auto, I, Jc, J)
    want = np.triu(np.ones((na, nb), np.uint32), 1) if auto else np.ones((na, nb), np.uint32)
    np.testing.assert_array_equal(cnt, want)
    assert pairs == int(want.sum())


def test_plan_pair_totals_at_full_scale(tpcf):
    for n, I, Jc, J in ((1_000_000, 2048, 2048, 2048), (999_999, 1024, 4096, 512),
                        (4_000_000, 2048, 8192, 2048), (8_000_000, 4096, 1024, 1024)):
        items, pairs, _ = tpcf.tpcf_plan_coverage(n, n, True, I, Jc, J, with_counts=False)
        assert pairs == n * (n - 1) // 2
        items, pairs, _ = tpcf.tpcf_plan_coverage(n, n // 2 + 5, False, I, Jc, J, with_counts=False)
        assert pairs == n * (n // 2 + 5)


# ------------------------------------------------------------------ estimator
def test_library_estimator_matches_oracle_bitwise(tpcf):
    rng = np.random.default_rng(4)
    for nd, nr in ((1000, 2000), (8192, 8192), (1_000_000, 1_000_000), (3, 5)):
        nb = 40
        dd = rng.integers(0, nd * (nd - 1) // 2 // nb + 1, nb).astype(np.uint64)
        rr = rng.integers(0, nr * (nr - 1) // 2 // nb + 1, nb).astype(np.uint64)
        dr = rng.integers(0, nd * nr // nb + 1, nb).astype(np.uint64)
        rr[3] = 0
        for est in (tpcf.TPCF_LS_EXACT, tpcf.TPCF_LS_PAPER):
            a = tpcf.tpcf_estimate(dd, dr, rr, nd, nr, est)
            b = oracle.estimate(dd, dr, rr, nd, nr, est)
            assert np.array_equal(a, b, equal_nan=True)


def test_estimator_rejects_bad_sizes(tpcf):
    with pytest.raises(tpcf.TpcfError):
        tpcf.tpcf_estimate([1], [1], [1], 1, 5)
    with pytest.raises(tpcf.TpcfError):
        tpcf.tpcf_estimate([1], [1], [1], 5, 5, estimator=7)


def test_server_entry_points_reject_null_context():
    from paper_1204_6630_gb300 import tpcf
    lib = tpcf.load()
    job = tpcf.tpcf_job()
    jid = ctypes.c_uint64(0)
    assert lib.tpcf_submit(None, ctypes.byref(job), ctypes.byref(jid)) == tpcf.TPCF_EINVAL
    assert lib.tpcf_poll(None, 1, 0, None) == tpcf.TPCF_EINVAL
    assert lib.tpcf_cancel(None, 1) == tpcf.TPCF_EINVAL


def test_graph_entry_points_reject_null():
    from paper_1204_6630_gb300 import tpcf
    lib = tpcf.load()
    h = ctypes.c_void_p()
    assert lib.tpcf_graph_create(None, 0, None, None, None, None, ctypes.byref(h)) == tpcf.TPCF_EINVAL
    assert lib.tpcf_graph_launch(None, None) == tpcf.TPCF_EINVAL
    assert lib.tpcf_graph_stats(None, None) == tpcf.TPCF_EINVAL
    assert lib.tpcf_graph_destroy(None) == tpcf.TPCF_EINVAL


def test_3d_thresholds_are_the_smallest_squares_reaching_each_edge():
    from paper_1204_6630_gb300 import tpcf
    rng = np.random.default_rng(9)
    edges = np.concatenate([[0.0], np.sort(rng.uniform(1e-3, 1e3, 60)), [5.0, 1e18]])
    edges = np.unique(edges)
    S, ver = tpcf.tpcf_bins_thresholds_3d(edges)
    assert S[0] == 0.0 and ver.all()
    for r, s in zip(edges[1:], S[1:]):
        assert math.sqrt(s) >= r
        assert math.sqrt(np.nextafter(s, 0.0)) < r
    s5 = S[list(edges).index(5.0)]
    assert s5 <= 25.0 and math.sqrt(s5) == 5.0  # doubles just below 25 already round up to 5
    with pytest.raises(tpcf.TpcfError):
        tpcf.tpcf_bins_thresholds_3d(np.array([1.0, 0.5]))


def test_binding_structs_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets
    (a C program compiled against include/tpcf.h prints them)."""
    import subprocess
    from paper_1204_6630_gb300 import tpcf as T
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = [T.tpcf_config, T.tpcf_stats, T.tpcf_job, T.tpcf_result]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tpcf.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                         text=True).stdout.splitlines())
    for st in structs:
        n = st.__name__
        assert int(got[n]) == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert int(got[f"{n}.{f}"]) == getattr(st, f).offset, f"{n}.{f}"
