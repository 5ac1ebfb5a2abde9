"""Planted mistakes in the oracle must be caught by its pins.

Each case copies ``oracle/oracle.c``, plants one plausible mistake (a dropped
term, a transposed operand, a wrong sign, a wrong loop bound, a lost clamp,
an inclusive/exclusive edge swap, a wrong normaliser), compiles the copy into
a temporary library and runs a battery of the closed-form pins against it.
At least one pin must fail for every mutant, and all pins pass for the
unmodified source.  Mistakes are planted on the CPU only.
"""
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1204_6630_gb300 import synth
from tests.golden import FIXTURES, load_fixture

DEG = math.pi / 180.0
SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "drop_z_term": ("d = (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];",
                    "d = (a[0] * b[0] + a[1] * b[1]);"),
    "transposed_operand": ("a[1] * b[1]", "a[1] * b[0]"),
    "edge_exclusive": ("if (edges[m] <= theta)", "if (edges[m] < theta)"),
    "self_pairs_included": ("for (uint64_t j = i + 1; j < n; ++j)\n            hist[bin_of_angle(pair_angle(",
                            "for (uint64_t j = i; j < n; ++j)\n            hist[bin_of_angle(pair_angle("),
    "cross_skips_first": ("for (uint64_t j = 0; j < nr; ++j)\n            hist[bin_of_angle(pair_angle(",
                          "for (uint64_t j = 1; j < nr; ++j)\n            hist[bin_of_angle(pair_angle("),
    "3d_drop_z_term": ("return sqrt((dx * dx + dy * dy) + dz * dz);", "return sqrt(dx * dx + dy * dy);"),
    "3d_sum_not_difference": ("double dy = a[1] - b[1];", "double dy = a[1] + b[1];"),
    "3d_squared_distance": ("return sqrt((dx * dx + dy * dy) + dz * dz);", "return (dx * dx + dy * dy) + dz * dz;"),
    "3d_self_pairs_included": ("for (uint64_t j = i + 1; j < n; ++j)\n            hist[bin_of_angle(pair_distance(",
                               "for (uint64_t j = i; j < n; ++j)\n            hist[bin_of_angle(pair_distance("),
    "no_clamp": ("    if (d > 1.0)\n        d = 1.0;\n", ""),
    "estimator_sign": ("((ndd - 2.0 * ndr) + nrr)", "((ndd + 2.0 * ndr) + nrr)"),
    "dr_normaliser": ("double pairs_dr = (double)nd * (double)nr;",
                      "double pairs_dr = (double)nd * (double)nd;"),
    "paper_factor": ("((2.0 * q) * ((double)dr[k] / rr_ordered))",
                     "((q) * ((double)dr[k] / rr_ordered))"),
}


def _clamp_vector():
    rng = np.random.default_rng(11)
    for _ in range(100000):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        if (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2] > 1.0:
            return v
    return None


def battery(lib) -> list[str]:
    """Run the closed-form pins against ``lib``; return the names that failed."""
    failed = []

    def check(name, ok):
        if not ok:
            failed.append(name)

    for fx_name in FIXTURES:
        fx = load_fixture(fx_name)
        if fx["kind"] == "auto":
            got = oracle.count_auto(fx["a"], fx["edges"], lib=lib)
        else:
            got = oracle.count_cross(fx["a"], fx["b"], fx["edges"], lib=lib)
        check("golden:" + fx_name, np.array_equal(got, fx["hist"]))

    x = synth.octant_small(n=300).data
    e = synth.linear_edges(0.0, 10.0, 40)
    check("total_auto", int(oracle.count_auto(x, e, lib=lib).sum()) == 300 * 299 // 2)
    check("total_cross", int(oracle.count_cross(x, x[:50], e, lib=lib).sum()) == 300 * 50)
    dd = oracle.count_auto(x, e, lib=lib)
    dr = oracle.count_cross(x, x, e, lib=lib)
    want = 2 * dd
    want[1] += 300
    check("dr_self_identity", np.array_equal(dr, want))

    v = _clamp_vector()
    if v is not None:
        h = oracle.count_auto(np.stack([v, v]), np.array([0.0, 1e-6, 1.0]), lib=lib)
        check("clamp", np.array_equal(h, [0, 1, 0, 0]))

    # 3-D variant: exact Pythagorean distances on bin edges, totals, a translated copy
    pts = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 2.0], [3.0, 4.0, 0.0], [2.0, 3.0, 6.0], [1.0, 4.0, 8.0]])
    e3 = np.array([0.5, 3.0, 5.0, 7.0, 9.0, 100.0])
    h3 = oracle.count_auto(pts[:1], e3, lib=lib, euclid=True)
    check("3d_single_point", int(h3.sum()) == 0)
    h3 = oracle.count_cross(pts[:1], pts[1:], e3, lib=lib, euclid=True)
    check("3d_pythagorean", np.array_equal(h3, [0, 0, 1, 1, 1, 1, 0]))
    g3 = np.random.default_rng(5).uniform(-20, 20, (60, 3))
    e3b = np.array([0.0, 4.0, 9.0, 20.0])
    check("3d_total", int(oracle.count_auto(g3, e3b, lib=lib, euclid=True).sum()) == 60 * 59 // 2)
    check("3d_translation", np.array_equal(oracle.count_cross(g3, g3[:10] + 64.0, e3b, lib=lib, euclid=True),
                                           oracle.count_cross(g3 - 64.0, g3[:10], e3b, lib=lib, euclid=True)))
    want3 = np.zeros(len(e3b) + 1, np.uint64)
    for a in g3[:20]:
        for b in g3[20:]:
            x, y, z = float(a[0]) - float(b[0]), float(a[1]) - float(b[1]), float(a[2]) - float(b[2])
            want3[sum(1 for t in e3b if t <= math.sqrt((x * x + y * y) + z * z))] += 1
    check("3d_brute_force", np.array_equal(oracle.count_cross(g3[:20], g3[20:], e3b, lib=lib, euclid=True), want3))

    w = oracle.estimate([6, 3, 0], [15, 10, 5], [10, 5, 10], 4, 5, oracle.LS_EXACT, lib=lib)
    check("estimator_exact", list(w) == [0.5, 0.0, 0.5])
    w = oracle.estimate([2], [8], [4], 4, 8, oracle.LS_PAPER, lib=lib)
    check("estimator_paper", list(w) == [-1.0])
    return failed


def _compile(tmp_path, text, name):
    src = tmp_path / f"{name}.c"
    src.write_text(text)
    out = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", *oracle.CFLAGS, str(src), "-o", str(out), "-lm"], check=True)
    return oracle.load(str(out))


def test_unmodified_oracle_passes_battery(tmp_path):
    lib = _compile(tmp_path, open(SRC).read(), "pristine")
    assert battery(lib) == []


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, mutant):
    text = open(SRC).read()
    old, new = MUTANTS[mutant]
    assert text.count(old) == 1, f"mutation site for {mutant} not unique"
    lib = _compile(tmp_path, text.replace(old, new), mutant)
    assert battery(lib), f"no pin caught the planted mistake {mutant}"
