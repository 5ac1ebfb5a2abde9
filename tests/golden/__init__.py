"""Hand-placed point sets with expected histograms fixed by exact geometry.

Written by ``make_golden.py`` in this folder (no implementation is called).
"""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURES = ["equator_ladder_linear", "meridian_cross_near_edges", "pole_fan",
            "duplicates_and_antipodes"]


def load_fixture(name):
    out = {"a": None, "b": None}
    with open(os.path.join(HERE, name + ".txt")) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    i = 0
    while i < len(lines):
        tok = lines[i].split()
        if tok[0] == "kind":
            out["kind"] = tok[1]
        elif tok[0] == "edges":
            out["edges"] = np.array([float(t) for t in tok[1:]])
        elif tok[0] in ("a", "b"):
            n = int(tok[1])
            out[tok[0]] = np.array([[float(c) for c in lines[i + 1 + k].split()] for k in range(n)])
            i += n
        elif tok[0] == "hist":
            out["hist"] = np.array([int(t) for t in tok[1:]], dtype=np.uint64)
        i += 1
    return out
