"""Regression of the oracle against its stored values (tests/golden/)."""
import os

import numpy as np

from tests.golden import make_golden

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read(name):
    out = {}
    for line in open(os.path.join(HERE, name)):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        out.setdefault(k, []).append([float(x) for x in v])
    return out


def test_c0_regression():
    g = read("c0_le_8cube.txt")
    a = make_golden.c0_samples()
    assert abs(a["compliance"] - g["compliance"][0][0]) <= 1e-12 * abs(g["compliance"][0][0])
    ref = np.array([r[1:] for r in g["u"]])
    assert np.abs(a["u"] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_nh_regression():
    g = read("nh_4cube_10steps.txt")
    b = make_golden.nh_samples()
    assert abs(b["reaction_x"] - g["reaction_x"][0][0]) <= 1e-9 * abs(g["reaction_x"][0][0])
    assert np.abs(b["u_centre"] - np.array(g["u"][0][1:])).max() <= 1e-10
