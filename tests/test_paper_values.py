"""Consistency of the numbers printed in the paper (tests/golden/paper_values.txt)."""
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def _load():
    vals = {}
    with open(os.path.join(HERE, "golden", "paper_values.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, v, e = line.split()[:3]
            vals[key] = (float(v), float(e))
    return vals


def test_luscher_coefficient_in_four_dimensions():
    """Section 1.1: the universal term is pi (d-2) / (24 r); d = 4 gives pi/12 = 0.2618."""
    v = _load()
    assert abs(math.pi * (4 - 2) / 24 - v["luscher_term_expected_d4"][0]) < 5e-5
    # the free fit agrees with it within its error (Section 3)
    fit, err = v["luscher_term_fit"]
    assert abs(fit - math.pi / 12) < err


def test_string_tensions_agree_and_widths_grow():
    v = _load()
    a, ea = v["string_tension_fixed_luscher"]
    b, eb = v["string_tension_free"]
    assert abs(a - b) < math.hypot(ea, eb)
    assert v["width2_r2"][0] < v["width2_r4"][0] < v["width2_r6"][0]
