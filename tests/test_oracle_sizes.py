"""Pins of the size / FLOP model against the numbers the paper prints (Section 2)."""
import json
import os

from oracle import sizes

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_sizes.json")))


def test_ffff_footprints():
    g = GOLD["ffff"]
    assert sizes.pyr(3 + 3) == g["N_p"] == g["N_q"]
    assert 8 * sizes.pyr(6) ** 2 == g["pq_bytes"]
    assert sizes.pyr(g["L"]) == g["N_r"]
    assert 8 * sizes.pyr(12) == g["r_bytes"]
    assert sizes.nfun(3, True) == g["nsolid_f"]
    assert sizes.pyr(6) * sizes.nfun(3, True) ** 2 == g["H_elements"]
    assert 8 * g["H_elements"] == g["H_bytes"]


def test_iiii_footprints():
    g = GOLD["iiii"]
    assert round(8 * sizes.pyr(24) / 1000) == g["r_kB"]
    assert round(8 * sizes.pyr(12) ** 2 / 1e6, 2) == g["pq_MB"]
    assert round(8 * sizes.pyr(12) * sizes.nfun(6, True) ** 2 / 1000) == g["H_kB"]


def test_arithmetic_intensity_eq_ai():
    g = GOLD["arith_intensity"]
    assert round(sizes.arithmetic_intensity(6, 6, 6, 6, solid=True), 1) == g["iiii"]
    assert round(sizes.arithmetic_intensity(3, 3, 3, 3, solid=True), 1) == g["ffff"]
