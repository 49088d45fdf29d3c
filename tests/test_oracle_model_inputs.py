"""Pins of the performance-model counters and of the seeded input generators (no GPU)."""
import json
import math
import os

import numpy as np

from oracle import model as M
from oracle.tt_svd_oracle import planned_ranks, unfolding_singular_values
from paper_2102_00104_gb300.inputs import (philox4x32_10, planted_tt, uniform_f64,
                                           uniform_tensor)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_model_constants():
    g = json.load(open(os.path.join(GOLDEN, "likwid_table_2p30.json")))["model_constants"]
    assert math.isclose(M.ttsvd_volume_bound(1.0, 1 / 16, es=1), g["volume_fbar_1_16"], rel_tol=0.01)
    assert math.isclose(M.ttsvd_volume_bound(1.0, 1 / 2, es=1), g["volume_fbar_1_2"], rel_tol=1e-12)
    assert math.isclose(M.ttsvd_flops_bound(1.0, 1, 1 / 16), g["flops_fbar_1_16"], rel_tol=0.01)
    assert math.isclose(M.ttsvd_flops_bound(1.0, 1, 1 / 2), g["flops_fbar_1_2"], rel_tol=1e-12)


def test_model_against_likwid_table():
    g = json.load(open(os.path.join(GOLDEN, "likwid_table_2p30.json")))
    nbar = g["nbar"]
    for row in g["rows"]:
        est_f = M.ttsvd_flops_bound(nbar, row["r_max"], row["fbar"]) / 1e9
        est_b = M.ttsvd_volume_bound(nbar, row["fbar"]) / 1e9
        assert abs(est_f - row["gflop_estimate"]) <= 0.6 + 0.02 * row["gflop_estimate"], row
        assert abs(est_b - row["gbyte_estimate"]) <= 0.6, row
    # exact per-step counts of Alg. 2 for the paper's shapes are close to the measurements
    shapes = {("plain", 1): (2,) * 30}
    k1 = M.thick_bounds_k((2,) * 30, 16, 0.5, 1)
    k31 = M.thick_bounds_k((2,) * 30, 16, 0.5, 31)
    shapes[("thick_bounds", 1)] = (2,) * (30 - k1) + (2 ** k1,)
    shapes[("thick_bounds", 31)] = (2,) * (30 - k31) + (2 ** k31,)
    for row in g["rows"]:
        dims = shapes[(row["case"], row["r_max"])]
        steps = M.ttsvd_step_counts(dims, planned_ranks(dims, row["r_max"]))
        gf = sum(s["flops"] for s in steps) / 1e9
        gb = sum(s["bytes"] for s in steps) / 1e9
        assert abs(gf - row["gflop_measured"]) <= 0.10 * row["gflop_measured"], (row, gf)
        assert abs(gb - row["gbyte_measured"]) <= 0.10 * row["gbyte_measured"], (row, gb)


def test_building_block_formulas():
    assert M.tsqr_flops(1000, 4, 10) == (1000 / 10) * 2 * 4 * 5 * 11
    assert math.isclose(M.tsqr_intensity(50, 10**9), 12.5, rel_tol=1e-6)  # m/4 for doubles
    assert math.isclose(M.tsmm_intensity(20, 10), 20 * 10 / (4 * 30))
    assert M.tsmm_bytes(100, 8, 2) == 8 * 100 * 10


def test_philox_known_answers():
    # Known-answer vectors of Philox4x32-10 (Salmon et al., SC'11 test vectors)
    cases = [((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
             ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
             ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
              (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1))]
    for c, k, out in cases:
        got = philox4x32_10([c[0]], [c[1]], [c[2]], [c[3]], k[0], k[1])
        assert tuple(int(x[0]) for x in got) == out


def test_uniform_known_answers():
    # entries 0 and 1 of seed 0 come from block 0, i.e. Philox4x32-10 of counter (0,0,0,0)
    # under key (0,0), whose published output words are 0x6627E8D5 0xE169C58D 0xBC57AC4C
    # 0x9B00DBD8; each pair of words (x, y) gives the 53-bit fraction
    # (floor(x / 2^5) 2^26 + floor(y / 2^6)) / 2^53, evaluated here with exact rationals
    from fractions import Fraction
    words = (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)
    expect = [Fraction((x // 32) * 2 ** 26 + y // 64, 2 ** 53) for x, y in (words[:2], words[2:])]
    got = uniform_f64(0, 2)
    assert [Fraction(float(v)) for v in got] == expect


def test_uniform_stream_properties():
    a = uniform_f64(7, 10001)
    assert np.all(a >= 0) and np.all(a < 1)
    assert abs(a.mean() - 0.5) < 0.02
    # any window of the stream equals the same slice of the full stream
    for start, cnt in [(1, 5), (2, 8), (333, 1000), (10000, 1)]:
        assert np.array_equal(uniform_f64(7, cnt, start), a[start:start + cnt])
    assert not np.array_equal(uniform_f64(8, 100), a[:100])
    X = uniform_tensor((3, 4, 5), seed=7, chunk=7)
    assert np.array_equal(X.ravel(order="F"), a[:60])


def test_planted_tensor_ranks():
    dims = (4, 3, 5, 4)
    X = planted_tt(dims, 2, seed=3, noise_rel=0.0)
    assert math.isclose(np.linalg.norm(X), 1.0, rel_tol=1e-12)
    for k in range(1, 4):
        s = unfolding_singular_values(X, k)
        planted = min(2, int(np.prod(dims[:k])), int(np.prod(dims[k:])))
        assert np.all(s[planted:] < 1e-12) and s[planted - 1] > 1e-6
    Y = planted_tt(dims, 2, seed=3, noise_rel=1e-6)
    assert math.isclose(np.linalg.norm(Y - X), 1e-6, rel_tol=1e-6)
