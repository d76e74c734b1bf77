"""Pins for the oracle's Philox and noise sampler (CPU only)."""

import math
import os
import random

import pytest

from oracle import philox
from oracle.circuit import flatten, option_count
from oracle.noise import U64_MAX, build_table, q64, sample_faults

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        assert philox.philox4x32_10(tuple(w[0:4]), tuple(w[4:6])) == tuple(w[6:10])
        n += 1
    assert n == 3


def test_meas_u_grid_and_top_bit():
    for shot in (0, 1, 127, 128, 1000, 2**40 + 3):
        for e in (0, 5, 77):
            u = philox.meas_u(9, shot, e)
            assert 0.0 <= u < 1.0
            assert (u * 2**53) == int(u * 2**53)
            assert (u >= 0.5) == bool(philox.meas_top_bit(9, shot, e))


def test_meas_u_uniform_chi2():
    bins = [0] * 16
    n = 16000
    for s in range(n):
        bins[int(philox.meas_u(3, s, s % 7) * 16)] += 1
    exp = n / 16
    chi2 = sum((b - exp) ** 2 / exp for b in bins)
    assert chi2 < 45  # 15 dof, p ~ 1e-4


def test_meas_top_bits_differ_across_shots_in_block():
    # the 128 shots of one block take distinct bits of one draw
    bits = [philox.meas_top_bit(1, s, 0) for s in range(128)]
    assert 40 < sum(bits) < 88


def test_q64_edges():
    assert q64(1.0) == U64_MAX
    assert q64(0.5) == 1 << 63
    assert q64(0.0) == 0
    assert q64(2.0 ** -64) == 1


def _sites(ps, kind="X"):
    return list(ps), [kind] * len(ps)


def test_survival_table_monotone_and_segments():
    rng = random.Random(5)
    ps = [rng.choice([0.0, 1e-3, 0.02, 0.3, 0.9]) for _ in range(400)]
    tab = build_table(*_sites(ps))
    for i in range(1, len(ps)):
        if tab.seg_start[i] == tab.seg_start[i - 1]:
            assert tab.q[i] <= tab.q[i - 1]
        else:
            assert tab.seg_start[i] == i
    # every segment's running survival stays >= 2^-16 except single-site segments
    for i in range(len(ps)):
        if tab.seg_start[i] != i:
            assert tab.q[i] >= q64(2.0 ** -16)


@pytest.mark.parametrize("ps", [
    [0.1, 0.0, 0.3, 1.0, 0.05, 0.5],
    [0.01] * 50 + [0.6] * 10 + [0.2] * 5,
])
def test_sampler_matches_independent_bernoulli(ps):
    """Per-site firing rates and a pair correlation against brute-force
    independent Bernoulli(p_i) (binomial bounds at ~5 sigma)."""
    tab = build_table(*_sites(ps))
    n = 6000
    counts = [0] * len(ps)
    pair = 0
    tot_faults = 0
    for s in range(n):
        f = sample_faults(tab, 77, s)
        tot_faults += len(f)
        for i in f:
            counts[i] += 1
        if 0 in f and 2 in f:
            pair += 1
    for i, p in enumerate(ps):
        sd = math.sqrt(max(p * (1 - p), 1e-12) / n)
        assert abs(counts[i] / n - p) <= 5 * sd + 1e-12, (i, counts[i] / n, p)
    sd = math.sqrt(ps[0] * ps[2] * (1 - ps[0] * ps[2]) / n)
    assert abs(pair / n - ps[0] * ps[2]) <= 5 * sd
    mean = sum(ps)
    var = sum(p * (1 - p) for p in ps)
    assert abs(tot_faults / n - mean) <= 5 * math.sqrt(var / n)


def test_sampler_options_uniform():
    flat = flatten("DEPOLARIZE2(0.5) 0 1\nDEPOLARIZE1(0.5) 2\nM 0 1 2\n")
    tab = build_table(flat.site_p, flat.site_kind)
    assert tab.k == [15, 3]
    c2 = [0] * 15
    c1 = [0] * 3
    for s in range(9000):
        f = sample_faults(tab, 1, s)
        if 0 in f:
            c2[f[0]] += 1
        if 1 in f:
            c1[f[1]] += 1
    for c in (c2, c1):
        exp = sum(c) / len(c)
        chi2 = sum((x - exp) ** 2 / exp for x in c)
        assert chi2 < 3 * len(c) + 20


def test_option_count():
    assert [option_count(k) for k in ("X", "Y", "Z", "D1", "D2", "FLIP")] == [1, 1, 1, 3, 15, 1]


def test_site_numbering_contract():
    flat = flatten("X_ERROR(0.1) 0 1\nM(0.2) 0 1\nDEPOLARIZE2(0.1) 0 1 1 0\nMR 0\nR 1\nM(0) 1\n")
    meas = [op for op in flat.ops if op.kind == "meas"]
    assert [op.event for op in meas] == [0, 1, 2, 3, 4]
    assert [op.record for op in meas] == [0, 1, 2, -1, 3]
    assert [op.site for op in meas] == [2, 3, -1, -1, -1]
    noise = [op.site for op in flat.ops if op.kind == "noise"]
    assert noise == [0, 1, 4, 5]
    assert flat.site_kind == ["X", "X", "FLIP", "FLIP", "D2", "D2"]
