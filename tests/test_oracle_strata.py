"""Pins for the oracle's stratified importance sampler (CPU only).

What fixes it independently of its own code:
* the stratum weights are the Poisson-binomial mass: the binomial closed form
  for equal probabilities, brute-force enumeration of every fault set for
  unequal ones, and total mass one;
* the jump sampler's path probabilities, multiplied out from the tables,
  equal the conditional distribution P(F | |F| = K) obtained by enumeration
  (a dropped factor, an off-by-one in W or in G_r(j + 1) fails this);
* the bisection equals the linear scan it stands for;
* Philox-driven shots have exactly K distinct faults whose subset frequencies
  fit the enumerated distribution (chi-square);
* records: every fault of an X_ERROR-before-M circuit flips exactly one
  measurement, so every shot of stratum K has exactly K ones.
"""

import itertools
import math
import random

import pytest

from oracle.factored import FactoredSim
from oracle.strata import (build_strata, first_quiet_end, g_value, sample_stratum_faults, strat_draw,
                           stratum_valid, stratum_weights)


def _brute_mass(ps):
    """P(|F| = K) and P(F) for every subset, by enumeration."""
    n = len(ps)
    mass = [0.0] * (n + 1)
    prob = {}
    for bits in range(1 << n):
        pr = 1.0
        for i, p in enumerate(ps):
            pr *= p if (bits >> i) & 1 else 1.0 - p
        f = tuple(i for i in range(n) if (bits >> i) & 1)
        prob[f] = pr
        mass[len(f)] += pr
    return mass, prob


def test_weights_binomial_closed_form():
    s, p = 60, 0.013
    w = stratum_weights([p] * s, 9)
    for k in range(10):
        exact = math.comb(s, k) * p ** k * (1 - p) ** (s - k)
        assert w[k] == pytest.approx(exact, rel=1e-12)


def test_weights_brute_force_and_total_mass():
    rng = random.Random(5)
    ps = [rng.uniform(0.0, 0.4) for _ in range(11)]
    mass, _ = _brute_mass(ps)
    w = stratum_weights(ps, len(ps))
    for k in range(len(ps) + 1):
        assert w[k] == pytest.approx(mass[k], rel=1e-12, abs=1e-300)
    assert sum(w) == pytest.approx(1.0, abs=1e-14)


@pytest.mark.parametrize("kk", [1, 2, 3, 4])
def test_path_probabilities_are_the_conditional_distribution(kk):
    rng = random.Random(11 + kk)
    ps = [rng.choice([0.0, rng.uniform(0.01, 0.5)]) for _ in range(9)]
    ps[0] = 0.2  # at least kk live sites
    ps[3] = 0.05
    ps[5] = 0.3
    ps[8] = 0.45
    t = build_strata(ps, ["X"] * len(ps), kk)
    assert stratum_valid(t, kk)
    mass, prob = _brute_mass(ps)
    total = 0.0
    for f in itertools.combinations(range(len(ps)), kk):
        st, path = 0, 1.0
        for m, j in enumerate(f):
            r = kk - m
            path *= (g_value(t, r, j) - g_value(t, r, j + 1)) / g_value(t, r, st)
            st = j + 1
        want = prob[f] / mass[kk]
        assert path == pytest.approx(want, rel=1e-9, abs=1e-15)
        if any(ps[j] == 0.0 for j in f):
            assert path == 0.0
        total += path
    assert total == pytest.approx(1.0, abs=1e-12)


def test_bisection_is_the_linear_scan():
    rng = random.Random(2)
    ps = [rng.uniform(0.0, 0.05) for _ in range(300)]
    t = build_strata(ps, ["D1"] * 300, 6)
    for _ in range(400):
        r = rng.randint(1, 6)
        st = rng.randint(0, 250)
        thr = rng.random() * g_value(t, r, st)
        want = next(j for j in range(st, 300) if g_value(t, r, j + 1) <= thr)
        assert first_quiet_end(t, r, st, thr) == want
    for r in range(1, 7):  # never increasing, zero at the end
        row = [g_value(t, r, j) for j in range(301)]
        assert all(a >= b for a, b in zip(row, row[1:]))
        assert row[-1] == 0.0


def test_draw_grid():
    for shot in (0, 5, 2 ** 40 + 1):
        for st in (0, 17):
            u, w2 = strat_draw(3, shot, st)
            assert 0.0 <= u < 1.0 and u * 2 ** 53 == int(u * 2 ** 53)
            assert 0 <= w2 < 2 ** 32


def test_sampler_counts_and_subset_frequencies():
    ps = [0.05, 0.3, 0.12, 0.2, 0.08, 0.25]
    kk = 2
    t = build_strata(ps, ["D1"] * len(ps), kk)
    mass, prob = _brute_mass(ps)
    counts = {}
    n = 6000
    for s in range(n):
        f = sample_stratum_faults(t, 77, s, kk)
        assert len(f) == kk
        assert all(0 <= o < 3 for o in f.values())
        key = tuple(sorted(f))
        counts[key] = counts.get(key, 0) + 1
    chi2 = 0.0
    for f in itertools.combinations(range(len(ps)), kk):
        e = n * prob[f] / mass[kk]
        chi2 += (counts.get(f, 0) - e) ** 2 / e
    assert chi2 < 45  # 14 dof, p ~ 5e-5


def test_special_strata():
    ps = [0.1, 0.0, 0.2, 0.0, 0.3]
    t = build_strata(ps, ["X"] * 5, 4)
    for s in range(50):
        assert sample_stratum_faults(t, 1, s, 0) == {}
        assert sorted(sample_stratum_faults(t, 1, s, 3)) == [0, 2, 4]  # every live site
        assert not ({1, 3} & set(sample_stratum_faults(t, 1, s, 2)))
    assert stratum_valid(t, 3)
    assert not stratum_valid(t, 4)  # more faults than live sites
    assert not stratum_valid(build_strata([0.5, 1.0], ["X", "X"], 1), 1)


def test_records_carry_exactly_k_flips():
    n = 7
    text = "\n".join([f"X_ERROR({0.01 * (q + 1)}) {q}" for q in range(n)] + ["M " + " ".join(map(str, range(n)))])
    sim = FactoredSim(text)
    t = build_strata(sim.flat.site_p, sim.flat.site_kind, 4)
    for kk in range(5):
        for s in range(40):
            f = sample_stratum_faults(t, 9, s, kk)
            raw = sim.run_raw(9, s, faults=f)[0]
            assert sum(raw) == kk


def _bad_first_quiet_end(t, r, st, thr):
    lo, hi = st, len(t.live) - 2
    while lo < hi:
        mid = (lo + hi) // 2
        if g_value(t, r, mid) <= thr:  # planted: G_r(j) instead of G_r(j + 1)
            hi = mid
        else:
            lo = mid + 1
    return lo


def _bad_suffix_counts(site_p, k_max):
    s = len(site_p)
    r = [[0.0] * (k_max + 1) for _ in range(s + 1)]
    r[s][0] = 1.0
    for j in range(s - 1, -1, -1):
        p = site_p[j]
        r[j][0] = (1.0 - p) * r[j + 1][0]
        for c in range(1, k_max + 1):
            r[j][c] = r[j + 1][c] + p * r[j + 1][c - 1]  # planted: (1 - p) dropped
    return r


def _bad_prefix_survival(site_p):
    return [1.0] * (len(site_p) + 1)  # planted: W dropped


@pytest.mark.parametrize("name,target,pin", [
    ("first_quiet_end", _bad_first_quiet_end, "test_sampler_counts_and_subset_frequencies"),
    ("suffix_counts", _bad_suffix_counts, "test_weights_brute_force_and_total_mass"),
    ("prefix_survival", _bad_prefix_survival, "test_path_probabilities_are_the_conditional_distribution"),
])
def test_planted_mistakes_fail_a_pin(monkeypatch, name, target, pin):
    """A mistake planted in the oracle (on the CPU) makes its pin fail (an
    assertion, or the sampler running past the last site)."""
    import oracle.strata as st
    monkeypatch.setattr(st, name, target)
    fn = globals()[pin]
    with pytest.raises((AssertionError, IndexError)):
        if pin == "test_path_probabilities_are_the_conditional_distribution":
            fn(3)
        else:
            fn()
