"""Stratified importance sampling of the noise sites (test infrastructure).

The paper's rare-event mode (Sec. 3.2, its closing paragraph on rare-event
estimates; used for the inject-and-cultivate study of Sec. 4.2.1): shots
are run in strata of a fixed number K of realised faults. Stratum K is
weighted by the exact probability of K faults, which for heterogeneous site
probabilities p_i is the Poisson-binomial distribution, and every shot of the
stratum has each noise site forced to fire or not to fire so that exactly K
sites fire, drawn from the conditional distribution

    P(F | |F| = K) = prod_{i in F} p_i prod_{i not in F} (1 - p_i) / P(|F| = K).

Readings (the paper names the construction, not its algorithm):

* Suffix table. R[j][r] = P(exactly r faults among sites j..S-1), by the
  recurrence R[S][0] = 1, R[S][r > 0] = 0 and
  R[j][r] = (1 - p_j) R[j + 1][r] + p_j R[j + 1][r - 1]
  (each product rounded, then the sum; no fused multiply-add). The stratum
  weight is R[0][K], the Poisson-binomial probability mass at K.
* Prefix survival. W[0] = 1, W[j + 1] = W[j] (1 - p_j).
* Jump table. G_r(j) = W[j] R[j][r]: the probability that sites 0..j-1 stay
  quiet and exactly r faults fall in j..S-1. It never increases with j, and
  G_r(S) = 0 for r >= 1. The table holds the running minimum
  min_{l <= j} fl(W[l] R[l][r]), so that rounding cannot break the
  monotonicity that the search relies on (it moves a value by an ulp at
  most).
* Conditional jump. A shot holding r remaining faults at site st puts its next
  fault at the first j >= st with G_r(j + 1) <= u * G_r(st), u uniform in
  [0, 1). Then P(no fault in st..j) = G_r(j + 1) / G_r(st), the path
  probabilities telescope to the conditional distribution above, and the
  search resumes at j + 1 with r - 1 faults.
* Draw. Philox(key, (s lo, s hi, TAG_STRAT, st)); u = (w0 | w1 << 32) >> 11
  times 2^-53 (exact), the product u * G_r(st) rounded once in FP64, and the
  fault's Pauli option floor(w2 * K_i / 2^32) as for independent noise.
* Valid strata: every p_i < 1, K at most the number of sites with p_i > 0,
  and every G_r(j) that should be positive a normal FP64 number.
"""

from __future__ import annotations

import sys
from dataclasses import dataclass

from .circuit import option_count
from .philox import MASK32, key_of, philox4x32_10

TAG_STRAT = 4  # stratified fault draw (per shot, per search start)
DBL_MIN = sys.float_info.min


@dataclass
class StrataTable:
    k_max: int
    g: list      # g[r - 1][j]: G_r(j) for r = 1..k_max, j = 0..S
    live: list   # live[j]: sites with p > 0 among j..S-1
    k: list      # option count per site
    any_certain: bool  # some p_i >= 1


def suffix_counts(site_p: list[float], k_max: int) -> list[list[float]]:
    s = len(site_p)
    r = [[0.0] * (k_max + 1) for _ in range(s + 1)]
    r[s][0] = 1.0
    for j in range(s - 1, -1, -1):
        p = site_p[j]
        q = 1.0 - p
        nxt, cur = r[j + 1], r[j]
        cur[0] = q * nxt[0]
        for c in range(1, k_max + 1):
            a = q * nxt[c]
            b = p * nxt[c - 1]
            cur[c] = a + b
    return r


def prefix_survival(site_p: list[float]) -> list[float]:
    w = [1.0]
    for p in site_p:
        w.append(w[-1] * (1.0 - p))
    return w


def build_strata(site_p: list[float], site_kind: list[str], k_max: int) -> StrataTable:
    s = len(site_p)
    r = suffix_counts(site_p, k_max)
    w = prefix_survival(site_p)
    g = []
    for c in range(1, k_max + 1):
        row = []
        run = float("inf")
        for j in range(s + 1):
            run = min(run, w[j] * r[j][c])
            row.append(run)
        g.append(row)
    live = [0] * (s + 1)
    for j in range(s - 1, -1, -1):
        live[j] = live[j + 1] + (1 if site_p[j] > 0.0 else 0)
    return StrataTable(k_max=k_max, g=g, live=live, k=[option_count(kd) for kd in site_kind],
                       any_certain=any(p >= 1.0 for p in site_p))


def stratum_weights(site_p: list[float], k_max: int) -> list[float]:
    """P(|F| = K) for K = 0..k_max (Poisson-binomial mass)."""
    return list(suffix_counts(site_p, k_max)[0])


def g_value(t: StrataTable, r: int, j: int) -> float:
    return t.g[r - 1][j]


def stratum_valid(t: StrataTable, kk: int) -> bool:
    """Stratum kk can be sampled in FP64 as read above."""
    if kk > t.k_max or t.any_certain or kk > t.live[0]:
        return False
    for r in range(1, kk + 1):
        for j in range(len(t.live)):
            if t.live[j] >= r and not g_value(t, r, j) >= DBL_MIN:
                return False
    return True


def strat_draw(seed: int, shot: int, start: int) -> tuple[float, int]:
    """(u in [0, 1) on the 53-bit grid, 32-bit option word)."""
    w = philox4x32_10((shot & MASK32, (shot >> 32) & MASK32, TAG_STRAT, start), key_of(seed))
    return ((w[0] | (w[1] << 32)) >> 11) * 2.0 ** -53, w[2]


def first_quiet_end(t: StrataTable, r: int, st: int, thr: float) -> int:
    """First j >= st with G_r(j + 1) <= thr (exists for r >= 1: G_r(S) = 0).
    G_r never increases, so bisection applies."""
    lo, hi = st, len(t.live) - 2
    while lo < hi:
        mid = (lo + hi) // 2
        if g_value(t, r, mid + 1) <= thr:
            hi = mid
        else:
            lo = mid + 1
    return lo


def sample_stratum_faults(t: StrataTable, seed: int, shot: int, kk: int) -> dict[int, int]:
    """The kk faults of one shot of stratum kk: {site index: option index}."""
    faults: dict[int, int] = {}
    st = 0
    for r in range(kk, 0, -1):
        u, w2 = strat_draw(seed, shot, st)
        thr = u * g_value(t, r, st)
        j = first_quiet_end(t, r, st, thr)
        faults[j] = (w2 * t.k[j]) >> 32
        st = j + 1
    return faults
