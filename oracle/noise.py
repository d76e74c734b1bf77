"""Noise-site sampler: the cumulative-hazard jump of Sec. 3.2 ("Sparse error
bottleneck"), restated in integer survival form so both sides agree bit for
bit.

Sites are taken in physical order and cut into segments. Inside a segment the
running survival S_i = prod_{j = start..i} (1 - p_j) is computed by FP64
multiplication in site order and stored as Q[i] = min(2^64 - 1,
floor(S_i * 2^64)). A new segment starts at site i (i > start) when S_i would
drop below 2^-16.

Per shot, a search starting at site ``st`` of segment [a, b) uses
Q_L = 2^64 - 1 if st == a else Q[st - 1], draws (u64, w2) =
gap_draw(seed, shot, st), sets T = floor(u64 * Q_L / 2^64) and puts the next
fault at the first i in [st, b) with Q[i] <= T; its Pauli option is
floor(w2 * K_i / 2^32). The next search starts at i + 1 (at b, the next
segment, when i + 1 == b). No such i: the next search starts at b.

P(no fault in [st, i]) = Q[i] / Q_L = S_i / S_{st-1}, so each site fires
independently with probability p_i (to 2^-48 quantisation).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

from .circuit import option_count
from .philox import gap_draw

U64_MAX = (1 << 64) - 1
SEGMENT_FLOOR = 2.0 ** -16


@dataclass
class SurvivalTable:
    q: list           # Q[i] as Python ints
    seg_start: list   # segment of each site -> start index
    seg_end: list     # segment of each site -> end index (exclusive)
    k: list           # option count per site


def q64(s: float) -> int:
    if s >= 1.0:
        return U64_MAX
    return min(U64_MAX, int(math.floor(s * 2.0 ** 64)))


def build_table(site_p: list[float], site_kind: list[str]) -> SurvivalTable:
    n = len(site_p)
    q = [0] * n
    seg_start = [0] * n
    seg_end = [0] * n
    start = 0
    run = 1.0
    bounds = []
    for i, p in enumerate(site_p):
        nxt = run * (1.0 - p)
        if nxt < SEGMENT_FLOOR and i > start:
            bounds.append((start, i))
            start = i
            nxt = 1.0 * (1.0 - p)
        run = nxt
        q[i] = q64(run)
    bounds.append((start, n))
    for a, b in bounds:
        for i in range(a, b):
            seg_start[i] = a
            seg_end[i] = b
    return SurvivalTable(q=q, seg_start=seg_start, seg_end=seg_end,
                         k=[option_count(kd) for kd in site_kind])


def _first_at_or_below(q: list, lo: int, hi: int, t: int) -> int:
    """First i in [lo, hi) with q[i] <= t, or -1. Q never increases inside a
    segment, so the predicate is monotone and bisection applies."""
    if lo >= hi or q[hi - 1] > t:
        return -1
    while lo < hi:
        mid = (lo + hi) // 2
        if q[mid] <= t:
            hi = mid
        else:
            lo = mid + 1
    return lo


def sample_faults(table: SurvivalTable, seed: int, shot: int) -> dict[int, int]:
    """All faults of one shot: {site index: option index}."""
    faults: dict[int, int] = {}
    n = len(table.q)
    st = 0
    while st < n:
        a, b = table.seg_start[st], table.seg_end[st]
        u64, w2 = gap_draw(seed, shot, st)
        q_l = U64_MAX if st == a else table.q[st - 1]
        t = (u64 * q_l) >> 64
        hit = _first_at_or_below(table.q, st, b, t)
        if hit < 0:
            st = b
            continue
        faults[hit] = (w2 * table.k[hit]) >> 32
        st = hit + 1
    return faults
