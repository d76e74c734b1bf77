"""Seeded synthetic circuit generators (extended Stim text).

These generators produce the inputs that both the CUDA sampler and the CPU
oracle consume. They contain none of the simulation method's arithmetic: each
function only writes circuit text (gate names, targets, noise strengths,
detector/observable annotations) from a seeded ``random.Random``.

Workload shapes follow the paper's benchmark families (Sec. 4.1, Table 1):
pure-Clifford surface-code memory (k_max = 0), low-magic fault-tolerant
gadgets (small k_max), the dense Quantum-Volume-like limit (k_max = N,
Sec. 4.1 / Fig. 5) and a batched mix. The paper's own circuit files are not
available; every circuit here is our own construction.
"""

from __future__ import annotations

import math
import random
from dataclasses import dataclass, field

__all__ = [
    "tiny_random",
    "surface_code_memory",
    "dense_random",
    "low_magic_gadgets",
    "sweep_mirror",
    "sweep_batch",
    "random_small",
    "mirror_small",
    "fig4_example",
    "ghz_t_parity",
]


class _Text:
    def __init__(self) -> None:
        self.lines: list[str] = []

    def op(self, name: str, targets, arg=None) -> None:
        targets = list(targets)
        if not targets:
            return
        head = name if arg is None else f"{name}({_fmt(arg)})"
        self.lines.append(head + " " + " ".join(str(t) for t in targets))

    def raw(self, line: str) -> None:
        self.lines.append(line)

    def text(self) -> str:
        return "\n".join(self.lines) + "\n"


def _fmt(x: float) -> str:
    return repr(float(x))


def _random_matching(rng: random.Random, qubits: list[int]) -> list[tuple[int, int]]:
    q = list(qubits)
    rng.shuffle(q)
    pairs = []
    for i in range(0, len(q) - 1, 2):
        a, b = q[i], q[i + 1]
        if rng.random() < 0.5:
            a, b = b, a
        pairs.append((a, b))
    return pairs


# --------------------------------------------------------------------------
# Workload 1: tiny random near-Clifford circuit (n=12, 30 layers, 6 T gates).
# --------------------------------------------------------------------------
def tiny_random(seed: int = 1, n: int = 12, layers: int = 30, n_t: int = 6,
                p2: float = 1e-3, pm: float = 1e-3) -> str:
    """Random H/S layer + CX on a random perfect matching with DEPOLARIZE2
    after each CX; n_t T gates at distinct (layer, qubit) slots (applied after
    that slot's single-qubit gate); X_ERROR then M on every qubit."""
    rng = random.Random(seed)
    slots = rng.sample([(l, q) for l in range(layers) for q in range(n)], n_t)
    tset = set(slots)
    c = _Text()
    for layer in range(layers):
        for q in range(n):
            c.op("H" if rng.random() < 0.5 else "S", [q])
            if (layer, q) in tset:
                c.op("T", [q])
        for a, b in _random_matching(rng, list(range(n))):
            c.op("CX", [a, b])
            c.op("DEPOLARIZE2", [a, b], p2)
    c.op("X_ERROR", range(n), pm)
    c.op("M", range(n))
    return c.text()


# --------------------------------------------------------------------------
# Workload 2: rotated surface-code memory (Z basis), d=5, 25 rounds, p=1e-3.
# --------------------------------------------------------------------------
@dataclass
class SurfaceLayout:
    d: int
    data: dict = field(default_factory=dict)      # (i, j) -> qubit
    plaquettes: list = field(default_factory=list)  # (kind, ancilla, [data or None]*4)


def surface_layout(d: int) -> SurfaceLayout:
    """Rotated surface code on a d x d data grid. Data (i, j) sit at
    (2i+1, 2j+1); a plaquette centred at (2i, 2j) touches the data at its four
    corners. Bulk plaquettes alternate X/Z in a checkerboard; weight-2
    boundary plaquettes are X-type on the top/bottom edges and Z-type on the
    left/right edges."""
    lay = SurfaceLayout(d=d)
    q = 0
    for j in range(d):
        for i in range(d):
            lay.data[(i, j)] = q
            q += 1
    corner = [(-1, -1), (-1, 0), (0, -1), (0, 0)]  # data offsets of NW, SW, NE, SE corners
    for j in range(d + 1):
        for i in range(d + 1):
            kind = "X" if (i + j) % 2 == 0 else "Z"
            inside = 1 <= i <= d - 1 and 1 <= j <= d - 1
            if not inside:
                top_bottom = (j == 0 or j == d) and 1 <= i <= d - 1
                left_right = (i == 0 or i == d) and 1 <= j <= d - 1
                if top_bottom and kind == "X":
                    pass
                elif left_right and kind == "Z":
                    pass
                else:
                    continue
            touched = []
            for di, dj in corner:
                key = (i + di, j + dj)
                touched.append(lay.data.get(key))
            lay.plaquettes.append((kind, None, touched, (i, j)))
    # assign ancilla indices after the data block
    out = []
    for kind, _, touched, pos in lay.plaquettes:
        out.append((kind, q, touched, pos))
        q += 1
    lay.plaquettes = out
    return lay


# CX order over the four corners [NW, SW, NE, SE]: the two stabiliser types
# visit the shared corners in orders that keep X and Z checks commuting.
_X_ORDER = [0, 1, 2, 3]   # NW, SW, NE, SE
_Z_ORDER = [0, 2, 1, 3]   # NW, NE, SW, SE


def surface_code_memory(d: int = 5, rounds: int = 25, p: float = 1e-3, theta: float = 0.0) -> str:
    """Rotated surface-code memory (Z basis). theta > 0 adds the coherent
    over-rotation R_Z(theta) on the targets of every depolarising channel
    (the coherent-noise family of the paper's Table 1)."""
    lay = surface_layout(d)
    anc = [a for _, a, _, _ in lay.plaquettes]
    xanc = [a for k, a, _, _ in lay.plaquettes if k == "X"]
    zanc = [a for k, a, _, _ in lay.plaquettes if k == "Z"]
    n_anc = len(anc)
    c = _Text()
    for r in range(rounds):
        c.op("R", anc)
        c.op("X_ERROR", anc, p)
        c.op("H", xanc)
        c.op("DEPOLARIZE1", xanc, p)
        if theta:
            c.op("R_Z", xanc, theta)
        for step in range(4):
            pairs = []
            for kind, a, touched, _ in lay.plaquettes:
                corner = (_X_ORDER if kind == "X" else _Z_ORDER)[step]
                dq = touched[corner]
                if dq is None:
                    continue
                pairs.append((a, dq) if kind == "X" else (dq, a))
            flat = [t for pr in pairs for t in pr]
            c.op("CX", flat)
            c.op("DEPOLARIZE2", flat, p)
            if theta:
                c.op("R_Z", flat, theta)
        c.op("H", xanc)
        c.op("DEPOLARIZE1", xanc, p)
        if theta:
            c.op("R_Z", xanc, theta)
        c.op("M", anc, p)
        # detectors
        for idx, (kind, a, _, _) in enumerate(lay.plaquettes):
            back = n_anc - idx
            if r == 0:
                if kind == "Z":
                    c.raw(f"DETECTOR rec[-{back}]")
            else:
                c.raw(f"DETECTOR rec[-{back}] rec[-{back + n_anc}]")
    data = [lay.data[(i, j)] for j in range(d) for i in range(d)]
    c.op("M", data, p)
    n_data = len(data)
    pos_of = {q: k for k, q in enumerate(data)}
    for idx, (kind, a, touched, _) in enumerate(lay.plaquettes):
        if kind != "Z":
            continue
        recs = [f"rec[-{n_data - pos_of[dq]}]" for dq in touched if dq is not None]
        recs.append(f"rec[-{n_data + n_anc - idx}]")
        c.raw("DETECTOR " + " ".join(recs))
    row = [lay.data[(i, 0)] for i in range(d)]
    c.raw("OBSERVABLE_INCLUDE(0) " + " ".join(f"rec[-{n_data - pos_of[q]}]" for q in row))
    return c.text()


# --------------------------------------------------------------------------
# Workload 3: dense limit, n=20, 40 layers of random {H, S, T} + CX matching.
# --------------------------------------------------------------------------
def dense_random(seed: int = 3, n: int = 20, layers: int = 40, mirror: bool = False) -> str:
    rng = random.Random(seed)
    body: list[tuple[str, list[int]]] = []
    for _ in range(layers):
        for q in range(n):
            body.append((rng.choice(["H", "S", "T"]), [q]))
        for a, b in _random_matching(rng, list(range(n))):
            body.append(("CX", [a, b]))
    c = _Text()
    for name, t in body:
        c.op(name, t)
    if mirror:
        inv = {"H": "H", "S": "S_DAG", "T": "T_DAG", "CX": "CX"}
        for name, t in reversed(body):
            c.op(inv[name], t)
    c.op("M", range(n))
    return c.text()


# --------------------------------------------------------------------------
# Workload 4: low-magic fault-tolerant-shaped circuit on a 5 x 10 grid.
# --------------------------------------------------------------------------
def _grid_neighbors(w: int, h: int):
    nb = {}
    for y in range(h):
        for x in range(w):
            q = y * w + x
            nb[q] = [yy * w + xx for xx, yy in ((x + 1, y), (x - 1, y), (x, y + 1), (x, y - 1))
                     if 0 <= xx < w and 0 <= yy < h]
    return nb


def low_magic_gadgets(seed: int = 4, p: float = 5e-4, width: int = 10, height: int = 5,
                      n_gadgets: int = 16, open_max: int = 10, checks: int = 6,
                      filler_depth: int = 13, filler_det_every: int = 3) -> str:
    """T/T_DAG pairs bracketing repeated ZZ parity checks of a Bell pair.

    Each gadget uses a line (a, b, c) of grid neighbours: Bell pair on (a, b),
    T on a, ``checks`` rounds of Z_a Z_b parity measured on ancilla c, T_DAG on
    a, un-prepare and measure a and b. The checks commute with the T rotation,
    so every measurement is deterministic without noise. Gadgets run in waves
    of at most ``open_max`` at once (so k_max <= open_max). Idle qubits run
    filler Clifford blocks U then U^dagger followed by M + R. Every detector
    is a single deterministic record. All checks are postselected.
    """
    rng = random.Random(seed)
    nq = width * height
    c = _Text()
    # gadget lines: horizontal triples (x, x+1, x+2) on each row
    triples = []
    for y in range(height):
        for x0 in (0, 3, 6):
            if x0 + 2 < width:
                base = y * width + x0
                triples.append((base, base + 1, base + 2))
    waves = []
    remaining = n_gadgets
    while remaining > 0:
        take = min(open_max, remaining, len(triples))
        waves.append(rng.sample(triples, take))
        remaining -= take
    nb = _grid_neighbors(width, height)
    n_meas = 0

    def one_q(qs):
        for q in qs:
            c.op(rng.choice(["H", "S", "S_DAG"]), [q])
            c.op("DEPOLARIZE1", [q], p)

    def filler_block(idle: list[int]):
        nonlocal n_meas
        if not idle:
            return 0
        body: list[tuple[str, list[int]]] = []
        idle_set = set(idle)
        for _ in range(filler_depth):
            for q in idle:
                body.append((rng.choice(["H", "S", "S_DAG"]), [q]))
            used = set()
            for q in idle:
                if q in used:
                    continue
                cand = [r for r in nb[q] if r in idle_set and r not in used]
                if cand and rng.random() < 0.8:
                    r = rng.choice(cand)
                    used.add(q)
                    used.add(r)
                    body.append(("CX", [q, r] if rng.random() < 0.5 else [r, q]))
        inv = {"H": "H", "S": "S_DAG", "S_DAG": "S", "CX": "CX"}
        for name, t in body + [(inv[nm], tt) for nm, tt in reversed(body)]:
            c.op(name, t)
            c.op("DEPOLARIZE2" if name == "CX" else "DEPOLARIZE1", t, p)
        c.op("X_ERROR", idle, p)
        c.op("M", idle)
        n_meas += len(idle)
        for k in range(len(idle)):
            if k % filler_det_every == 0:
                c.raw(f"DETECTOR rec[-{len(idle) - k}]")
        c.op("R", idle)
        c.op("X_ERROR", idle, p)
        return len(idle)

    obs_records: list[int] = []
    for wave in waves:
        busy = sorted({q for tr in wave for q in tr})
        idle = [q for q in range(nq) if q not in set(busy)]
        for a, b, anc in wave:
            c.op("H", [a])
            c.op("DEPOLARIZE1", [a], p)
            c.op("CX", [a, b])
            c.op("DEPOLARIZE2", [a, b], p)
            c.op("T", [a])
        for _ in range(checks):
            for a, b, anc in wave:
                c.op("CX", [a, anc])
                c.op("DEPOLARIZE2", [a, anc], p)
                c.op("CX", [b, anc])
                c.op("DEPOLARIZE2", [b, anc], p)
            ancs = [tr[2] for tr in wave]
            c.op("X_ERROR", ancs, p)
            c.op("M", ancs)
            n_meas += len(ancs)
            for k in range(len(ancs)):
                c.raw(f"DETECTOR rec[-{len(ancs) - k}]")
            c.op("R", ancs)
            c.op("X_ERROR", ancs, p)
            quarter = len(idle) // 4
            part = _ % 4
            filler_block(idle[part * quarter: (part + 1) * quarter if part < 3 else len(idle)])
        for a, b, anc in wave:
            c.op("T_DAG", [a])
            c.op("CX", [a, b])
            c.op("DEPOLARIZE2", [a, b], p)
            c.op("H", [a])
            c.op("DEPOLARIZE1", [a], p)
        ab = [q for tr in wave for q in tr[:2]]
        c.op("X_ERROR", ab, p)
        c.op("M", ab)
        n_meas += len(ab)
        for k in range(len(ab)):
            c.raw(f"DETECTOR rec[-{len(ab) - k}]")
        c.raw(f"OBSERVABLE_INCLUDE(0) rec[-{len(ab)}]")
        c.op("R", ab)
        c.op("X_ERROR", ab, p)
    return c.text()


# --------------------------------------------------------------------------
# Workload 5: batched sweep of mirror circuits of uneven size.
# --------------------------------------------------------------------------
@dataclass
class SweepCircuit:
    text: str
    n: int
    depth: int
    t: int
    p: float
    shots: int


def sweep_mirror(c_index: int) -> SweepCircuit:
    rng = random.Random(5000 + c_index)
    n = rng.randint(20, 80)
    depth = rng.randint(50, 400)
    t = rng.randint(0, 14)
    p = math.exp(rng.uniform(math.log(1e-4), math.log(5e-3)))
    shots = int(round(math.exp(rng.uniform(math.log(1e6), math.log(1e8)))))
    w = int(math.ceil(math.sqrt(n)))
    h = (n + w - 1) // w
    nb = _grid_neighbors(w, h)
    nb = {q: [r for r in v if r < n] for q, v in nb.items() if q < n}
    # choose the layers (first half of U) that carry a T gate
    t_layers = sorted(rng.sample(range(max(1, depth // 2)), min(t, max(1, depth // 2)))) if t else []
    cliff1 = ["H", "S", "S_DAG", "X", "Y", "Z"]
    body: list[tuple[str, list[int]]] = []
    t_iter = iter(t_layers)
    next_t = next(t_iter, None)
    placed = 0
    for layer in range(depth):
        for q in range(n):
            body.append((rng.choice(cliff1), [q]))
        if next_t is not None and layer == next_t and placed < t:
            q = rng.randrange(n)
            body.append(("H", [q]))
            body.append(("T", [q]))
            placed += 1
            next_t = next(t_iter, None)
        used = set()
        order = list(range(n))
        rng.shuffle(order)
        for q in order:
            if q in used:
                continue
            cand = [r for r in nb[q] if r not in used]
            if cand:
                r = rng.choice(cand)
                used.add(q)
                used.add(r)
                body.append(("CX", [q, r] if rng.random() < 0.5 else [r, q]))
    inv = {"H": "H", "S": "S_DAG", "S_DAG": "S", "X": "X", "Y": "Y", "Z": "Z",
           "T": "T_DAG", "CX": "CX"}
    c = _Text()
    for name, tg in body + [(inv[nm], tt) for nm, tt in reversed(body)]:
        c.op(name, tg)
        if name == "CX":
            c.op("DEPOLARIZE2", tg, p)
        elif name not in ("T", "T_DAG"):
            c.op("DEPOLARIZE1", tg, p)
    c.op("X_ERROR", range(n), p)
    c.op("M", range(n))
    c.raw("OBSERVABLE_INCLUDE(0) " + " ".join(f"rec[-{k}]" for k in range(1, n + 1)))
    return SweepCircuit(text=c.text(), n=n, depth=depth, t=placed, p=p, shots=shots)


def sweep_batch(count: int = 64) -> list[SweepCircuit]:
    return [sweep_mirror(i) for i in range(count)]


# --------------------------------------------------------------------------
# Small test families (pins and parity cases).
# --------------------------------------------------------------------------
_ONE_Q = ["H", "S", "S_DAG", "X", "Y", "Z", "SQRT_X", "SQRT_X_DAG"]
_ROT = ["T", "T_DAG", "R_Z", "R_X", "R_Y"]


def random_small(seed: int, n: int = 5, n_ops: int = 60, p_noise: float = 0.0,
                 t_frac: float = 0.2, meas_frac: float = 0.1, feedforward: bool = True,
                 rotations: bool = True, detectors: bool = False) -> str:
    """Random small circuit exercising every supported instruction kind:
    Clifford gates, Pauli rotations, Z/X measurements, resets, measure-reset,
    noise channels, record flips and classically controlled Paulis."""
    rng = random.Random(seed)
    c = _Text()
    n_rec = 0
    for _ in range(n_ops):
        r = rng.random()
        if rotations and r < t_frac:
            g = rng.choice(_ROT)
            q = rng.randrange(n)
            if g in ("R_Z", "R_X", "R_Y"):
                c.op(g, [q], rng.uniform(-math.pi, math.pi))
            else:
                c.op(g, [q])
        elif r < t_frac + meas_frac:
            g = rng.choice(["M", "MX", "MR", "R", "M"])
            q = rng.randrange(n)
            if g in ("M", "MX", "MR") and p_noise > 0 and rng.random() < 0.5:
                c.op(g, [q], p_noise)
            else:
                c.op(g, [q])
            if g != "R":
                n_rec += 1
                if feedforward and rng.random() < 0.3:
                    tq = rng.randrange(n)
                    c.raw(f"{rng.choice(['CX', 'CZ', 'CY'])} rec[-1] {tq}")
        elif r < t_frac + meas_frac + 0.45:
            c.op(rng.choice(_ONE_Q), [rng.randrange(n)])
        else:
            a, b = rng.sample(range(n), 2)
            c.op(rng.choice(["CX", "CZ", "SWAP", "CY"]), [a, b])
            if p_noise > 0 and rng.random() < 0.5:
                c.op(rng.choice(["DEPOLARIZE2"]), [a, b], p_noise)
        if p_noise > 0 and rng.random() < 0.3:
            ch = rng.choice(["X_ERROR", "Y_ERROR", "Z_ERROR", "DEPOLARIZE1"])
            c.op(ch, [rng.randrange(n)], p_noise)
    c.op("M", range(n))
    return c.text()


def with_probes(text: str, seed: int, count: int = 6, max_weight: int = 3) -> str:
    """Insert `count` EXPVAL lines (random Pauli products over the circuit's
    qubits) at random top-level positions of a circuit without REPEAT."""
    rng = random.Random(seed)
    lines = text.splitlines()
    n = 1 + max((int(t) for ln in lines for t in ln.split()[1:] if t.isdigit()), default=0)
    for _ in range(count):
        w = rng.randint(1, min(max_weight, n))
        qs = rng.sample(range(n), w)
        prod = "*".join(f"{rng.choice('XYZ')}{q}" for q in qs)
        lines.insert(rng.randint(0, len(lines)), f"EXPVAL {prod}")
    return "\n".join(lines) + "\n"


def mirror_small(seed: int, n: int = 6, depth: int = 12, n_t: int = 4) -> str:
    """Noiseless U U^dagger with Clifford+T layers; every record must be 0."""
    rng = random.Random(seed)
    body: list[tuple[str, list[int], float | None]] = []
    for _ in range(depth):
        for q in range(n):
            g = rng.choice(["H", "S", "S_DAG", "SQRT_X", "T", "T_DAG", "I"])
            if g == "I":
                continue
            body.append((g, [q], None))
        for a, b in _random_matching(rng, list(range(n))):
            body.append((rng.choice(["CX", "CZ"]), [a, b], None))
        if rng.random() < 0.3:
            q = rng.randrange(n)
            body.append(("R_Z", [q], rng.uniform(-3, 3)))
    inv = {"H": "H", "S": "S_DAG", "S_DAG": "S", "SQRT_X": "SQRT_X_DAG", "T": "T_DAG",
           "T_DAG": "T", "CX": "CX", "CZ": "CZ", "R_Z": "R_Z"}
    c = _Text()
    for g, t, a in body:
        c.op(g, t, a)
    for g, t, a in reversed(body):
        c.op(inv[g], t, None if a is None else -a)
    c.op("M", range(n))
    return c.text()


def fig4_example(p: float = 0.001) -> str:
    """The worked example of Fig. 3/4, as printed."""
    return (
        "H 0\nT 0\nT 0\nT 0\nCX 0 1\n"
        f"DEPOLARIZE1({_fmt(p)}) 0 1\n"
        "CX 0 1\nT_DAG 0\nH 0\nM 0 1\n"
    )


def ghz_t_parity(n: int) -> str:
    """GHZ_n, T on every qubit, then MX on all (X^n parity from the records)."""
    c = _Text()
    c.op("H", [0])
    for q in range(n - 1):
        c.op("CX", [q, q + 1])
    c.op("T", range(n))
    c.op("MX", range(n))
    return c.text()
