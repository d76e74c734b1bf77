"""Oracle-side parser for the extended-Stim circuit subset.

The circuit model is the paper's (Sec. 2.1): passive Clifford gates, and
active operations — Pauli rotations, projective Pauli measurements,
stochastic Pauli noise and classically controlled Paulis. The text format is
Stim's, extended with non-Clifford gates as described in Sec. 3.1 (stage 1).

``flatten`` unrolls REPEAT blocks and assigns the physical indices that key
the random draws (identical rule on the CUDA side):

* measurement events ``e``: every M, MX, MR and R target, in order;
* records ``r``: every M, MX, MR target, in order;
* noise sites ``i``: every noise-channel target (or target pair) in order,
  plus one record-flip site right after each M(p)/MX(p)/MR(p) target with
  p > 0;
* expectation probes ``j``: every target of EXPVAL, in order. A target is a
  Pauli product such as ``X0*Y1*Z5`` (Stim's product syntax); the probe
  reports <psi|P|psi> / <psi|psi> of the shot's state at that point
  (Sec. 3.2: expectation-value probes act on the runtime state; the
  instruction name and syntax are this implementation's).

Gate conventions: T = diag(1, e^{i pi/4}) and R_P(theta) = exp(-i theta P / 2),
so T equals exp(-i (pi/8) Z) up to a global phase (Fig. 1 / App. B.1).
"""

from __future__ import annotations

import math
import re
from dataclasses import dataclass

import numpy as np

ONE_Q_CLIFFORD = {"I", "H", "S", "S_DAG", "X", "Y", "Z", "SQRT_X", "SQRT_X_DAG",
                  "SQRT_Y", "SQRT_Y_DAG"}
TWO_Q_CLIFFORD = {"CX", "CY", "CZ", "SWAP"}
ROTATIONS = {"T", "T_DAG", "R_Z", "R_X", "R_Y"}
MEASURES = {"M", "MX", "MR", "R"}
NOISE_1Q = {"X_ERROR", "Y_ERROR", "Z_ERROR", "DEPOLARIZE1"}
NOISE_2Q = {"DEPOLARIZE2"}
ALIASES = {"CNOT": "CX", "ZCX": "CX", "ZCY": "CY", "ZCZ": "CZ", "MZ": "M", "RZ": "R",
           "MRZ": "MR", "SQRT_Z": "S", "SQRT_Z_DAG": "S_DAG"}
IGNORED = {"TICK", "QUBIT_COORDS", "SHIFT_COORDS"}


class CircuitError(ValueError):
    pass


# 2x2 / 4x4 unitaries of every gate (qubit order for 4x4: first target is the
# more significant of the two local bits... see ``gate_matrix``).
def one_q_matrix(name: str, angle: float | None = None) -> np.ndarray:
    s2 = 1 / math.sqrt(2)
    if name == "I":
        return np.eye(2, dtype=complex)
    if name == "H":
        return np.array([[s2, s2], [s2, -s2]], dtype=complex)
    if name == "S":
        return np.diag([1, 1j])
    if name == "S_DAG":
        return np.diag([1, -1j])
    if name == "X":
        return np.array([[0, 1], [1, 0]], dtype=complex)
    if name == "Y":
        return np.array([[0, -1j], [1j, 0]], dtype=complex)
    if name == "Z":
        return np.diag([1, -1]).astype(complex)
    if name == "SQRT_X":
        return 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]])
    if name == "SQRT_X_DAG":
        return 0.5 * np.array([[1 - 1j, 1 + 1j], [1 + 1j, 1 - 1j]])
    if name == "SQRT_Y":
        return 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]])
    if name == "SQRT_Y_DAG":
        return 0.5 * np.array([[1 - 1j, 1 - 1j], [-1 + 1j, 1 - 1j]])
    if name == "T":
        return np.diag([1, np.exp(1j * math.pi / 4)])
    if name == "T_DAG":
        return np.diag([1, np.exp(-1j * math.pi / 4)])
    if name in ("R_Z", "R_X", "R_Y"):
        c, s = math.cos(angle / 2), math.sin(angle / 2)
        if name == "R_Z":
            return np.diag([complex(c, -s), complex(c, s)])
        if name == "R_X":
            return np.array([[c, -1j * s], [-1j * s, c]])
        return np.array([[c, -s], [s, c]], dtype=complex)
    raise CircuitError(f"no matrix for {name}")


def two_q_matrix(name: str) -> np.ndarray:
    """4x4 unitary on (a, b) with basis index 2*bit_a + bit_b."""
    m = np.zeros((4, 4), dtype=complex)
    for ia in range(2):
        for ib in range(2):
            src = 2 * ia + ib
            if name == "CX":
                m[2 * ia + (ib ^ ia), src] = 1
            elif name == "CZ":
                m[src, src] = -1 if (ia and ib) else 1
            elif name == "SWAP":
                m[2 * ib + ia, src] = 1
            elif name == "CY":
                if ia == 0:
                    m[src, src] = 1
                else:
                    # Y|0> = i|1>, Y|1> = -i|0>
                    m[2 + (1 - ib), src] = 1j if ib == 0 else -1j
            else:
                raise CircuitError(f"no matrix for {name}")
    return m


@dataclass
class Op:
    kind: str                  # 'gate' | 'noise' | 'meas' | 'ff' | 'det' | 'obs'
    name: str = ""
    qubits: tuple = ()
    arg: float | None = None   # angle or probability
    event: int = -1            # measurement event index (meas)
    record: int = -1           # record index (meas with a record; ff: control record)
    site: int = -1             # noise site index (noise) / flip site (meas)
    reset: bool = False        # meas followed by conditional X (R, MR)
    recs: tuple = ()           # det / obs record lists
    index: int = -1            # detector / observable / probe index
    paulis: tuple = ()         # probe: ((qubit, 'X' | 'Y' | 'Z'), ...)


@dataclass
class Flat:
    ops: list
    n_qubits: int
    n_events: int
    n_records: int
    n_sites: int
    n_detectors: int
    n_observables: int
    site_p: list               # probability of every site, in site order
    site_kind: list            # 'X','Y','Z','D1','D2','FLIP'
    n_probes: int = 0


_TOKEN = re.compile(r"^([A-Za-z_][A-Za-z0-9_]*)(?:\(([^)]*)\))?\s*(.*)$")


def _lines(text: str):
    for raw in text.splitlines():
        line = raw.split("#", 1)[0].strip()
        if line:
            yield line


def _parse_block(lines: list[str], pos: int, depth: int):
    out = []
    while pos < len(lines):
        line = lines[pos]
        if line == "}":
            if depth == 0:
                raise CircuitError("unmatched '}'")
            return out, pos + 1
        m = re.match(r"^REPEAT\s+(\d+)\s*\{$", line)
        if m:
            body, pos = _parse_block(lines, pos + 1, depth + 1)
            out.append(("REPEAT", int(m.group(1)), body))
            continue
        tm = _TOKEN.match(line)
        if not tm:
            raise CircuitError(f"cannot parse line: {line!r}")
        name = tm.group(1).upper()
        args = [float(a) for a in tm.group(2).split(",")] if tm.group(2) not in (None, "") else []
        targets = tm.group(3).split()
        out.append((ALIASES.get(name, name), args, targets))
        pos += 1
    if depth:
        raise CircuitError("unterminated REPEAT block")
    return out, pos


def _unroll(block):
    for item in block:
        if item[0] == "REPEAT":
            for _ in range(item[1]):
                yield from _unroll(item[2])
        else:
            yield item


def _rec_target(t: str, n_records: int) -> int:
    m = re.match(r"^rec\[-(\d+)\]$", t)
    if not m:
        raise CircuitError(f"bad record target {t!r}")
    k = int(m.group(1))
    if k < 1 or k > n_records:
        raise CircuitError(f"record target {t!r} out of range")
    return n_records - k


def _qubit(t: str) -> int:
    if not re.match(r"^\d+$", t):
        raise CircuitError(f"bad qubit target {t!r}")
    return int(t)


def _pauli_product(t: str) -> tuple:
    out = []
    for f in t.split("*"):
        m = re.match(r"^([XYZ])(\d+)$", f)
        if not m:
            raise CircuitError(f"bad Pauli product target {t!r}")
        out.append((int(m.group(2)), m.group(1)))
    if len({q for q, _ in out}) != len(out):
        raise CircuitError(f"qubit repeated in {t!r}")
    return tuple(out)


def flatten(text: str) -> Flat:
    lines = list(_lines(text))
    block, _ = _parse_block(lines, 0, 0)
    ops: list[Op] = []
    n_q = 0
    ev = rec = site = det = probe = 0
    n_obs = 0
    site_p: list[float] = []
    site_kind: list[str] = []
    for name, args, targets in _unroll(block):
        if name in IGNORED:
            continue
        if name == "DETECTOR":
            recs = tuple(_rec_target(t, rec) for t in targets)
            ops.append(Op("det", recs=recs, index=det))
            det += 1
            continue
        if name == "OBSERVABLE_INCLUDE":
            if len(args) != 1:
                raise CircuitError("OBSERVABLE_INCLUDE needs an index")
            o = int(args[0])
            recs = tuple(_rec_target(t, rec) for t in targets)
            ops.append(Op("obs", recs=recs, index=o))
            n_obs = max(n_obs, o + 1)
            continue
        if name == "EXPVAL":
            if args or not targets:
                raise CircuitError("EXPVAL takes Pauli product targets and no argument")
            for t in targets:
                ps = _pauli_product(t)
                n_q = max(n_q, max(q for q, _ in ps) + 1)
                ops.append(Op("probe", paulis=ps, index=probe))
                probe += 1
            continue
        if name in ("CX", "CY", "CZ") and any(t.startswith("rec[") for t in targets):
            if len(targets) % 2:
                raise CircuitError(f"{name} needs target pairs")
            for k in range(0, len(targets), 2):
                a, b = targets[k], targets[k + 1]
                if a.startswith("rec[") and not b.startswith("rec["):
                    r, q = _rec_target(a, rec), _qubit(b)
                elif name == "CZ" and b.startswith("rec[") and not a.startswith("rec["):
                    r, q = _rec_target(b, rec), _qubit(a)
                else:
                    raise CircuitError(f"unsupported classical control in {name}")
                n_q = max(n_q, q + 1)
                ops.append(Op("ff", name={"CX": "X", "CY": "Y", "CZ": "Z"}[name], qubits=(q,), record=r))
            continue
        qs = [_qubit(t) for t in targets]
        if qs:
            n_q = max(n_q, max(qs) + 1)
        if name in ONE_Q_CLIFFORD:
            if args:
                raise CircuitError(f"{name} takes no argument")
            for q in qs:
                ops.append(Op("gate", name=name, qubits=(q,)))
        elif name in TWO_Q_CLIFFORD:
            if len(qs) % 2:
                raise CircuitError(f"{name} needs target pairs")
            for k in range(0, len(qs), 2):
                if qs[k] == qs[k + 1]:
                    raise CircuitError(f"{name} on the same qubit twice")
                ops.append(Op("gate", name=name, qubits=(qs[k], qs[k + 1])))
        elif name in ROTATIONS:
            if name in ("T", "T_DAG"):
                if args:
                    raise CircuitError(f"{name} takes no argument")
                angle = None
            else:
                if len(args) != 1:
                    raise CircuitError(f"{name} needs one angle")
                angle = args[0]
            for q in qs:
                ops.append(Op("gate", name=name, qubits=(q,), arg=angle))
        elif name in MEASURES:
            p = 0.0
            if args:
                if name == "R" or len(args) != 1:
                    raise CircuitError(f"bad arguments for {name}")
                p = args[0]
                if not 0.0 <= p <= 1.0:
                    raise CircuitError("probability out of range")
            for q in qs:
                o = Op("meas", name=name, qubits=(q,), event=ev, reset=name in ("R", "MR"))
                ev += 1
                if name != "R":
                    o.record = rec
                    rec += 1
                    if p > 0:
                        o.site = site
                        o.arg = p
                        site_p.append(p)
                        site_kind.append("FLIP")
                        site += 1
                ops.append(o)
        elif name in NOISE_1Q or name in NOISE_2Q:
            if len(args) != 1 or not 0.0 <= args[0] <= 1.0:
                raise CircuitError(f"bad probability for {name}")
            p = args[0]
            width = 2 if name in NOISE_2Q else 1
            if len(qs) % width:
                raise CircuitError(f"{name} needs target pairs")
            kind = {"X_ERROR": "X", "Y_ERROR": "Y", "Z_ERROR": "Z", "DEPOLARIZE1": "D1",
                    "DEPOLARIZE2": "D2"}[name]
            for k in range(0, len(qs), width):
                ops.append(Op("noise", name=kind, qubits=tuple(qs[k:k + width]), arg=p, site=site))
                site_p.append(p)
                site_kind.append(kind)
                site += 1
        else:
            raise CircuitError(f"unsupported instruction {name}")
    return Flat(ops=ops, n_qubits=n_q, n_events=ev, n_records=rec, n_sites=site,
                n_detectors=det, n_observables=n_obs, site_p=site_p, site_kind=site_kind, n_probes=probe)


def option_count(kind: str) -> int:
    """Number of Pauli options K of a site kind (identity excluded)."""
    return {"D1": 3, "D2": 15}.get(kind, 1)


def option_paulis(kind: str, option: int) -> list[str]:
    """Physical Pauli letters (per target) of option ``option`` of a site.

    DEPOLARIZE1 options 0..2 are X, Y, Z. DEPOLARIZE2 option j is the pair
    with base-4 digits (j + 1) over I, X, Y, Z, the first target being the
    more significant digit (identity pair skipped).
    """
    letters = "IXYZ"
    if kind == "D1":
        return ["XYZ"[option]]
    if kind == "D2":
        j = option + 1
        return [letters[j >> 2], letters[j & 3]]
    if kind in ("X", "Y", "Z"):
        return [kind]
    raise ValueError(kind)
