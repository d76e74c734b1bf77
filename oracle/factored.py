"""O-A: the frame-factored method, step by step, in FP64 (test infrastructure).

State (Def. 2): |psi> = gamma U_C P~ (|phi>_A (x) |0>_D). The global scalar
gamma only carries phase and normalisation here: phases are dropped and phi
is renormalised at every active measurement (the paper allows lazy
normalisation; eager renormalisation with probabilities taken relative to
S0 + S1 is the reading used here, and the dormant convention after an active
measurement is x_v ^= b, preceded by H_v for an X measurement).

Plan (shot independent, Thm. 1): walk the physical circuit keeping the map
M(P) = U_C^dagger P U_C as the images of every physical X_j and Z_j
(Def. 1). Clifford gates update M; every active operation is Heisenberg
mapped and, if needed, Pauli-localised (Lemma 1, App. A) by a virtual
Clifford sequence V, after which U_C <- U_C V^dagger, i.e. M <- V M V^dagger
(Sec. 2.3). Localisation rule (App. A, with the pivot reading):

* x != 0: pivot v = lowest dormant qubit with x_v = 1, else the lowest active
  one; CX(v -> q) for every other q with x_q = 1 (ascending q); then
  CZ(v, q) for every other q with z_q = 1 (ascending q); then S_v if the
  result is Y_v (S Y S^dagger = -X).
* x == 0: pivot v = lowest active qubit with z_v = 1; CX(q -> v) for every
  other q with z_q = 1 (ascending q). No active z-support: no localisation
  (a dormant Z string: scalar phase for a rotation, a static parity for a
  measurement).

With a dormant pivot every gate of V is controlled by a dormant qubit or is
diagonal on it, so V acts as the identity on phi (x) 0_D (Lemma 2); gates
between two active qubits act on phi; V never entangles a dormant qubit.

Run (per shot): the frame (x, z) is conjugated by every V; rotations,
measurements and conditional Paulis update phi and the frame as in Sec. 2.4
and App. B:

* rotation exp(-i theta alpha P_v): commuting it through the frame flips the
  angle when the frame anticommutes with P_v (App. B.1). Dormant X_v: V gains
  H_v, v becomes active (phi <- phi (x) |+>), then exp(-i theta' Z_v).
* measurement (App. B.2), b the virtual outcome, m the physical one,
  b = m ^ a ^ p with alpha = (-1)^a and p the frame anticommutation bit:
  dormant Z: m = a ^ p (static); dormant X: uniform, then H_v and x_v ^= b;
  active Z: mask; active X: fold (phi_0 + (-1)^b phi_1)/sqrt(2), then H_v;
  in both active cases renormalise, x_v ^= b, demote v (the top position
  moves into v's position) and k <- k - 1.
* conditional Pauli E (noise, resets, classical control): P~ <- M(E) P~
  (App. B.3), phase dropped.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from functools import lru_cache

import numpy as np

from .circuit import Flat, flatten, one_q_matrix, option_paulis, two_q_matrix
from .noise import build_table, sample_faults
from .philox import meas_u
from .records import ShotRecords, assemble, raw_parities

_PAULI_M = {
    (0, 0): np.eye(2, dtype=complex),
    (1, 0): np.array([[0, 1], [1, 0]], dtype=complex),
    (0, 1): np.diag([1, -1]).astype(complex),
}
_PAULI_M[(1, 1)] = _PAULI_M[(1, 0)] @ _PAULI_M[(0, 1)]      # X Z (= -iY)


# --------------------------------------------------------------------------
# Signed Paulis i^ph X^x Z^z (x, z bit masks; X^x Z^z = prod X_j^x_j prod Z_j^z_j)
# --------------------------------------------------------------------------
def pmul(a, b):
    x1, z1, p1 = a
    x2, z2, p2 = b
    return (x1 ^ x2, z1 ^ z2, (p1 + p2 + 2 * bin(z1 & x2).count("1")) % 4)


def herm_sign(p) -> int:
    """Sign bit s of a Hermitian Pauli written as (-1)^s prod sigma_j."""
    x, z, ph = p
    d = (ph - bin(x & z).count("1")) % 4
    assert d in (0, 2), "not Hermitian"
    return d // 2


def _local_matrix(bits_x: int, bits_z: int, width: int) -> np.ndarray:
    mats = [_PAULI_M[((bits_x >> j) & 1, (bits_z >> j) & 1)] for j in range(width)]
    # local qubit 0 is the more significant factor (matches two_q_matrix)
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


def _as_local_pauli(m: np.ndarray, width: int):
    for x in range(1 << width):
        for z in range(1 << width):
            base = _local_matrix(x, z, width)
            for ph in range(4):
                if np.allclose(m, (1j ** ph) * base, atol=1e-12):
                    return x, z, ph
    raise AssertionError("not a Pauli")


def _gate_matrix(name: str) -> tuple[np.ndarray, int]:
    if name in ("CX", "CZ", "CY", "SWAP"):
        return two_q_matrix(name), 2
    return one_q_matrix(name), 1


@lru_cache(maxsize=None)
def conj_table(name: str, inverse: bool = False):
    """Images G g G^dagger of the local generators g = X_0, Z_0 (, X_1, Z_1),
    derived numerically from the gate's unitary. ``inverse`` uses G^dagger."""
    u, w = _gate_matrix(name)
    if inverse:
        u = u.conj().T
    out = []
    for j in range(w):
        for kind in ("X", "Z"):
            g = _local_matrix(1 << j if kind == "X" else 0, 1 << j if kind == "Z" else 0, w)
            out.append(_as_local_pauli(u @ g @ u.conj().T, w))
    return tuple(out)   # (img X_0, img Z_0[, img X_1, img Z_1]) as local paulis


def conjugate(p, name: str, qubits: tuple, inverse: bool = False):
    """G P G^dagger for a gate G on ``qubits`` (global qubit indices)."""
    x, z, ph = p
    tab = conj_table(name, inverse)
    mask = 0
    for q in qubits:
        mask |= 1 << q
    acc = (x & ~mask, z & ~mask, ph)
    loc_x = [(x >> q) & 1 for q in qubits]
    loc_z = [(z >> q) & 1 for q in qubits]

    def glob(lp):
        lx, lz, lph = lp
        gx = gz = 0
        for j, q in enumerate(qubits):
            if (lx >> j) & 1:
                gx |= 1 << q
            if (lz >> j) & 1:
                gz |= 1 << q
        return gx, gz, lph

    for j in range(len(qubits)):
        if loc_x[j]:
            acc = pmul(acc, glob(tab[2 * j]))
    for j in range(len(qubits)):
        if loc_z[j]:
            acc = pmul(acc, glob(tab[2 * j + 1]))
    return acc


# --------------------------------------------------------------------------
# Plan
# --------------------------------------------------------------------------
@dataclass
class Step:
    kind: str
    a: dict = field(default_factory=dict)


ROT_GEN = {"T": ("Z", math.pi / 8), "T_DAG": ("Z", -math.pi / 8)}


class FactoredSim:
    def __init__(self, text_or_flat, k_limit: int = 24):
        self.flat: Flat = flatten(text_or_flat) if isinstance(text_or_flat, str) else text_or_flat
        self.n = max(1, self.flat.n_qubits)
        self.k_limit = k_limit
        self.table = build_table(self.flat.site_p, self.flat.site_kind)
        self.steps: list[Step] = []
        self.k_max = 0
        self._plan()
        ref_meas = self.run_raw(0, 0, noisy=False, argmax=True)[0]
        self.ref_det, self.ref_obs = raw_parities(self.flat, ref_meas)

    # M(P) for a physical Pauli given per physical qubit as letters
    def _map(self, paulis: dict[int, str]):
        acc = (0, 0, 0)
        xs = [q for q, l in sorted(paulis.items()) if l in "XY"]
        zs = [q for q, l in sorted(paulis.items()) if l in "ZY"]
        for q in xs:
            acc = pmul(acc, self.img[("X", q)])
        for q in zs:
            acc = pmul(acc, self.img[("Z", q)])
        ny = sum(1 for l in paulis.values() if l == "Y")
        # Y = i X Z per qubit
        return acc[0], acc[1], (acc[2] + ny) % 4

    def _physical_gate(self, name: str, qubits: tuple):
        new = {}
        for j, q in enumerate(qubits):
            for kind in ("X", "Z"):
                g = (1 << q if kind == "X" else 0, 1 << q if kind == "Z" else 0, 0)
                pre = conjugate(g, name, qubits, inverse=True)   # C^dagger g C
                # evaluate M_old on pre
                acc = (0, 0, pre[2])
                for qq in qubits:
                    if (pre[0] >> qq) & 1:
                        acc = pmul(acc, self.img[("X", qq)])
                for qq in qubits:
                    if (pre[1] >> qq) & 1:
                        acc = pmul(acc, self.img[("Z", qq)])
                new[(kind, q)] = acc
        self.img.update(new)

    def _virtual_gate(self, name: str, vq: tuple):
        """U_C <- U_C V^dagger for one virtual gate V; also emits the step."""
        for key in self.img:
            self.img[key] = conjugate(self.img[key], name, vq)
        act = self.active
        on_state = all(q in act for q in vq)
        pos = tuple(act.index(q) for q in vq) if on_state else None
        self.steps.append(Step("vg", dict(name=name, vq=vq, pos=pos)))

    def _localize(self, p):
        """Apply the localising sequence to p; returns (v, 'X'|'Z', a) or None
        for a dormant Z string (x == 0 with no active z-support)."""
        x, z, _ = p
        act = set(self.active)
        if x:
            xs = [q for q in range(self.n) if (x >> q) & 1]
            dormant = [q for q in xs if q not in act]
            v = dormant[0] if dormant else xs[0]
            if v in act:
                assert all(q in act for q in xs)
            for q in xs:
                if q != v:
                    p = conjugate(p, "CX", (v, q))
                    self._virtual_gate("CX", (v, q))
            for q in range(self.n):
                if q != v and (p[1] >> q) & 1:
                    p = conjugate(p, "CZ", (v, q))
                    self._virtual_gate("CZ", (v, q))
            if (p[1] >> v) & 1:
                p = conjugate(p, "S", (v,))
                self._virtual_gate("S", (v,))
            assert p[0] == 1 << v and p[1] == 0
            return v, "X", herm_sign(p)
        zs = [q for q in range(self.n) if (z >> q) & 1]
        az = [q for q in zs if q in act]
        if not az:
            return None
        v = az[0]
        for q in zs:
            if q != v:
                p = conjugate(p, "CX", (q, v))
                self._virtual_gate("CX", (q, v))
        assert p[0] == 0 and p[1] == 1 << v
        return v, "Z", herm_sign(p)

    def _plan(self):
        n = self.n
        self.img = {}
        for q in range(n):
            self.img[("X", q)] = (1 << q, 0, 0)
            self.img[("Z", q)] = (0, 1 << q, 0)
        self.active: list[int] = []
        steps = self.steps
        for i, op in enumerate(self.flat.ops):
            if op.kind == "gate" and op.name not in ("T", "T_DAG", "R_Z", "R_X", "R_Y"):
                self._physical_gate(op.name, op.qubits)
            elif op.kind == "gate":
                q = op.qubits[0]
                if op.name in ROT_GEN:
                    letter, theta = ROT_GEN[op.name]
                else:
                    letter, theta = op.name[-1], op.arg / 2.0
                p = self._map({q: letter})
                loc = self._localize(p)
                if loc is None:
                    continue  # scalar phase on the dormant |0>: dropped
                v, kind, a = loc
                ta = theta * (-1 if a else 1)
                if kind == "X" and v not in self.active:
                    self._virtual_gate("H", (v,))
                    self.active.append(v)
                    self.k_max = max(self.k_max, len(self.active))
                    if len(self.active) > self.k_limit:
                        raise ValueError("active dimension over the oracle's limit")
                    steps.append(Step("expand", dict(v=v, theta=ta)))
                else:
                    steps.append(Step("rot", dict(kind=kind, v=v, pos=self.active.index(v), theta=ta)))
            elif op.kind == "meas":
                q = op.qubits[0]
                p = self._map({q: "X" if op.name == "MX" else "Z"})
                common = dict(event=op.event, record=op.record, flip=op.site)
                x, z, _ = p
                act = set(self.active)
                if x == 0 and not any((z >> j) & 1 for j in act):
                    steps.append(Step("mstatic", dict(zmask=z, s=herm_sign(p), **common)))
                else:
                    v, kind, a = self._localize(p)
                    if v not in act:
                        assert kind == "X"
                        steps.append(Step("mrand", dict(v=v, a=a, **common)))
                        self._virtual_gate("H", (v,))   # records H_v, x_v ^= b follows
                        steps.append(Step("xflip", dict(v=v)))
                    else:
                        pos = self.active.index(v)
                        steps.append(Step("mact", dict(kind=kind, v=v, pos=pos, a=a, **common)))
                        top = self.active[-1]
                        self.active[pos] = top
                        self.active.pop()
                        if kind == "X":
                            self._virtual_gate("H", (v,))
                        steps.append(Step("xflip", dict(v=v)))
                if op.reset:
                    e = self._map({q: "X"})
                    steps.append(Step("reset", dict(event=op.event, ex=e[0], ez=e[1])))
            elif op.kind == "ff":
                e = self._map({op.qubits[0]: op.name})
                steps.append(Step("ff", dict(record=op.record, ex=e[0], ez=e[1])))
            elif op.kind == "probe":
                # <P> = <phi (x) 0| Pt^dag M(P) Pt |phi (x) 0> / <phi|phi>: zero if
                # M(P) has x-support on a dormant qubit; dormant Z factors read +1
                x, z, ph = self._map({q: l for q, l in op.paulis})
                act = self.active
                zero = any((x >> q) & 1 and q not in act for q in range(self.n))
                mx = sum(1 << act.index(q) for q in act if (x >> q) & 1)
                mz = sum(1 << act.index(q) for q in act if (z >> q) & 1)
                steps.append(Step("probe", dict(index=op.index, x=x, z=z, ph=ph, mx=mx, mz=mz, zero=zero)))
            elif op.kind == "noise":
                from .circuit import option_count
                opts = []
                for j in range(option_count(op.name)):
                    letters = option_paulis(op.name, j)
                    e = self._map({q: l for q, l in zip(op.qubits, letters) if l != "I"})
                    opts.append((e[0], e[1]))
                steps.append(Step("noise", dict(site=op.site, opts=opts)))

    # ----------------------------------------------------------------------
    # Run
    # ----------------------------------------------------------------------
    def run_raw(self, seed: int, shot: int, noisy: bool = True, faults=None,
                stop_event: int = -1, trace: dict | None = None, argmax: bool = False):
        """Returns (records, frame (x, z), phi, active list). ``trace`` gets
        'p1' {event: P(m=1)}, 'probe' {probe index: expectation value} and
        'k' / 'norm' lists for invariant checks. argmax: every measurement
        takes its more likely outcome, 0 on a tie (the reference trajectory)."""
        f = self.flat
        if faults is None:
            faults = sample_faults(self.table, seed, shot) if noisy else {}
        fx = fz = 0
        phi = np.ones(1, dtype=complex)
        act: list[int] = []
        meas = [0] * f.n_records
        outcome: dict[int, int] = {}
        b_last = 0

        def bit(v, w):
            return (w >> v) & 1

        for st in self.steps:
            a = st.a
            k = len(act)
            if st.kind == "vg":
                fx, fz = _frame_conj(a["name"], a["vq"], fx, fz)
                if a["pos"] is not None:
                    phi = _apply_gate(phi, k, a["name"], a["pos"])
            elif st.kind == "expand":
                v = a["v"]
                th = a["theta"] * (-1 if bit(v, fx) else 1)
                phi = np.concatenate([phi * (np.exp(-1j * th) / math.sqrt(2)),
                                      phi * (np.exp(1j * th) / math.sqrt(2))])
                act.append(v)
            elif st.kind == "rot":
                v, pos = a["v"], a["pos"]
                if a["kind"] == "Z":
                    th = a["theta"] * (-1 if bit(v, fx) else 1)
                    u = np.diag([np.exp(-1j * th), np.exp(1j * th)])
                else:
                    th = a["theta"] * (-1 if bit(v, fz) else 1)
                    u = np.array([[math.cos(th), -1j * math.sin(th)],
                                  [-1j * math.sin(th), math.cos(th)]])
                phi = _apply_1q(phi, k, pos, u)
            elif st.kind in ("mstatic", "mrand", "mact"):
                if a["event"] == stop_event:
                    return meas, (fx, fz), phi, list(act)
                if st.kind == "mstatic":
                    par = bin(fx & a["zmask"]).count("1") & 1
                    m = a["s"] ^ par
                    p1 = float(m)
                elif st.kind == "mrand":
                    p1 = 0.5
                    m = 0 if argmax else (1 if meas_u(seed, shot, a["event"]) < p1 else 0)
                    b_last = m ^ a["a"] ^ bit(a["v"], fz)
                else:
                    v, pos = a["v"], a["pos"]
                    t = phi.reshape([2] * k)
                    ax = k - 1 - pos
                    t0 = np.take(t, 0, axis=ax)
                    t1 = np.take(t, 1, axis=ax)
                    if a["kind"] == "Z":
                        pbit = bit(v, fx)
                        br = (t0, t1)
                    else:
                        pbit = bit(v, fz)
                        br = ((t0 + t1) / math.sqrt(2), (t0 - t1) / math.sqrt(2))
                    s = [float(np.sum(np.abs(x) ** 2)) for x in br]
                    tot = s[0] + s[1]
                    p1 = s[1 ^ a["a"] ^ pbit] / tot
                    m = (1 if p1 > 0.5 else 0) if argmax else (1 if meas_u(seed, shot, a["event"]) < p1 else 0)
                    b = m ^ a["a"] ^ pbit
                    kept = br[b] / math.sqrt(s[b])
                    phi = _relocate(kept, k, pos)
                    act[pos] = act[-1]
                    act.pop()
                    b_last = b
                if trace is not None:
                    trace.setdefault("p1", {})[a["event"]] = p1
                outcome[a["event"]] = m
                if a["record"] >= 0:
                    flip = 1 if (a["flip"] >= 0 and a["flip"] in faults) else 0
                    meas[a["record"]] = m ^ flip
            elif st.kind == "xflip":
                if b_last:
                    fx ^= 1 << a["v"]
            elif st.kind == "reset":
                if outcome[a["event"]]:
                    fx ^= a["ex"]
                    fz ^= a["ez"]
            elif st.kind == "ff":
                if meas[a["record"]]:
                    fx ^= a["ex"]
                    fz ^= a["ez"]
            elif st.kind == "noise":
                opt = faults.get(a["site"])
                if opt is not None:
                    ex, ez = a["opts"][opt]
                    fx ^= ex
                    fz ^= ez
            elif st.kind == "probe" and trace is not None:
                trace.setdefault("probe", {})[a["index"]] = probe_value(a, fx, fz, phi)
            if trace is not None:
                trace.setdefault("k", []).append(len(act))
                trace.setdefault("norm", []).append(float(np.sum(np.abs(phi) ** 2)))
        return meas, (fx, fz), phi, list(act)

    def sample(self, seed: int, shot: int, postselect: bool = False) -> ShotRecords:
        meas = self.run_raw(seed, shot)[0]
        return assemble(self.flat, meas, self.ref_det, self.ref_obs, postselect)


def probe_value(a: dict, fx: int, fz: int, phi: np.ndarray) -> float:
    """<P> of the factored state for a probe step (image i^ph X^x Z^z, active
    position masks mx / mz, dormant-x flag zero) under the frame (fx, fz)."""
    if a["zero"]:
        return 0.0
    # frame conjugation: sign of the anticommutation with the frame
    om = (bin(fx & a["z"]).count("1") + bin(fz & a["x"]).count("1")) & 1
    idx = np.arange(len(phi))
    sg = 1 - 2 * (np.array([bin(int(i) & a["mz"]).count("1") & 1 for i in idx]))
    acc = np.sum(np.conj(phi[idx ^ a["mx"]]) * sg * phi)
    return float(((-1) ** om * (1j ** a["ph"]) * acc).real / np.sum(np.abs(phi) ** 2))


def _frame_conj(name: str, vq: tuple, fx: int, fz: int):
    x, z, _ = conjugate((fx, fz, 0), name, vq)
    return x, z


def _apply_1q(phi, k, pos, u):
    v = phi.reshape(1 << (k - pos - 1), 2, 1 << pos)
    return np.einsum("ab,xby->xay", u, v).reshape(-1)


def _apply_gate(phi, k, name, pos):
    if len(pos) == 1:
        return _apply_1q(phi, k, pos[0], one_q_matrix(name))
    t = phi.reshape([2] * k)
    axes = (k - 1 - pos[0], k - 1 - pos[1])
    t = np.moveaxis(t, axes, (0, 1))
    shp = t.shape
    t = (two_q_matrix(name) @ t.reshape(4, -1)).reshape(shp)
    t = np.moveaxis(t, (0, 1), axes)
    return np.ascontiguousarray(t).reshape(-1)


def _relocate(kept: np.ndarray, k: int, pos: int) -> np.ndarray:
    """``kept`` has the k-1 axes of the old positions (descending, without
    ``pos``). The old top position k-1 takes the freed position ``pos``;
    returns the length 2^(k-1) array indexed by the new positions."""
    old_desc = [p for p in range(k - 1, -1, -1) if p != pos]
    new_of = {p: (pos if (p == k - 1 and pos != k - 1) else p) for p in old_desc}
    if k - 1 == 0:
        return kept.reshape(1)
    # axis order wanted: new positions descending
    want = sorted(old_desc, key=lambda p: -new_of[p])
    perm = [old_desc.index(p) for p in want]
    return np.ascontiguousarray(np.transpose(kept, perm)).reshape(-1)
