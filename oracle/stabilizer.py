"""O-D: physical Pauli-frame simulation of Clifford + noise circuits, any N.

A second plain definition of the sampler's output for Clifford circuits, in
the physical basis, independent of the frame-factored method:

1. A noiseless reference run on a CHP stabilizer tableau (Aaronson and
   Gottesman, PRA 70, 052328 (2004)) gives, for every measurement event e, its
   reference outcome m_ref[e] (random outcomes are taken as 0), whether it is
   random, and for a random one a stabiliser g_e of the pre-measurement state
   that anticommutes with the measured Pauli (so |psi_1> ~ g_e |psi_0>).
2. Each shot propagates a phase-free physical Pauli frame E (the difference
   between the noisy state and the reference) through the Clifford gates;
   fired noise multiplies E; a measurement of Z_a reads c = x_a(E) and gives
   m = m_ref ^ c (deterministic) or m = [u < 1/2] with E <- E g_e when
   m ^ c ^ m_ref = 1 (random); resets and classically controlled Paulis
   multiply E by the Pauli that the noisy and reference runs apply
   differently.

Gates are decomposed into H, S and CX (the CHP primitive set).
"""

from __future__ import annotations

import numpy as np

from .circuit import Flat, flatten, option_paulis
from .noise import build_table, sample_faults
from .philox import meas_u
from .records import ShotRecords, assemble, raw_parities

# Decompositions into the CHP primitives, applied left to right.
_DECOMP_1Q = {
    "I": [], "H": ["H"], "S": ["S"], "S_DAG": ["S", "S", "S"],
    "X": ["H", "S", "S", "H"], "Z": ["S", "S"], "Y": ["S", "S", "H", "S", "S", "H"],
    "SQRT_X": ["H", "S", "H"], "SQRT_X_DAG": ["H", "S", "S", "S", "H"],
    "SQRT_Y": ["S", "S", "H"], "SQRT_Y_DAG": ["H", "S", "S"],
}


def _decomp_2q(name: str, a: int, b: int):
    if name == "CX":
        return [("CX", a, b)]
    if name == "CZ":
        return [("H", b), ("CX", a, b), ("H", b)]
    if name == "CY":
        return [("S", b), ("S", b), ("S", b), ("CX", a, b), ("S", b)]
    if name == "SWAP":
        return [("CX", a, b), ("CX", b, a), ("CX", a, b)]
    raise ValueError(name)


def primitive_ops(op):
    if len(op.qubits) == 1:
        return [(g, op.qubits[0]) for g in _DECOMP_1Q[op.name]]
    return _decomp_2q(op.name, *op.qubits)


class Tableau:
    """CHP tableau: rows 0..n-1 destabilisers, n..2n-1 stabilisers, 2n scratch."""

    def __init__(self, n: int):
        self.n = n
        self.x = np.zeros((2 * n + 1, n), dtype=np.uint8)
        self.z = np.zeros((2 * n + 1, n), dtype=np.uint8)
        self.r = np.zeros(2 * n + 1, dtype=np.uint8)
        for i in range(n):
            self.x[i, i] = 1
            self.z[n + i, i] = 1

    def h(self, a):
        self.r ^= self.x[:, a] & self.z[:, a]
        self.x[:, a], self.z[:, a] = self.z[:, a].copy(), self.x[:, a].copy()

    def s(self, a):
        self.r ^= self.x[:, a] & self.z[:, a]
        self.z[:, a] ^= self.x[:, a]

    def cx(self, a, b):
        self.r ^= self.x[:, a] & self.z[:, b] & (self.x[:, b] ^ self.z[:, a] ^ 1)
        self.x[:, b] ^= self.x[:, a]
        self.z[:, a] ^= self.z[:, b]

    def apply(self, g, *q):
        {"H": self.h, "S": self.s, "CX": self.cx}[g](*q)

    def _rowsum(self, h: int, i: int):
        x1, z1 = self.x[i].astype(np.int64), self.z[i].astype(np.int64)
        x2, z2 = self.x[h].astype(np.int64), self.z[h].astype(np.int64)
        g = np.where((x1 == 0) & (z1 == 0), 0,
            np.where((x1 == 1) & (z1 == 1), z2 - x2,
            np.where((x1 == 1) & (z1 == 0), z2 * (2 * x2 - 1), x2 * (1 - 2 * z2))))
        tot = (2 * int(self.r[h]) + 2 * int(self.r[i]) + int(g.sum())) % 4
        self.r[h] = 0 if tot == 0 else 1
        self.x[h] ^= self.x[i]
        self.z[h] ^= self.z[i]

    def measure_z(self, a: int, forced: int = 0):
        """Returns (outcome, random?, anticommuting stabiliser (x, z) or None)."""
        n = self.n
        rows = np.nonzero(self.x[n:2 * n, a])[0]
        if len(rows):
            p = n + int(rows[0])
            gx = self.x[p].copy()
            gz = self.z[p].copy()
            for i in range(2 * n):
                if i != p and self.x[i, a]:
                    self._rowsum(i, p)
            self.x[p - n] = self.x[p]
            self.z[p - n] = self.z[p]
            self.r[p - n] = self.r[p]
            self.x[p] = 0
            self.z[p] = 0
            self.z[p, a] = 1
            self.r[p] = forced
            return forced, True, (gx, gz)
        s = 2 * n
        self.x[s] = 0
        self.z[s] = 0
        self.r[s] = 0
        for i in range(n):
            if self.x[i, a]:
                self._rowsum(s, i + n)
        return int(self.r[s]), False, None

    def pauli_x(self, a):
        # conjugating stabilisers by X_a flips the sign of rows with z_a = 1
        self.r ^= self.z[:, a]


def _bits(v: np.ndarray) -> int:
    out = 0
    for j in np.nonzero(v)[0]:
        out |= 1 << int(j)
    return out


class FrameSim:
    """Clifford + noise circuits only (raises on rotations)."""

    def __init__(self, text_or_flat):
        self.flat: Flat = flatten(text_or_flat) if isinstance(text_or_flat, str) else text_or_flat
        f = self.flat
        for op in f.ops:
            if op.kind == "gate" and op.name in ("T", "T_DAG", "R_Z", "R_X", "R_Y"):
                raise ValueError("O-D handles Clifford circuits only")
        self.table = build_table(f.site_p, f.site_kind)
        n = max(1, f.n_qubits)
        tab = Tableau(n)
        self.m_ref = {}
        self.random = {}
        self.flip = {}
        ref_meas = [0] * f.n_records
        for op in f.ops:
            if op.kind == "gate":
                for prim in primitive_ops(op):
                    tab.apply(prim[0], *prim[1:])
            elif op.kind == "meas":
                a = op.qubits[0]
                if op.name == "MX":
                    tab.h(a)
                m, rnd, g = tab.measure_z(a, forced=0)
                if op.name == "MX":
                    tab.h(a)
                self.m_ref[op.event] = m
                self.random[op.event] = rnd
                if rnd:
                    self.flip[op.event] = (_bits(g[0]), _bits(g[1]))
                if op.reset and m:
                    tab.pauli_x(a)
                if op.record >= 0:
                    ref_meas[op.record] = m
            elif op.kind == "ff":
                if ref_meas[op.record]:
                    for prim in _pauli_prims(op.name, op.qubits[0]):
                        tab.apply(prim[0], *prim[1:])
        self.ref_meas = ref_meas
        raw, _ = self.run_raw(0, 0, noisy=False, argmax=True)
        self.ref_det, self.ref_obs = raw_parities(f, raw)

    def run_raw(self, seed: int, shot: int, noisy: bool = True, faults=None, argmax: bool = False):
        """argmax: random measurements take 0 (the reference trajectory)."""
        f = self.flat
        if faults is None:
            faults = sample_faults(self.table, seed, shot) if noisy else {}
        ex = ez = 0
        meas = [0] * f.n_records
        for op in f.ops:
            if op.kind == "gate":
                for prim in primitive_ops(op):
                    ex, ez = _conj(prim, ex, ez)
            elif op.kind == "noise":
                opt = faults.get(op.site)
                if opt is not None:
                    for q, letter in zip(op.qubits, option_paulis(op.name, opt)):
                        if letter in "XY":
                            ex ^= 1 << q
                        if letter in "ZY":
                            ez ^= 1 << q
            elif op.kind == "meas":
                a = op.qubits[0]
                if op.name == "MX":
                    ex, ez = _conj(("H", a), ex, ez)
                c = (ex >> a) & 1
                mr = self.m_ref[op.event]
                if self.random[op.event]:
                    m = 0 if argmax else (1 if meas_u(seed, shot, op.event) < 0.5 else 0)
                    if m ^ c ^ mr:
                        gx, gz = self.flip[op.event]
                        ex ^= gx
                        ez ^= gz
                else:
                    m = mr ^ c
                if op.name == "MX":
                    ex, ez = _conj(("H", a), ex, ez)
                if op.reset and (m ^ mr):
                    ex ^= 1 << a
                if op.record >= 0:
                    meas[op.record] = m ^ (1 if (op.site >= 0 and op.site in faults) else 0)
            elif op.kind == "ff":
                if meas[op.record] ^ self.ref_meas[op.record]:
                    q = op.qubits[0]
                    if op.name in "XY":
                        ex ^= 1 << q
                    if op.name in "ZY":
                        ez ^= 1 << q
        return meas, (ex, ez)

    def sample(self, seed: int, shot: int, postselect: bool = False) -> ShotRecords:
        meas, _ = self.run_raw(seed, shot)
        return assemble(self.flat, meas, self.ref_det, self.ref_obs, postselect)


def _pauli_prims(letter: str, q: int):
    return [(g, q) for g in _DECOMP_1Q[letter]]


def _conj(prim, ex: int, ez: int):
    g = prim[0]
    if g == "H":
        a = prim[1]
        bx, bz = (ex >> a) & 1, (ez >> a) & 1
        if bx != bz:
            ex ^= 1 << a
            ez ^= 1 << a
    elif g == "S":
        a = prim[1]
        if (ex >> a) & 1:
            ez ^= 1 << a
    elif g == "CX":
        a, b = prim[1], prim[2]
        if (ex >> a) & 1:
            ex ^= 1 << b
        if (ez >> b) & 1:
            ez ^= 1 << a
    return ex, ez
