"""O-B: dense state-vector simulation of the physical circuit (N <= ~14).

This is the plain definition of what the sampler computes (Sec. 2.1 circuit
model, Def. 2 is only a faster representation of the same state): the
physical state |psi> in C^{2^N} (qubit q is bit q of the basis index) is
evolved gate by gate, a fired noise site applies its physical Pauli, and a
measurement of Z_q (X_q: conjugated by H) draws u from the contract of
``oracle.philox`` and reads m = [u < P(m = 1)], with P taken relative to the
current norm; the state is then projected and renormalised. R and MR apply X
when the (unflipped) outcome is 1. A record-flip site flips only the record.
Classically controlled Paulis read the (possibly flipped) record.
"""

from __future__ import annotations

import numpy as np

from .circuit import Flat, flatten, one_q_matrix, option_paulis, two_q_matrix
from .noise import build_table, sample_faults
from .philox import meas_u
from .records import ShotRecords, assemble, raw_parities


def _apply_1q(psi: np.ndarray, n: int, q: int, u: np.ndarray) -> np.ndarray:
    v = psi.reshape(1 << (n - q - 1), 2, 1 << q)
    return np.einsum("ab,xby->xay", u, v).reshape(-1)


def _apply_2q(psi: np.ndarray, n: int, a: int, b: int, u: np.ndarray) -> np.ndarray:
    # view psi as a rank-n tensor with axis (n-1-q) for qubit q
    t = psi.reshape([2] * n)
    ax_a, ax_b = n - 1 - a, n - 1 - b
    t = np.moveaxis(t, (ax_a, ax_b), (0, 1))
    shp = t.shape
    t = (u @ t.reshape(4, -1)).reshape(shp)
    t = np.moveaxis(t, (0, 1), (ax_a, ax_b))
    return np.ascontiguousarray(t).reshape(-1)


_PAULI = {"X": one_q_matrix("X"), "Y": one_q_matrix("Y"), "Z": one_q_matrix("Z")}


class DenseSim:
    """Physical-picture simulator; also reports P(m = 1) of every event."""

    def __init__(self, text_or_flat, max_qubits: int = 16):
        self.flat: Flat = flatten(text_or_flat) if isinstance(text_or_flat, str) else text_or_flat
        if self.flat.n_qubits > max_qubits:
            raise ValueError(f"dense oracle limited to {max_qubits} qubits")
        self.table = build_table(self.flat.site_p, self.flat.site_kind)
        ref_meas, _, _ = self.run_raw(0, 0, noisy=False, argmax=True)
        self.ref_det, self.ref_obs = raw_parities(self.flat, ref_meas)

    def run_raw(self, seed: int, shot: int, noisy: bool = True, faults=None, stop_event: int = -1,
                probes: dict | None = None, argmax: bool = False):
        """Returns (records, {event: P(m=1)}, state at the stop point).
        ``probes`` (if given) receives {probe index: <psi|P|psi> / <psi|psi>}.
        argmax: every measurement takes its more likely outcome, 0 on a tie
        (the reference trajectory)."""
        f = self.flat
        n = max(1, f.n_qubits)
        psi = np.zeros(1 << n, dtype=complex)
        psi[0] = 1.0
        if faults is None:
            faults = sample_faults(self.table, seed, shot) if noisy else {}
        meas = [0] * f.n_records
        probs: dict[int, float] = {}
        for op in f.ops:
            if op.kind == "gate":
                if len(op.qubits) == 1:
                    psi = _apply_1q(psi, n, op.qubits[0], one_q_matrix(op.name, op.arg))
                else:
                    psi = _apply_2q(psi, n, op.qubits[0], op.qubits[1], two_q_matrix(op.name))
            elif op.kind == "noise":
                opt = faults.get(op.site)
                if opt is not None:
                    for q, letter in zip(op.qubits, option_paulis(op.name, opt)):
                        if letter != "I":
                            psi = _apply_1q(psi, n, q, _PAULI[letter])
            elif op.kind == "meas":
                if op.event == stop_event:
                    return meas, probs, psi
                q = op.qubits[0]
                xb = op.name == "MX"
                if xb:
                    psi = _apply_1q(psi, n, q, one_q_matrix("H"))
                v = psi.reshape(1 << (n - q - 1), 2, 1 << q)
                s0 = float(np.sum(np.abs(v[:, 0, :]) ** 2))
                s1 = float(np.sum(np.abs(v[:, 1, :]) ** 2))
                p1 = s1 / (s0 + s1)
                probs[op.event] = p1
                m = (1 if p1 > 0.5 else 0) if argmax else (1 if meas_u(seed, shot, op.event) < p1 else 0)
                keep = np.zeros_like(v)
                keep[:, m, :] = v[:, m, :]
                psi = keep.reshape(-1) / np.sqrt(s1 if m else s0)
                if xb:
                    psi = _apply_1q(psi, n, q, one_q_matrix("H"))
                if op.reset and m:
                    psi = _apply_1q(psi, n, q, _PAULI["X"])
                if op.record >= 0:
                    flip = 1 if (op.site >= 0 and op.site in faults) else 0
                    meas[op.record] = m ^ flip
            elif op.kind == "ff":
                if meas[op.record]:
                    psi = _apply_1q(psi, n, op.qubits[0], _PAULI[op.name])
            elif op.kind == "probe" and probes is not None:
                ppsi = psi
                for q, letter in op.paulis:
                    ppsi = _apply_1q(ppsi, n, q, _PAULI[letter])
                probes[op.index] = float(np.vdot(psi, ppsi).real / np.vdot(psi, psi).real)
        return meas, probs, psi

    def sample(self, seed: int, shot: int, postselect: bool = False) -> ShotRecords:
        meas, _, _ = self.run_raw(seed, shot)
        return assemble(self.flat, meas, self.ref_det, self.ref_obs, postselect)
