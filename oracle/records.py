"""Detector / observable / postselection assembly (shared by O-A, O-B, O-D).

Reading of the paper (Sec. 3.2, "Post-selection overhead"; detector
references are not described there):

* a detector's value is the XOR of its records XOR its reference, the value
  it takes on the reference trajectory: noise disabled and every measurement
  taking its more likely outcome (0 on a tie). For a deterministic detector
  that is its value on every noiseless trajectory; for one that small
  coherent rotations make slightly random it is the value of the rotation-free
  limit. Observables likewise;
* with postselection on all detectors, a shot is rejected at its first
  detector that reads 1: that detector still reports 1, every later record
  and detector reports 0, all observables report 0 and ``kept`` is 0.
"""

from __future__ import annotations

from dataclasses import dataclass

from .circuit import Flat


@dataclass
class ShotRecords:
    meas: list        # n_records bits
    det: list         # n_detectors bits
    obs: list         # n_observables bits
    kept: int


def raw_parities(flat: Flat, meas: list[int]) -> tuple[list[int], list[int]]:
    det = [0] * flat.n_detectors
    obs = [0] * flat.n_observables
    for op in flat.ops:
        if op.kind == "det":
            v = 0
            for r in op.recs:
                v ^= meas[r]
            det[op.index] = v
        elif op.kind == "obs":
            for r in op.recs:
                obs[op.index] ^= meas[r]
    return det, obs


def assemble(flat: Flat, meas: list[int], ref_det: list[int], ref_obs: list[int],
             postselect: bool) -> ShotRecords:
    out_meas = list(meas)
    det = [0] * flat.n_detectors
    obs = [0] * flat.n_observables
    alive = True
    n_seen = 0
    cutoff = flat.n_records
    for op in flat.ops:
        if op.kind == "meas" and op.record >= 0:
            n_seen = op.record + 1
        elif op.kind == "det":
            v = ref_det[op.index]
            for r in op.recs:
                v ^= meas[r]
            det[op.index] = v if alive else 0
            if postselect and alive and v:
                alive = False
                cutoff = n_seen
        elif op.kind == "obs":
            for r in op.recs:
                obs[op.index] ^= meas[r]
    obs = [o ^ ref for o, ref in zip(obs, ref_obs)]
    if not alive:
        for r in range(cutoff, flat.n_records):
            out_meas[r] = 0
        obs = [0] * flat.n_observables
    return ShotRecords(meas=out_meas, det=det, obs=obs, kept=1 if alive else 0)


def probe_alive(flat: Flat, meas: list[int], ref_det: list[int], postselect: bool) -> list[int]:
    """1 for every probe that runs while the shot is still kept (always 1
    without postselection). A rejected shot reports 0 for every later probe."""
    alive = True
    out = [1] * flat.n_probes
    for op in flat.ops:
        if op.kind == "det":
            v = ref_det[op.index]
            for r in op.recs:
                v ^= meas[r]
            if postselect and alive and v:
                alive = False
        elif op.kind == "probe":
            out[op.index] = 1 if alive else 0
    return out
