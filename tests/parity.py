"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the oracle shot by shot, flagging near-ties.

Near-tie rule: a shot is excluded from the exact record comparison when, for
some measurement event with a real draw, |u - P(m = 1)| < 1e-6 with u from
the draw contract and P from the FP64 oracle (the FP32 path may then round
the other way). Integer paths (no active amplitude, k_max = 0) are compared
without any exclusion.
"""

from __future__ import annotations

import numpy as np

from oracle.philox import meas_u

NEAR_TIE = 1e-6


def unpack(rows, shots):
    import paper_2604_27058_gb300 as nc
    return nc.unpack_rows(rows, shots)


def gpu_records(prog, shots, seed, precision="fp32", postselect=False, shot_offset=0, tune=None, stratum=None):
    import paper_2604_27058_gb300 as nc
    res = nc.sample(prog, shots, seed, precision=precision, postselect=postselect,
                    shot_offset=shot_offset, tune=tune, stratum=stratum)
    i = prog.info
    out = {
        "meas": unpack(res["meas"], shots)[: i.n_meas],
        "det": unpack(res["det"], shots)[: i.n_det],
        "obs": unpack(res["obs"], shots)[: i.n_obs],
        "kept": unpack(res["kept"], shots)[0],
        "shots_kept": res["shots_kept"],
        "raw": res,
    }
    return out


def near_tie(p1: dict, seed: int, shot: int) -> bool:
    for e, p in p1.items():
        if abs(meas_u(seed, shot, e) - p) < NEAR_TIE:
            return True
    return False


def compare(oracle, gpu, shots_idx, seed, global_offset=0, postselect=False, exact=False,
            local_idx=None, faults=None):
    """Compare oracle shots (global indices) against the GPU record columns
    (local indices). faults(s), if given, supplies the fault set of global
    shot s (stratified sampling). Returns (n_compared, n_flagged)."""
    from oracle.records import assemble
    flagged = 0
    n = 0
    for j, s in enumerate(shots_idx):
        col = local_idx[j] if local_idx is not None else s - global_offset
        tr = {}
        kw = {} if faults is None else {"faults": faults(s)}
        if hasattr(oracle, "steps"):
            meas = oracle.run_raw(seed, s, trace=tr, **kw)[0]
        else:
            meas = oracle.run_raw(seed, s, **kw)[0]
        if not exact and tr and near_tie(tr.get("p1", {}), seed, s):
            flagged += 1
            continue
        r = assemble(oracle.flat, meas, oracle.ref_det, oracle.ref_obs, postselect)
        got_m = [int(v) for v in gpu["meas"][:, col]] if gpu["meas"].shape[0] else []
        got_d = [int(v) for v in gpu["det"][:, col]] if gpu["det"].shape[0] else []
        got_o = [int(v) for v in gpu["obs"][:, col]] if gpu["obs"].shape[0] else []
        assert got_m == r.meas, f"meas mismatch at shot {s}"
        assert got_d == r.det, f"det mismatch at shot {s}"
        assert got_o == r.obs, f"obs mismatch at shot {s}"
        assert int(gpu["kept"][col]) == r.kept, f"kept mismatch at shot {s}"
        n += 1
    return n, flagged


def state_error(phi_gpu: np.ndarray, phi_ref: np.ndarray) -> float:
    """Norm-wise relative error modulo a global phase."""
    ov = np.vdot(phi_ref, phi_gpu)
    ph = ov / abs(ov) if abs(ov) > 0 else 1.0
    return float(np.linalg.norm(phi_gpu - ph * phi_ref) / np.linalg.norm(phi_ref))
