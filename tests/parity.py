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


# ---------------------------------------------------------------------------
# Slow oracle jobs in parallel (k = 20 workloads: tens of seconds per shot).
# The pool uses "spawn" so that no worker is forked from a process holding a
# CUDA context; start it before the first GPU call of the test.
# ---------------------------------------------------------------------------
_SIMS: dict = {}


def _oracle_job(args):
    text, k_limit, kind, seed, shot, stop_event = args
    from oracle.factored import FactoredSim
    sim = _SIMS.get(text)
    if sim is None:
        sim = _SIMS[text] = FactoredSim(text, k_limit=k_limit)
    if kind == "dump":
        _, frame, phi, act = sim.run_raw(seed, shot, stop_event=stop_event)
        return frame, phi, act
    tr = {}
    meas = sim.run_raw(seed, shot, trace=tr)[0]
    return meas, tr.get("p1", {})


def oracle_jobs(text: str, jobs, k_limit: int = 24, workers: int | None = None):
    """Run FactoredSim jobs ("dump", seed, shot, event) -> (frame, phi, act)
    and ("run", seed, shot) -> (raw records, {event: P(m = 1)}) in a spawn
    process pool; results in job order."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    args = [(text, k_limit, j[0], j[1], j[2], j[3] if len(j) > 3 else -1) for j in jobs]
    n = workers or max(1, min(len(args), os.cpu_count() or 1))
    with ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_oracle_job, args))


# ---------------------------------------------------------------------------
# Rates: logical-error-rate agreement as a two-proportion test at 99 %
# ---------------------------------------------------------------------------
Z99 = 2.576


def two_proportion_ok(k1: int, n1: int, k2: int, n2: int, z: float = Z99) -> bool:
    """|k1/n1 - k2/n2| <= z * sqrt(pbar (1 - pbar) (1/n1 + 1/n2)), pbar the
    pooled rate (equal rates required when pbar is 0 or 1)."""
    pbar = (k1 + k2) / (n1 + n2)
    se = (pbar * (1 - pbar) * (1 / n1 + 1 / n2)) ** 0.5
    return abs(k1 / n1 - k2 / n2) <= z * se


_RATE_SIM = None


def _rate_init(text):
    global _RATE_SIM
    from oracle.factored import FactoredSim
    _RATE_SIM = FactoredSim(text, k_limit=24)


def _rate_chunk(args):
    seed, start, count, postselect = args
    kept = obs_fail = any_fail = 0
    for s in range(start, start + count):
        r = _RATE_SIM.sample(seed, s, postselect=postselect)
        if r.kept:
            kept += 1
            obs_fail += 1 if (r.obs and r.obs[0]) else 0
            any_fail += 1 if any(r.meas) else 0
    return kept, obs_fail, any_fail


def oracle_rates(text: str, seed: int, shots: int, postselect: bool = False, workers: int | None = None):
    """Oracle counts over global shots 0..shots-1 in a spawn pool: (shots,
    kept, kept with observable 0 flipped, kept with any nonzero record)."""
    import multiprocessing as mp
    import os
    n = workers or (os.cpu_count() or 1)
    chunk = max(1, shots // (4 * n))
    jobs = [(seed, a, min(chunk, shots - a), postselect) for a in range(0, shots, chunk)]
    with mp.get_context("spawn").Pool(n, initializer=_rate_init, initargs=(text,)) as pool:
        parts = pool.map(_rate_chunk, jobs)
    return (shots,) + tuple(sum(p[i] for p in parts) for i in range(3))


def _popcount_rows(words) -> int:
    a = np.ascontiguousarray(words.cpu().numpy()).view(np.uint8)
    return int(np.unpackbits(a).sum())


def gpu_rates(prog, shots: int, seed: int, postselect: bool = False):
    """The same counts from one nc_sample call (reduced with torch on the
    device, bits counted on the host)."""
    import paper_2604_27058_gb300 as nc
    res = nc.sample(prog, shots, seed, postselect=postselect)
    i = prog.info
    kept = res["kept"][0]
    obs_fail = _popcount_rows(res["obs"][0] & kept) if i.n_obs else 0
    any_m = None
    for r in range(i.n_meas):
        any_m = res["meas"][r].clone() if any_m is None else any_m | res["meas"][r]
    any_fail = _popcount_rows(any_m & kept) if any_m is not None else 0
    return shots, _popcount_rows(kept), obs_fail, any_fail
