#!/usr/bin/env python
"""Benchmark of the sample-many phase (shots/s) on GB300.

Default workload: rotated surface-code memory, d = 5, 25 rounds, p = 1e-3
(49 qubits, k_max = 0), 10^8 shots per step, FP32 batched executor. One
step = one nc_sample call over the whole hot path. The records of a step
(~15 GB) are far larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0). Under torchrun every rank samples its own
disjoint shot range (shot_offset = rank * shots): weak scaling, no
collective on the data path.

--impl reference times the CPU oracle (the frame-factored FP64 oracle) on
the host cores on a bounded sample of the same workload.

--stratum K runs the same workload in stratified importance sampling
(exactly K faults per shot); the line then names the stratum and its weight.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "shots/sec at stated peak active dim (FP32 batched vs FP64 plain); % HBM roofline"


def workload_name(args) -> str:
    name = workload(args.workload)[0]
    return name if args.stratum is None else f"{name}_stratum{args.stratum}"


def workload(name: str):
    from gen import circuits as gc
    if name == "surface":
        return ("surface_code_d5_r25_p1e-3", gc.surface_code_memory(d=5, rounds=25, p=1e-3), 100_000_000, False)
    if name == "tiny":
        return ("tiny_n12_l30_t6", gc.tiny_random(seed=1), 10_000, False)
    if name == "dense":
        return ("dense_n20_l40", gc.dense_random(seed=3, n=20, layers=40), 4096, False)
    if name == "lowmagic":
        # postselection on every detector being zero
        return ("low_magic_n50_k10_p5e-4_postselected", gc.low_magic_gadgets(), 100_000_000, True)
    if name == "coherent":
        return ("coherent_surface_d3_r3_p1e-3_theta0.02",
                gc.surface_code_memory(d=3, rounds=3, p=1e-3, theta=0.02), 10_000_000, False)
    raise SystemExit(f"unknown workload {name}")


def record_bytes_per_shot(info) -> float:
    return (info.n_meas + info.n_det + info.n_obs + 1) / 8.0


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in ("kernels.cu", "kernels.cuh", "program.h", "affine_kernel.cu", "warp_kernel.cu"):
        h.update(open(os.path.join(ROOT, "paper_2604_27058_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def ncu_traffic(workload_name: str, shape=None):
    """DRAM bytes per shot from the committed ncu summary, if it was taken
    on the current kernel source and in the same launch shape."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    except Exception:
        return None
    e = d.get(workload_name)
    if not e or e.get("kernel_sha") != kernel_sha():
        return None
    if shape and e.get("launch_shape") and e["launch_shape"] != shape:
        return None
    return e.get("dram_bytes_per_shot")


class Clocks:
    """nvidia-smi sampling (every 100 ms) around the timed region. A reader
    thread stamps each sample on arrival; start() returns once the sampler
    is producing lines, and only samples stamped inside [start(), stop()]
    are summarised (the first later one if the region was shorter than the
    sampling period)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line))

    def start(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()
        deadline = time.monotonic() + 3.0
        while not self.lines and time.monotonic() < deadline:
            time.sleep(0.01)
        self.t0 = time.monotonic()

    def stop(self):
        if not self.proc:
            return None
        self.t1 = time.monotonic()
        time.sleep(0.25)  # one more sample after the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        inside = [ln for t, ln in self.lines if self.t0 <= t <= self.t1]
        if not inside:
            inside = [ln for t, ln in self.lines if t > self.t1][:1]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in inside:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle leg
# ---------------------------------------------------------------------------
_ORACLE = None


_STRATA = None


def _oracle_init(text, stratum=None):
    global _ORACLE, _STRATA
    from oracle.factored import FactoredSim
    _ORACLE = FactoredSim(text, k_limit=22)
    if stratum is not None:
        from oracle.strata import build_strata
        _STRATA = (build_strata(_ORACLE.flat.site_p, _ORACLE.flat.site_kind, max(stratum, 1)), stratum)


def _oracle_chunk(args):
    seed, start, count = args
    for s in range(start, start + count):
        if _STRATA is None:
            _ORACLE.sample(seed, s)
        else:
            from oracle.records import assemble
            from oracle.strata import sample_stratum_faults
            f = sample_stratum_faults(_STRATA[0], seed, s, _STRATA[1])
            assemble(_ORACLE.flat, _ORACLE.run_raw(seed, s, faults=f)[0], _ORACLE.ref_det, _ORACLE.ref_obs, False)
    return count


def cpu_oracle_rate(text: str, seed: int, budget_s: float, cores: int, stratum=None):
    """Shots/s of the oracle on `cores` processes over a bounded sample."""
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_oracle_init, initargs=(text, stratum)) as pool:
        # warm every worker on one shot (which also calibrates slow
        # workloads), then calibrate on up to 16 shots per worker
        t0 = time.perf_counter()
        pool.map(_oracle_chunk, [(seed, 20_000_000 + i, 1) for i in range(cores)])
        per_shot = time.perf_counter() - t0
        n_cal = max(0, min(16, int(budget_s / 4 / max(per_shot, 1e-6))))
        if n_cal:
            t0 = time.perf_counter()
            pool.map(_oracle_chunk, [(seed, 10_000_000 + i * 16, n_cal) for i in range(cores)])
            per_shot = (time.perf_counter() - t0) / n_cal
        per_worker = max(1, int(budget_s / max(per_shot, 1e-6)))
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_chunk, [(seed, i * per_worker, per_worker) for i in range(cores)]))
        dt = time.perf_counter() - t0
    return done / dt, done, dt


# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    _, text, shots, _ = workload(args.workload)
    wname = workload_name(args)
    cores = os.cpu_count() or 1
    rates = []
    total = 0
    for _ in range(args.warmup):
        cpu_oracle_rate(text, 2002, args.ref_budget / 4, cores, args.stratum)
    for _ in range(args.steps):
        r, n, dt = cpu_oracle_rate(text, 2002, args.ref_budget, cores, args.stratum)
        rates.append(r)
        total += n
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * (total / args.steps) / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": wname, "shots_per_step": total // max(args.steps, 1)},
        "cpu_baseline": {"value": value, "unit": "shots/s", "cores": cores, "kind": "oracle",
                         "sample": f"{total // max(args.steps, 1)} shots per step of {wname}, "
                                   f"frame-factored FP64 oracle, {cores} spawn processes"},
        "e2e": {"value": value, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    _, text, shots, ps = workload(args.workload)
    wname = workload_name(args)
    if args.shots:
        shots = args.shots

    cpu = None
    if rank == 0 and not args.no_cpu:
        cores = os.cpu_count() or 1
        r, n, dt = cpu_oracle_rate(text, 2002, args.cpu_budget, cores, args.stratum)
        cpu = {"value": r, "unit": "shots/s", "cores": cores, "kind": "oracle",
               "sample": f"{n} shots of {wname} in {dt:.1f} s (frame-factored FP64 oracle, "
                         f"{cores} spawn processes)"}

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2604_27058_gb300 import build as nb
    nb.build()
    import paper_2604_27058_gb300 as nc

    prog = nc.compile(text)
    info = prog.info
    bufs = nc.alloc_records(prog, shots)
    from paper_2604_27058_gb300 import shard
    offset, shots = shard.weak(shots, rank)
    stream = torch.cuda.current_stream()
    # launch shape chosen by the autotuner (nc_autotune) unless given
    shape = args.tune
    if shape is None and not args.no_autotune:
        shape = nc.autotune(prog, min(shots, 1 << 22), postselect=ps, stratum=args.stratum)

    def step(precision="fp32", out=None, host=False):
        if host:
            return nc.sample_host(prog, shots, 2002, precision=precision, shot_offset=offset, out=out,
                                  tune=args.tune, stratum=args.stratum, postselect=ps)
        return nc.sample(prog, shots, 2002, precision=precision, shot_offset=offset, out=out or bufs,
                         tune=args.tune, stratum=args.stratum, postselect=ps)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        import torch.distributed as dist
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def timed(precision, steps, warmup, host=False, out=None):
        for _ in range(warmup):
            step(precision, out=out, host=host)
        clocks = Clocks(torch.cuda.current_device())
        barrier()
        torch.cuda.synchronize()
        clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kms, ems, launches = [], [], 0
        for _ in range(steps):
            r = step(precision, out=out, host=host)
            kms.append(r["kernel_ms"])
            ems.append(r["exec_ms"])
            launches += r["launches"]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ck = clocks.stop()
        ms = max_over_ranks(e0.elapsed_time(e1))
        return ms, {"call_ms": kms, "exec_ms": ems, "launches": launches}, ck, r

    ms, tk, ck, last = timed("fp32", args.steps, args.warmup)
    value = shots * world * args.steps / (ms / 1000.0)
    call_ms = statistics.mean(tk["call_ms"])
    exec_ms = statistics.mean(tk["exec_ms"])

    fp64 = None
    if not args.no_fp64:
        # the plain form keeps one 2^k FP64 vector per shot in global memory;
        # past k = 14 that no longer fits for a whole launch, and the FP64
        # batched executor stands in for it
        plain = info.k_max <= 14
        p_steps = max(1, min(args.steps, 3))
        ms64, tk64, _, _ = timed("fp64" if plain else "fp64_batched", p_steps, 1)
        fp64 = {"value": shots * world * p_steps / (ms64 / 1000.0), "unit": "shots/s",
                "ms_per_step": ms64 / p_steps, "exec_ms": statistics.mean(tk64["exec_ms"]),
                "executor": "exec_plain (one thread per shot, FP64)" if plain
                else "exec_batched<double> (FP64 batched; the plain form does not fit at this k)"}

    # FP32 error: the batched FP32 state against the FP64 batched state of the
    # same shots, just before the first measurement event (norm-wise relative
    # error modulo global phase; max-abs amplitude error beside it)
    fp32_err = None
    if info.k_max > 0 and rank == 0 and not args.no_fp64:
        import numpy as np
        errs, aerr, kk = [], [], 0
        for s in range(4 if info.k_max < 16 else 2):
            _, _, p32, k32 = nc.debug_dump(prog, 2002, s, 0, precision="fp32")
            _, _, p64, k64 = nc.debug_dump(prog, 2002, s, 0, precision="fp64_batched")
            if k32 != k64 or k32 == 0:
                continue
            ov = np.vdot(p64, p32)
            ph = ov / abs(ov) if abs(ov) > 0 else 1.0
            errs.append(float(np.linalg.norm(p32 - ph * p64) / np.linalg.norm(p64)))
            aerr.append(float(np.max(np.abs(p32 - ph * p64))))
            kk = k32
        if errs:
            fp32_err = {"state_rel_l2_max": max(errs), "amp_abs_max": max(aerr), "k": kk, "shots": len(errs),
                        "at": "before measurement event 0", "vs": "FP64 batched executor, same shots"}

    e2e = None
    if not args.no_e2e:
        hb = nc.alloc_host_records(prog, shots)
        e_steps = max(1, min(args.steps, 3))
        mse, _, _, rh = timed("fp32", e_steps, 1, host=True, out=hb)
        d2h = sum(b.nbytes for k, b in hb.items() if k != "words_per_record" and b is not None)
        e2e = {"value": shots * world * e_steps / (mse / 1000.0), "unit": "shots/s",
               "h2d_bytes_per_step": 0, "d2h_bytes_per_step": int(d2h),
               "path": "kernels write the pinned host buffers directly" if rh.get("path", 0) & 2
               else "device staging, chunked, copies overlapped on a side stream"}
        del hb
        # host-link peak: a plain pinned device-to-host copy (2 GiB or a step's
        # bytes, whichever is smaller), CUDA events on the same stream
        nbytes = int(min(d2h, 2 << 30)) // 8 * 8
        if nbytes > 0:
            src = torch.ones(nbytes // 8, dtype=torch.int64, device="cuda")
            dst = torch.empty(nbytes // 8, dtype=torch.int64, pin_memory=True)
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            for _ in range(3):
                dst.copy_(src, non_blocking=True)
            c1.record(stream)
            torch.cuda.synchronize()
            gbs = 3 * nbytes / (c0.elapsed_time(c1) / 1000.0) / 1e9
            e2e["host_link"] = {"d2h_gbs": gbs, "bytes": nbytes,
                                "how": "torch pinned copy_ from device, 3 copies, CUDA events"}
            e2e["host_link_frac"] = e2e["value"] * (d2h / shots) / 1e9 / gbs
            del src, dst

    # roofline of the dominant kernel (the record-tile kernel of the k_max = 0
    # path, else the batched executor): algorithmic bytes = the records it
    # must write and the active-vector traversals of the instruction list
    # (before fusion), over its own summed launch time
    peaks, peak_src = measured_peaks()
    # records, plus the active-vector traversals of a program with active axes;
    # with the shared prefix the executor starts every shot from the prefix's
    # vector (one write of it per shot) and runs only the rest of the list
    per_shot = record_bytes_per_shot(info) + info.array_bytes_fp32
    if last.get("path", 0) & 1:
        per_shot += 8.0 * 2 ** info.prefix_k - info.prefix_bytes_fp32
    alg = per_shot * shots
    achieved = alg / (exec_ms / 1000.0) / 1e9
    tr = ncu_traffic(wname, shape)
    affine = info.k_max == 0 and "a=0" not in (args.tune or "")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": (tr * shots) if tr else None,
            "kernel": "sample_affine" if affine else "exec_warp" if "lw=1" in (shape or "")
            else "exec_plain<float>" if "lp=1" in (shape or "") else "exec_batched",
            "peak_source": f"{peak_src} (hbm_gbs, burst copy)",
            "algorithmic_bytes_per_launch": alg, "kernel_ms": exec_ms, "call_ms": call_ms,
            # the DRAM-measured fraction beside the effective one: committed ncu
            # bytes per shot x shots over the same kernel time
            "traffic_frac": (tr * shots / (exec_ms / 1000.0) / 1e9 / peaks["hbm_gbs"]) if tr else None,
            "bytes_model": "records written + active-vector traversals of the unfused instruction list "
                           "(Sec. 2.6 traversal count, 8 B per FP32 amplitude); fused passes, vectors kept in "
                           "shared memory and a shared prefix read as effective bandwidth above the copy peak"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "shots/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32" if info.k_max == 0 else "f32",
            "data": "synthetic",
            "config": {"workload": wname, "shots_per_step_per_gpu": shots, "n_qubits": info.n_qubits,
                       "k_max": info.k_max, "noise_sites": info.n_noise_sites,
                       "record_bits_per_shot": info.n_meas + info.n_det + info.n_obs + 1,
                       "precision": "fp32_batched", "postselect": ps, "launch_shape": shape or "heuristic",
                       "l2": "records per step >> L2 (no flush needed)",
                       "parallelism": f"replicas{world}"},
            **({} if args.stratum is None else
               {"stratum": {"faults_per_shot": args.stratum,
                            "weight": nc.stratum_weights(prog, args.stratum)[0][args.stratum],
                            "sampler": "exactly K faults per shot, conditional jumps (stratified importance "
                                       "sampling)"}}),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "fp64_plain": fp64,
            "fp32_error": fp32_err,
            "gpu_launches": tk["launches"],
            "clocks": ck,
            "shots_kept_last_step": last["shots_kept"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_sweep(args):
    """Batched sweep: 64 seeded circuits of uneven size and active dimension
    (k_max 0..14) sampled by one captured CUDA graph of nc_sample_batch_async
    per step. Shots per circuit are the generator's (10^6..10^8) times
    --sweep-scale. Every program is autotuned first (nc_autotune)."""
    import numpy as np
    import torch
    from gen import circuits as gc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2604_27058_gb300 import build as nb
    nb.build()
    import paper_2604_27058_gb300 as nc

    sweep = gc.sweep_batch(64)
    progs = [nc.compile(c.text) for c in sweep]
    shots = [max(128, int(c.shots * args.sweep_scale)) for c in sweep]
    seeds = [5005 + i for i in range(64)]
    tuned = []
    for p, s in zip(progs, shots):
        nc.prepare(p)
        tuned.append(nc.autotune(p, min(s, 1 << 20)) if not args.no_autotune else "")
    # per-circuit rates, one call each (exec = dominant kernel)
    per = []
    for p, s, sd in zip(progs, shots, seeds):
        nc.sample(p, s, sd)
        r = nc.sample(p, s, sd)
        per.append(s / (r["kernel_ms"] / 1000.0))
    outs = [nc.alloc_records(p, s) for p, s in zip(progs, shots)]
    kept = torch.zeros(len(progs), dtype=torch.int64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = torch.cuda.CUDAGraph()
    one = "mp=1" if args.sweep_one_launch else None
    with torch.cuda.graph(g):
        nc.sample_batch_async(progs, shots, seeds, outs, kept, err, tune=one)
    for _ in range(args.warmup):
        g.replay()
    clocks = Clocks(torch.cuda.current_device())
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    assert int(err.item()) == 0
    total = sum(shots)
    # failure rate per circuit: any nonzero final record (mirror circuits)
    fail = []
    for p, o, s in zip(progs, outs, shots):
        m = nc.unpack_rows(o["meas"][:p.info.n_meas], s)
        fail.append(float(m.any(axis=0).mean()))
    if rank == 0:
        line = {
            "metric": METRIC, "value": total * world * args.steps / (ms / 1000.0), "unit": "shots/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sweep_64_circuits", "shots_per_step_per_gpu": total,
                       "shots_scale": args.sweep_scale, "k_max": [p.info.k_max for p in progs],
                       "graph": "one CUDA graph of nc_sample_batch_async per step: "
                                + ("ONE persistent thread-per-shot executor launch over a work list of every "
                                   "circuit's 128-shot items" if one else
                                   "up to 16 branches, each circuit with its autotuned launch shape"),
                       "parallelism": f"replicas{world}"},
            "per_circuit_shots_per_s": {"min": min(per), "median": float(np.median(per)), "max": max(per)},
            "failure_rate": {"min": min(fail), "median": float(np.median(fail)), "max": max(fail)},
            "autotuned": tuned,
            "gpu_launches": None,
            "clocks": ck,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="surface")
    ap.add_argument("--shots", type=int, default=0)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tune", default=None, help="executor tuning override, e.g. g=64,t=64")
    ap.add_argument("--sweep-scale", type=float, default=0.01, help="sweep workload: shots per circuit scale")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--sweep-one-launch", action="store_true",
                    help="sweep workload: every circuit in one executor launch (tune mp=1)")
    ap.add_argument("--stratum", type=int, default=None,
                    help="stratified importance sampling: exactly K faults per shot")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and not os.environ.get("NC_BENCH_ALLOW_SHORT"):
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "sweep":
        run_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
