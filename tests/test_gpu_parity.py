"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: records bit-exact (integer paths without any
exclusion; paths with active amplitudes excluding flagged near-ties with
|u - P| < 1e-6); amplitudes norm-wise relative error modulo global phase
<= 1e-5 for the FP32 batched form and <= 1e-10 for the FP64 plain form;
frames bit-exact.
"""

import math

import numpy as np
import pytest

from gen import circuits as gc
from oracle.circuit import flatten
from oracle.dense import DenseSim
from oracle.factored import FactoredSim
from oracle.records import assemble
from oracle.stabilizer import FrameSim

from parity import compare, gpu_records, near_tie, state_error, unpack

pytestmark = pytest.mark.gpu

FP32_AMP_TOL = 1e-5
FP64_AMP_TOL = 1e-10


@pytest.fixture(scope="module")
def nc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_27058_gb300 import build
    build.build()
    import paper_2604_27058_gb300 as m
    return m


def torch_equal(a, b) -> bool:
    import torch
    return bool(torch.equal(a, b))


def _check(oracle_run, ref_det, ref_obs, flat, gpu, seed, shots_idx, cols=None, postselect=False,
           exact=False):
    n = flagged = 0
    for j, s in enumerate(shots_idx):
        col = cols[j] if cols is not None else s
        meas, p1 = oracle_run(s)
        if not exact and p1 and near_tie(p1, seed, s):
            flagged += 1
            continue
        r = assemble(flat, meas, ref_det, ref_obs, postselect)
        assert [int(v) for v in gpu["meas"][:, col]] == r.meas, f"meas mismatch shot {s}"
        assert [int(v) for v in gpu["det"][:, col]] == r.det, f"det mismatch shot {s}"
        assert [int(v) for v in gpu["obs"][:, col]] == r.obs, f"obs mismatch shot {s}"
        assert int(gpu["kept"][col]) == r.kept, f"kept mismatch shot {s}"
        n += 1
    return n, flagged


def _dense_run(sim, seed):
    def f(s):
        m, p, _ = sim.run_raw(seed, s)
        return m, p
    return f


def _factored_run(sim, seed):
    def f(s):
        tr = {}
        m = sim.run_raw(seed, s, trace=tr)[0]
        return m, tr.get("p1", {})
    return f


def _frame_run(sim, seed):
    def f(s):
        return sim.run_raw(seed, s)[0], None
    return f


# ---------------------------------------------------------------------------
# random small circuits: every instruction kind, both forms, several tiles
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision,tune", [("fp32", "g=2,t=64"), ("fp32", None), ("fp64", None),
                                            ("fp32", "sw=0")])
@pytest.mark.parametrize("seed", range(10))
def test_random_small_vs_dense(nc, seed, precision, tune):
    n = 3 + seed % 5
    text = gc.random_small(7000 + seed, n=n, n_ops=70, p_noise=0.04 if seed % 2 else 0.0,
                           t_frac=0.3, meas_frac=0.12)
    prog = nc.compile(text)
    sim = DenseSim(text)
    shots = 300
    g = gpu_records(prog, shots, 31, precision=precision, tune=tune)
    n_ok, flagged = _check(_dense_run(sim, 31), sim.ref_det, sim.ref_obs, sim.flat, g, 31, range(shots))
    assert n_ok + flagged == shots and flagged <= 3


# ---------------------------------------------------------------------------
# workload 1: tiny near-Clifford circuit (n = 12, k_max <= 6)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tiny_workload(nc, precision):
    text = gc.tiny_random(seed=1)
    prog = nc.compile(text)
    assert prog.info.k_max <= 6
    sim = FactoredSim(text)
    shots = 2500
    g = gpu_records(prog, shots, 1001, precision=precision)
    n_ok, flagged = _check(_factored_run(sim, 1001), sim.ref_det, sim.ref_obs, sim.flat, g, 1001,
                           range(shots))
    assert flagged <= 5 and n_ok + flagged == shots


def test_tiny_workload_full_size_sampled(nc):
    text = gc.tiny_random(seed=1)
    prog = nc.compile(text)
    sim = FactoredSim(text)
    shots = 10_000
    for precision in ("fp32", "fp64"):
        g = gpu_records(prog, shots, 1001, precision=precision)
        idx = list(range(0, shots, 97)) + [shots - 1]
        n_ok, flagged = _check(_factored_run(sim, 1001), sim.ref_det, sim.ref_obs, sim.flat, g, 1001, idx)
        assert flagged <= 2


# ---------------------------------------------------------------------------
# workload 2: surface-code memory d=5, 25 rounds (k_max = 0): bit-exact
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision,tune", [("fp32", "a=0,g=4,t=128"), ("fp32", None), ("fp64", None),
                                            ("fp32", "a=0"), ("fp32", "a=0,b=0,ps=1"), ("fp32", "a=0,g=32,t=32,ps=1"),
                                            ("fp32", "aw=4"), ("fp32", "aw=32"), ("fp64", "a=0")])
def test_surface_code_bit_exact(nc, precision, tune):
    text = gc.surface_code_memory(d=5, rounds=25, p=1e-3)
    prog = nc.compile(text)
    sim = FrameSim(text)
    shots = 700
    g = gpu_records(prog, shots, 2002, precision=precision, tune=tune)
    n_ok, _ = _check(_frame_run(sim, 2002), sim.ref_det, sim.ref_obs, sim.flat, g, 2002, range(shots),
                     exact=True)
    assert n_ok == shots
    assert int(g["det"].sum()) > 0


@pytest.mark.parametrize("tune", [None, "aw=8", "ai=0", "ao=1", "ac=100", "av=2048", "a=0", "a=0,ps=1",
                                  "a=0,g=64,t=64,ps=1", "a=0,b=0,ps=1"])
def test_surface_code_many_warp_tiles(nc, tune):
    """Several tiles and a ragged last tile: the record-level propagation
    sampler (default for k_max = 0; faults sampled in a separate pass, or in
    the tile kernel with ai=0, or after an item list overflows with ac=100,
    or in passes of 2048 shots with av=2048, or overlapped with the tile
    kernel on a side stream with ao=1), the executor with bucketed
    noise (a=0,ps=1), with per-shot fault lists (a=0,b=0,ps=1) and with
    faults sampled inside the executor (a=0: calls this small skip the
    pre-sampling passes unless ps=1) give the oracle's records on shots
    spread over every tile."""
    text = gc.surface_code_memory(d=5, rounds=25, p=1e-3)
    prog = nc.compile(text)
    sim = FrameSim(text)
    shots = 9_000
    g = gpu_records(prog, shots, 2003, precision="fp32", tune=tune)
    idx = sorted(set(range(0, shots, 61)) | {1023, 1024, 4095, 4096, shots - 1})
    n_ok, _ = _check(_frame_run(sim, 2003), sim.ref_det, sim.ref_obs, sim.flat, g, 2003, idx, exact=True)
    assert n_ok == len(idx)


@pytest.mark.parametrize("name", ["surface", "random_ff_reset", "random_ff_reset_b"])
def test_affine_sampler_equals_executor(nc, name):
    """k_max = 0: the record-level propagation sampler and the bytecode
    executor give identical records, bit for bit, on every shot (random
    dormant measurements, resets, feed-forward, record flips, detectors)."""
    text = {"surface": lambda: gc.surface_code_memory(d=5, rounds=25, p=1e-3),
            "random_ff_reset": lambda: gc.random_small(41, n=6, n_ops=120, p_noise=0.05, t_frac=0.0),
            "random_ff_reset_b": lambda: gc.random_small(42, n=8, n_ops=200, p_noise=0.03, t_frac=0.0)}[name]()
    prog = nc.compile(text)
    assert prog.info.k_max == 0
    info = prog.info
    rows = {"meas": info.n_meas, "det": info.n_det, "obs": info.n_obs, "kept": 1}
    for shots, off in ((100_003, 0), (777, 128 * 5)):
        a = nc.sample(prog, shots, 99, shot_offset=off)
        b = nc.sample(prog, shots, 99, shot_offset=off, tune="a=0")
        c = nc.sample(prog, shots, 99, shot_offset=off, tune="ai=0")
        for key, n in rows.items():
            assert torch_equal(a[key][:n], b[key][:n]), key
            assert torch_equal(a[key][:n], c[key][:n]), key
        assert a["shots_kept"] == b["shots_kept"] == shots


def test_surface_code_full_size_sampled(nc):
    """10^8 shots in the benchmark's launch configuration; sampled shots are
    recomputed one by one by the oracle."""
    import torch
    text = gc.surface_code_memory(d=5, rounds=25, p=1e-3)
    prog = nc.compile(text)
    sim = FrameSim(text)
    shots = 100_000_000
    res = nc.sample(prog, shots, 2002)
    rng = np.random.default_rng(0)
    idx = sorted(set(rng.integers(0, shots, 40).tolist()) | {0, 63, 64, shots - 1})
    words = torch.tensor([i // 64 for i in idx], device="cuda")
    sub = {k: res[k].index_select(1, words).cpu().numpy() for k in ("meas", "det", "obs", "kept")}
    cols = [i % 64 for i in idx]
    g = {k: np.unpackbits(sub[k].view(np.uint8).reshape(sub[k].shape[0], -1, 8), axis=2,
                          bitorder="little").reshape(sub[k].shape[0], -1)
         for k in sub}
    g = {k: np.stack([g[k][:, j * 64 + c] for j, c in enumerate(cols)], axis=1) for k in g}
    g["kept"] = g["kept"][0]
    n_ok, _ = _check(_frame_run(sim, 2002), sim.ref_det, sim.ref_obs, sim.flat, g, 2002, idx,
                     cols=list(range(len(idx))), exact=True)
    assert n_ok == len(idx)
    assert res["shots_kept"] == shots


# ---------------------------------------------------------------------------
# workload 3: dense limit (k = N); smaller dense case at full parity
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp64_batched"])
def test_dense_small_records_and_amplitudes(nc, precision):
    text = gc.dense_random(seed=33, n=10, layers=12)
    prog = nc.compile(text)
    sim = FactoredSim(text)
    shots = 400
    g = gpu_records(prog, shots, 3003, precision=precision, tune="g=2,t=256" if precision == "fp32" else None)
    n_ok, flagged = _check(_factored_run(sim, 3003), sim.ref_det, sim.ref_obs, sim.flat, g, 3003, range(shots))
    assert flagged <= 4
    tol = FP32_AMP_TOL if precision == "fp32" else FP64_AMP_TOL
    plain = nc.compile(text, peephole=False)  # intermediate states of the plain method
    for shot in (0, 5, 130):
        for ev in (0, 3, 7):
            fx, fz, phi, k = nc.debug_dump(plain, 3003, shot, ev, precision=precision)
            _, (ox, oz), ophi, act = sim.run_raw(3003, shot, stop_event=ev)
            assert k == len(act)
            assert (fx, fz) == (ox, oz)
            assert state_error(phi, ophi) <= tol


def test_dense_k20_mirror_returns_to_zero(nc):
    """n = 20, 12 layers of random H/S/T + CX matchings, then U^dagger: the
    active dimension reaches 20 and every record is 0 (FP32 batched). The
    plain method is compiled: the HIR passes cancel every T against its
    T_DAG and leave no active axis (checked too)."""
    text = gc.dense_random(seed=3, n=20, layers=12, mirror=True)
    prog = nc.compile(text, peephole=False)
    assert prog.info.k_max == 20
    g = gpu_records(prog, 32, 3003, precision="fp32")
    assert int(g["meas"].sum()) == 0
    opt = nc.compile(text)
    assert opt.info.k_max == 0
    assert int(gpu_records(opt, 32, 3003, precision="fp32")["meas"].sum()) == 0


def test_dense_k20_fp32_vs_fp64(nc):
    """n = 20, k = 20: the FP32 batched form against the same layout in FP64
    (records, flagged near-ties aside, and the amplitudes just before the
    final measurements)."""
    text = gc.dense_random(seed=3, n=20, layers=12)
    prog = nc.compile(text, peephole=False)  # the HIR reorder measures earlier (k_max 17)
    assert prog.info.k_max == 20
    shots = 32
    a = gpu_records(prog, shots, 3003, precision="fp32")
    b = gpu_records(prog, shots, 3003, precision="fp64_batched")
    same = (a["meas"] == b["meas"]).all(axis=0)
    assert same.sum() >= shots - 2
    _, _, p32, k32 = nc.debug_dump(prog, 3003, 0, 0, precision="fp32")
    _, _, p64, k64 = nc.debug_dump(prog, 3003, 0, 0, precision="fp64_batched")
    assert k32 == k64 == 20
    assert state_error(p32, p64) <= FP32_AMP_TOL
    assert abs(np.linalg.norm(p64) - 1) < 1e-10


def test_dense_k20_40_layers_vs_oracle(nc):
    """The dense workload at its stated shape (n = 20, 40 layers, k = 20):
    FP32 and FP64-batched amplitudes before the final measurements against
    the FP64 oracle on two shots (the dumps start from the shared noiseless
    prefix, as sampling calls do), and the records of the 4096-shot call on
    four shots, near-ties flagged. The oracle runs in a spawn pool."""
    from parity import oracle_jobs
    text = gc.dense_random(seed=3, n=20, layers=40)
    dump_shots, rec_shots = (0, 77), range(4)
    res = oracle_jobs(text, [("dump", 3003, s, 0) for s in dump_shots] + [("run", 3003, s) for s in rec_shots])
    plain = nc.compile(text, peephole=False)  # the intermediate states of the plain method
    assert plain.info.k_max == 20 and plain.info.prefix_k == 20
    for j, s in enumerate(dump_shots):
        (ox, oz), ophi, act = res[j]
        assert len(act) == 20
        for precision, tol in (("fp32", FP32_AMP_TOL), ("fp64_batched", FP64_AMP_TOL)):
            fx, fz, phi, k = nc.debug_dump(plain, 3003, s, 0, precision=precision)
            assert k == 20 and (fx, fz) == (ox, oz)
            assert state_error(phi, ophi) <= tol, (s, precision)
    prog = nc.compile(text)
    runs = res[len(dump_shots):]
    flat = flatten(text)  # no detectors or observables: empty references
    for precision, shots in (("fp32", 4096), ("fp64_batched", 64)):
        g = gpu_records(prog, shots, 3003, precision=precision)
        n_ok, flagged = _check(lambda s: runs[s], [], [], flat, g, 3003, rec_shots)
        assert n_ok + flagged == len(rec_shots) and flagged <= 1


@pytest.mark.parametrize("precision", ["fp32", "fp64_batched", "fp64"])
def test_dense_k13_amplitudes_vs_oracle(nc, precision):
    text = gc.dense_random(seed=3, n=14, layers=10)
    prog = nc.compile(text, peephole=False)
    sim = FactoredSim(text)
    assert prog.info.k_max == sim.k_max == 13
    tol = FP32_AMP_TOL if precision == "fp32" else FP64_AMP_TOL
    for shot in (0, 77):
        fx, fz, phi, k = nc.debug_dump(prog, 3003, shot, 0, precision=precision)
        _, (ox, oz), ophi, act = sim.run_raw(3003, shot, stop_event=0)
        assert k == len(act) == 13
        assert (fx, fz) == (ox, oz)
        assert state_error(phi, ophi) <= tol


# ---------------------------------------------------------------------------
# workload 4: low-magic gadgets with postselection
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_low_magic_postselected(nc, precision):
    text = gc.low_magic_gadgets()
    prog = nc.compile(text)
    assert prog.info.k_max <= 10
    sim = FactoredSim(text)
    shots = 300
    g = gpu_records(prog, shots, 4004, precision=precision, postselect=True)
    n_ok, flagged = _check(_factored_run(sim, 4004), sim.ref_det, sim.ref_obs, sim.flat, g, 4004,
                           range(shots), postselect=True)
    assert flagged <= 3
    assert g["shots_kept"] == int(g["kept"].sum())


# ---------------------------------------------------------------------------
# workload 5: batched sweep (several circuits in one call)
# ---------------------------------------------------------------------------
def test_sweep_batch_vs_oracle(nc):
    circs = [gc.sweep_mirror(i) for i in range(64)]
    pick = sorted(range(64), key=lambda i: circs[i].n * circs[i].depth)[:4]
    progs = [nc.compile(circs[i].text) for i in pick]
    shots = [200, 333, 64, 129]
    seeds = [5005 + i for i in pick]
    res = nc.sample_batch(progs, shots, seeds)
    for j, i in enumerate(pick):
        sim = FactoredSim(circs[i].text, k_limit=16)
        g = {k: unpack(res[j][k], shots[j]) for k in ("meas", "det", "obs", "kept")}
        g["kept"] = g["kept"][0]
        g["meas"] = g["meas"][: progs[j].info.n_meas]
        g["det"] = g["det"][: progs[j].info.n_det]
        g["obs"] = g["obs"][: progs[j].info.n_obs]
        n_ok, flagged = _check(_factored_run(sim, seeds[j]), sim.ref_det, sim.ref_obs, sim.flat, g,
                               seeds[j], range(0, shots[j], 3))
        assert flagged <= 2


# ---------------------------------------------------------------------------
# edge cases and API semantics
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shots", [1, 31, 32, 33, 64, 65, 129, 4097])
def test_ragged_shot_counts(nc, shots):
    text = gc.surface_code_memory(d=3, rounds=3, p=0.01)
    prog = nc.compile(text)
    sim = FrameSim(text)
    for precision in ("fp32", "fp64"):
        g = gpu_records(prog, shots, 9, precision=precision)
        idx = sorted(set([0, shots - 1] + list(range(0, shots, max(1, shots // 20)))))
        n_ok, _ = _check(_frame_run(sim, 9), sim.ref_det, sim.ref_obs, sim.flat, g, 9, idx, exact=True)
        assert n_ok == len(idx)
        # padding bits beyond `shots` are zero
        raw = g["raw"]
        for key in ("meas", "det", "kept"):
            words = raw[key].cpu().numpy().view(np.uint64)
            if shots % 64:
                assert int(words[:, -1].max() >> np.uint64(shots % 64)) == 0


def test_zero_shots_is_noop(nc):
    prog = nc.compile("H 0\nM 0\n")
    res = nc.sample(prog, 0, 1)
    assert res["shots_run"] == 0


def test_shot_offset_sharding_is_exact(nc):
    text = gc.tiny_random(seed=2)
    prog = nc.compile(text)
    for precision in ("fp32", "fp64"):
        full = gpu_records(prog, 512, 77, precision=precision)
        a = gpu_records(prog, 256, 77, precision=precision, shot_offset=0)
        b = gpu_records(prog, 256, 77, precision=precision, shot_offset=256)
        assert (np.concatenate([a["meas"], b["meas"]], axis=1) == full["meas"]).all()


def test_bad_shot_offset_rejected(nc):
    prog = nc.compile("H 0\nM 0\n")
    with pytest.raises(nc.NcError) as e:
        nc.sample(prog, 64, 1, shot_offset=5)
    assert e.value.name == "NC_E_ARG"


def test_host_output_path_equals_device(nc):
    text = gc.surface_code_memory(d=3, rounds=4, p=0.01)
    prog = nc.compile(text)
    d = nc.sample(prog, 1000, 5)
    h = nc.sample_host(prog, 1000, 5)
    for key in ("meas", "det", "obs", "kept"):
        assert (d[key].cpu().numpy() == h[key]).all()
    assert d["shots_kept"] == h["shots_kept"] == 1000


@pytest.mark.parametrize("case", ["surface", "low_magic_postselected", "fig4"])
def test_host_outputs_direct_and_staged(nc, case):
    """Host outputs reach the caller's pinned buffers straight from the
    kernels (pinned memory the device addresses, with native host atomics:
    path bit 2) or through device staging chunk by chunk with the copies
    overlapped (forced by hd=0; hc= sets the chunk, here three chunks with a
    ragged last one: path bit 4). Both equal the device-buffer records."""
    text, ps = {"surface": (gc.surface_code_memory(d=3, rounds=4, p=0.01), False),
                "low_magic_postselected": (gc.low_magic_gadgets(), True),
                "fig4": (gc.fig4_example(0.05), False)}[case]
    prog = nc.compile(text)
    shots = 3000
    d = nc.sample(prog, shots, 5, postselect=ps)
    for tune, bit in ((None, 2), ("hd=0,hc=1024", 4), ("hd=0", 4)):
        h = nc.sample_host(prog, shots, 5, postselect=ps, tune=tune)
        if tune is None and not h["path"] & 2:
            continue  # this device cannot write the caller's pinned memory directly
        assert h["path"] & bit, (tune, h["path"])
        info = prog.info
        for key, n in (("meas", info.n_meas), ("det", info.n_det), ("obs", info.n_obs), ("kept", 1)):
            assert (d[key][:n].cpu().numpy() == h[key][:n]).all(), (tune, key)
        assert d["shots_kept"] == h["shots_kept"]


def test_deserialized_program_same_records(nc):
    text = gc.low_magic_gadgets()
    p = nc.compile(text)
    q = nc.Program.deserialize(p.serialize())
    a = nc.sample(p, 700, 8, postselect=True)
    b = nc.sample(q, 700, 8, postselect=True)
    for key in ("meas", "det", "obs", "kept"):
        assert (a[key].cpu().numpy() == b[key].cpu().numpy()).all()


def test_batch_equals_individual(nc):
    texts = [gc.surface_code_memory(d=3, rounds=2, p=0.02), gc.tiny_random(seed=4), gc.fig4_example(0.1)]
    progs = [nc.compile(t) for t in texts]
    shots = [100, 300, 65]
    seeds = [1, 2, 3]
    res = nc.sample_batch(progs, shots, seeds)
    for p, s, sd, r in zip(progs, shots, seeds, res):
        one = nc.sample(p, s, sd)
        assert (one["meas"].cpu().numpy() == r["meas"].cpu().numpy()).all()


@pytest.mark.parametrize("postselect", [False, True])
def test_one_launch_batch_equals_individual(nc, postselect):
    """tune "mp=1": every program of a batch (k_max 0 to 10, ragged shot
    counts) in one persistent thread-per-shot launch over a work list of
    128-shot items. Its records equal the thread-per-shot layout run program
    by program (same arithmetic), bit for bit; and the oracle's on sampled
    shots."""
    texts = [gc.surface_code_memory(d=3, rounds=2, p=0.02), gc.tiny_random(seed=4), gc.fig4_example(0.1),
             gc.low_magic_gadgets(), gc.dense_random(seed=33, n=10, layers=12),
             gc.surface_code_memory(d=3, rounds=1, p=1e-3, theta=0.02)]
    progs = [nc.compile(t) for t in texts]
    shots = [1000, 3001, 65, 777, 129, 2048]
    seeds = [1, 2, 3, 4, 5, 6]
    res = nc.sample_batch(progs, shots, seeds, tune="mp=1", postselect=postselect)
    for p, s, sd, r, t in zip(progs, shots, seeds, res, texts):
        assert r["path"] & 8
        one = nc.sample(p, s, sd, tune="lp=1", postselect=postselect)
        info = p.info
        for key, n in (("meas", info.n_meas), ("det", info.n_det), ("obs", info.n_obs), ("kept", 1)):
            assert torch_equal(one[key][:n], r[key][:n]), key
        assert one["shots_kept"] == r["shots_kept"]
        sim = FactoredSim(t)
        g = {k: nc.unpack_rows(r[k], s)[:n] for k, n in (("meas", info.n_meas), ("det", info.n_det),
                                                         ("obs", info.n_obs), ("kept", 1))}
        g["kept"] = g["kept"][0]
        n_ok, flagged = compare(sim, g, range(0, s, max(1, s // 40)), sd, postselect=postselect)
        assert flagged <= 2


def test_one_launch_graph_equals_batch(nc):
    """nc_sample_batch_async with tune "mp=1" captured in a CUDA graph (six
    sweep circuits): one executor launch, the records of nc_sample_batch
    with the same tune, on two replays."""
    import torch
    sweep = gc.sweep_batch(64)
    picks = sorted(range(64), key=lambda i: (gc.sweep_mirror(i).n, i))[:6]
    progs = [nc.compile(sweep[i].text) for i in picks]
    shots = [5_000 + 1_000 * j for j in range(len(progs))]
    seeds = [5005 + i for i in picks]
    ref = nc.sample_batch(progs, shots, seeds, tune="mp=1")
    for p in progs:
        nc.prepare(p)
    outs = [nc.alloc_records(p, s) for p, s in zip(progs, shots)]
    kept = torch.zeros(len(progs), dtype=torch.int64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        nc.sample_batch_async(progs, shots, seeds, outs, kept, err, tune="mp=1")
    for _ in range(2):
        for o in outs:
            for key in ("meas", "det", "obs", "kept"):
                if o[key] is not None:
                    o[key].zero_()
        kept.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        for p, o, r in zip(progs, outs, ref):
            info = p.info
            for key, n in (("meas", info.n_meas), ("det", info.n_det), ("obs", info.n_obs), ("kept", 1)):
                assert torch_equal(o[key][:n], r[key][:n]), key
        assert [int(x) for x in kept.cpu()] == shots


def test_noiseless_option(nc):
    prog = nc.compile(gc.surface_code_memory(d=3, rounds=5, p=0.05))
    r = nc.sample(prog, 5000, 3, noiseless=True)
    assert int(r["det"].abs().sum()) == 0


def test_nondeterministic_detector_reported(nc):
    prog = nc.compile("H 0\nM 0\nDETECTOR rec[-1]\n")
    with pytest.raises(nc.NcError) as e:
        nc.sample(prog, 64, 1)
    assert e.value.name == "NC_E_NONDET_DETECTOR"


def test_near_deterministic_detectors_take_the_likely_reference(nc):
    """R_X(0.1) before M: P(m = 1) = sin^2(0.05); the reference is 0 and
    the detector reads 1 exactly when the measurement reads 1."""
    prog = nc.compile("R_X(0.1) 0\nM 0\nDETECTOR rec[-1]\n")
    res = nc.sample(prog, 100_000, 5)
    meas = nc.unpack_rows(res["meas"], 100_000)[0]
    det = nc.unpack_rows(res["det"], 100_000)[0]
    assert (meas == det).all()
    p = math.sin(0.05) ** 2
    assert abs(meas.mean() - p) < 6 * math.sqrt(p / 100_000)


def test_tuning_variants_agree(nc):
    text = gc.tiny_random(seed=6)
    prog = nc.compile(text)
    base = gpu_records(prog, 1000, 12, precision="fp32")
    for tune in ("g=1,t=32", "g=1,t=1024", "g=8,t=256", "g=4,t=64", "b=0", "g=64,t=64", "g=32,t=256,ps=1",
                 "ps=1,b=0", "g=8,t=512,ps=1", "sw=0", "g=2,t=256,sw=0"):
        g = gpu_records(prog, 1000, 12, precision="fp32", tune=tune)
        assert (g["meas"] == base["meas"]).mean() > 0.999


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_closed_form_t_on_plus_statistics(nc, precision):
    prog = nc.compile("H 0\nT 0\nMX 0\n")
    shots = 200_000
    g = gpu_records(prog, shots, 5, precision=precision)
    p1 = float(g["meas"][0].mean())
    exp = 1 - math.cos(math.pi / 8) ** 2
    assert abs(p1 - exp) <= 5 * math.sqrt(exp * (1 - exp) / shots)


# ---------------------------------------------------------------------------
# batching: many circuits in one captured CUDA graph; the autotuner
# ---------------------------------------------------------------------------
def test_graph_captured_batch_equals_batch(nc):
    """nc_sample_batch_async captured in a CUDA graph (the uneven sweep mix,
    k_max 0..14) gives the records of nc_sample_batch, on two replays."""
    import torch
    sweep = gc.sweep_batch(64)
    picks = sorted(range(64), key=lambda i: (gc.sweep_mirror(i).n, i))[:6]
    progs = [nc.compile(sweep[i].text) for i in picks]
    shots = [5_000 + 1_000 * j for j in range(len(progs))]
    seeds = [5005 + i for i in picks]
    ref = nc.sample_batch(progs, shots, seeds)
    for p in progs:
        nc.prepare(p)
    outs = [nc.alloc_records(p, s) for p, s in zip(progs, shots)]
    kept = torch.zeros(len(progs), dtype=torch.int64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        nc.sample_batch_async(progs, shots, seeds, outs, kept, err)
    for _ in range(2):
        kept.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        for p, o, r, s in zip(progs, outs, ref, shots):
            info = p.info
            for key, n in (("meas", info.n_meas), ("det", info.n_det), ("obs", info.n_obs), ("kept", 1)):
                assert torch_equal(o[key][:n], r[key][:n]), key
        assert [int(x) for x in kept.cpu()] == shots


def test_autotune_keeps_records(nc):
    for text in (gc.surface_code_memory(d=3, rounds=3, p=0.01), gc.tiny_random(seed=2)):
        prog = nc.compile(text)
        before = nc.sample(prog, 20_000, 77)
        best = nc.autotune(prog, 200_000)
        assert best
        after = nc.sample(prog, 20_000, 77)
        info = prog.info
        for key, n in (("meas", info.n_meas), ("det", info.n_det), ("obs", info.n_obs), ("kept", 1)):
            assert torch_equal(before[key][:n], after[key][:n]), (best, key)


# ---------------------------------------------------------------------------
# degenerate and large programs
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("text", ["", "H 0\n", "X_ERROR(0.5) 0 1 2\n", "DEPOLARIZE1(0.2) 0\nH 1\nT 1\n"])
def test_programs_without_records(nc, text):
    """No measurements at all: nothing but the kept row is written, every
    shot is kept."""
    prog = nc.compile(text)
    assert prog.info.n_meas == 0
    res = nc.sample(prog, 1000, 5)
    assert res["shots_kept"] == 1000
    kept = nc.unpack_rows(res["kept"][:1], 1000)
    assert kept.all()


def test_wide_clifford_circuit_bit_exact(nc):
    """1000 qubits (2002 frame planes), noisy CX layers, measurements with
    record flips and detectors: records equal the oracle's frame simulator,
    through the record-level path and through the bytecode executor."""
    import random
    rng = random.Random(9)
    n = 1000
    lines = []
    for layer in range(4):
        q = list(range(n))
        rng.shuffle(q)
        pairs = [q[i:i + 2] for i in range(0, n - 1, 2)]
        lines.append("H " + " ".join(str(x) for x in range(0, n, 3)))
        lines.append("CX " + " ".join(f"{a} {b}" for a, b in pairs))
        lines.append("DEPOLARIZE2(0.002) " + " ".join(f"{a} {b}" for a, b in pairs))
        lines.append("H " + " ".join(str(x) for x in range(0, n, 3)))
    sel = list(range(0, n, 7))
    lines.append("M(0.01) " + " ".join(str(x) for x in sel))
    lines.append("M " + " ".join(str(x) for x in sel))
    for j in range(len(sel)):
        lines.append(f"DETECTOR rec[-{len(sel) - j}] rec[-{2 * len(sel) - j}]")
    text = "\n".join(lines) + "\n"
    prog = nc.compile(text)
    assert prog.info.k_max == 0 and prog.info.n_qubits == n
    sim = FrameSim(text)
    shots = 3000
    idx = sorted(set(range(0, shots, 97)) | {shots - 1})
    for tune in (None, "a=0"):
        g = gpu_records(prog, shots, 4242, tune=tune)
        n_ok, _ = _check(_frame_run(sim, 4242), sim.ref_det, sim.ref_obs, sim.flat, g, 4242, idx, exact=True)
        assert n_ok == len(idx)


# ---------------------------------------------------------------------------
# coherent-noise surface code (R_Z(theta) beside every depolarising channel)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision,tune", [("fp32", None), ("fp64", None), ("fp32", "g=4,t=128"),
                                            ("fp64_batched", None)])
def test_coherent_surface_code(nc, precision, tune):
    """d = 3, 3 rounds, theta = 0.02: every over-rotation is an active
    rotation (k_max = 8); records equal the oracle's shot by shot except
    flagged near-ties."""
    text = gc.surface_code_memory(d=3, rounds=3, p=1e-3, theta=0.02)
    prog = nc.compile(text)
    assert prog.info.k_max == 8
    sim = FactoredSim(text)
    shots = 400
    g = gpu_records(prog, shots, 6006, precision=precision, tune=tune)
    n_ok, flagged = _check(_factored_run(sim, 6006), sim.ref_det, sim.ref_obs, sim.flat, g, 6006, range(shots))
    assert flagged <= 2
    assert n_ok + flagged == shots


def test_coherent_surface_code_amplitudes(nc):
    """The FP32 and FP64 active vectors of the coherent circuit, compiled
    without the HIR peephole (the plain method's k-schedule), equal the
    oracle's just before several measurement events."""
    text = gc.surface_code_memory(d=3, rounds=1, p=1e-3, theta=0.02)
    prog = nc.compile(text, peephole=False)
    sim = FactoredSim(text)
    assert prog.info.k_max == sim.k_max == 8
    for ev in (8, 12, 16, 20):
        for s in (0, 5):
            _, (ox, oz), phi_ref, act = sim.run_raw(7, s, stop_event=ev)
            for precision, tol in (("fp32", FP32_AMP_TOL), ("fp64", FP64_AMP_TOL)):
                fx, fz, amps, k = nc.debug_dump(prog, 7, s, ev, precision=precision)
                assert k == len(act), (ev, s, precision)
                assert (fx, fz) == (ox, oz)
                assert state_error(amps, phi_ref) <= tol, (ev, s, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_peephole_keeps_records(nc, precision):
    """The HIR peephole drops rotations only a phase per measurement branch
    can see: programs compiled with it (k_max 4) and without it (k_max 8)
    give the plain oracle's records shot by shot, near-ties aside."""
    text = gc.surface_code_memory(d=3, rounds=1, p=1e-2, theta=0.05)
    opt, plain = nc.compile(text), nc.compile(text, peephole=False)
    assert (opt.info.k_max, plain.info.k_max) == (4, 8)
    sim = FactoredSim(text)
    shots = 500
    for prog in (opt, plain):
        g = gpu_records(prog, shots, 6116, precision=precision)
        n_ok, flagged = _check(_factored_run(sim, 6116), sim.ref_det, sim.ref_obs, sim.flat, g, 6116,
                               range(shots))
        assert flagged <= 2 and n_ok + flagged == shots
        assert int(g["det"].sum()) > 0


# ---------------------------------------------------------------------------
# shared noiseless prefix (computed once per call, then every shot resumes)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp32", "fp64_batched"])
def test_shared_prefix_equals_per_shot_execution(nc, precision):
    """A dense circuit whose gates all precede its measurements: with the
    prefix computed once (px=2) the records equal the oracle's and the
    per-shot execution (px=0), near-ties aside."""
    text = gc.dense_random(seed=33, n=10, layers=12)
    prog = nc.compile(text)
    assert prog.info.prefix_k == prog.info.k_max >= 8
    sim = FactoredSim(text)
    shots = 256
    shared = gpu_records(prog, shots, 19, precision=precision, tune="px=2")
    assert shared["raw"]["path"] & 1
    plain = gpu_records(prog, shots, 19, precision=precision, tune="px=0")
    assert not plain["raw"]["path"] & 1
    n_ok, flagged = _check(_factored_run(sim, 19), sim.ref_det, sim.ref_obs, sim.flat, shared, 19, range(shots))
    assert flagged <= 3 and n_ok + flagged == shots
    differ = int((shared["meas"] != plain["meas"]).any(axis=0).sum())
    assert differ <= flagged


def test_shared_prefix_k20_mirror_returns_to_zero(nc):
    """The k = 20 mirror circuit through the shared prefix: every record 0
    (the plain method: the HIR passes collapse the mirror to k_max = 0)."""
    prog = nc.compile(gc.dense_random(seed=3, n=20, layers=12, mirror=True), peephole=False)
    res = nc.sample(prog, 256, 3)
    assert res["path"] & 1
    assert int(res["meas"][: prog.info.n_meas].count_nonzero()) == 0
