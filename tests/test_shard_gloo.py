"""The multi-GPU path is replicas with disjoint shot ranges. Two gloo ranks on
CPU take their ranges from paper_2604_27058_gb300.shard, compute their shots'
records at the global shot indices (with the oracle, and with the library's
compiled program run by the CPU interpreter of its instruction list), and
the gathered records must equal a single run over the union; the
max-over-ranks reduction the benchmark uses is checked on the same group."""

import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2604_27058_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, mode, q):
    import torch
    import torch.distributed as dist
    from gen import circuits as gc
    from oracle.stabilizer import FrameSim
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sim = FrameSim(gc.surface_code_memory(d=3, rounds=3, p=0.02))
    if mode == "weak":
        off, n = shard.weak(150, rank)
    else:
        off, n = shard.strong(300, rank, world)
    recs = [(off + s, tuple(r.det), tuple(r.obs)) for s in range(n)
            for r in [sim.sample(5, off + s)]]
    out = [None] * world
    dist.all_gather_object(out, recs)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((out, float(t.item())))
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["weak", "strong"])
def test_two_rank_shards_equal_single_run(mode):
    from gen import circuits as gc
    from oracle.stabilizer import FrameSim
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert tmax == 2.0
    flat = [x for part in gathered for x in part]
    idx = [x[0] for x in flat]
    assert len(set(idx)) == len(idx)  # disjoint ranges
    assert all(off % shard.ALIGN == 0 for off in
               ([shard.weak(150, r)[0] for r in range(2)] if mode == "weak" else
                [shard.strong(300, r, 2)[0] for r in range(2)]))
    if mode == "strong":
        assert sorted(idx) == list(range(300))
    sim = FrameSim(gc.surface_code_memory(d=3, rounds=3, p=0.02))
    for s, det, obs in flat:
        r = sim.sample(5, s)
        assert (tuple(r.det), tuple(r.obs)) == (det, obs)


def test_strong_split_covers_exactly():
    for total in (0, 1, 127, 128, 129, 10_000, 10**8 + 3):
        for world in (1, 2, 3, 8):
            parts = [shard.strong(total, r, world) for r in range(world)]
            assert sum(n for _, n in parts) == total
            assert all(off % 128 == 0 for off, _ in parts)
            end = 0
            for off, n in parts:
                if n:
                    assert off == end
                    end = off + n


def _rank_lib(rank, world, port, q):
    """One rank of the library path: compile through libnc (host compiler),
    agree on the program across ranks (blob digest), and run this rank's
    shot range of the compiled instruction list (the CPU interpreter of the
    bytecode) at global shot indices."""
    import hashlib
    import sys

    import torch.distributed as dist
    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "helpers"))
    from bytecode_emu import Program
    from gen import circuits as gc
    from oracle.circuit import flatten

    import paper_2604_27058_gb300 as nc
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    text = gc.surface_code_memory(d=3, rounds=2, p=0.03)
    blob = nc.compile(text).serialize()
    digests = [None] * world
    dist.all_gather_object(digests, hashlib.sha256(blob).hexdigest())
    fl = flatten(text)
    emu = Program(blob, fl.site_p, fl.site_kind)
    off, n = shard.strong(260, rank, world)
    recs = []
    for s in range(off, off + n):
        r = emu.run(9, s)
        recs.append((s, tuple(r["meas"]), tuple(r["det"]), tuple(r["obs"])))
    out = [None] * world
    dist.all_gather_object(out, recs)
    if rank == 0:
        q.put((digests, out))
    dist.destroy_process_group()


def test_two_rank_library_shards_equal_oracle():
    """Two gloo ranks compile the same circuit through the library and get
    the same program; their shot ranges of the compiled program, gathered,
    cover every shot once and equal the oracle's records shot by shot."""
    from gen import circuits as gc
    from oracle.factored import FactoredSim
    from oracle.records import assemble
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_lib, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    digests, gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert digests[0] == digests[1]
    flat = [x for part in gathered for x in part]
    assert sorted(x[0] for x in flat) == list(range(260))
    text = gc.surface_code_memory(d=3, rounds=2, p=0.03)
    sim = FactoredSim(text)
    for s, meas, det, obs in flat:
        want = assemble(sim.flat, sim.run_raw(9, s)[0], sim.ref_det, sim.ref_obs, False)
        assert (list(meas), list(det), list(obs)) == (want.meas, want.det, want.obs), s
