"""The warp-per-shot layout (exec_warp, tune "lw=1": every shot on one
warp, its active vector in shared memory, its frame in registers) and the
FP32 thread-per-shot layout (exec_plain<float>, tune "lp=1": every shot on
one thread, its vector in global memory, FP64 measurement sums), also in its
persistent form (exec_plain_multi, tune "mp=1", "mg" resident CTAs per SM:
one vector slot per resident thread, reused shot after shot). Records
against the dense oracle (random small circuits with every instruction kind)
and the factored oracle (the workloads), near-ties flagged; records equal
those of the tile layout shot by shot except near-ties; tile boundaries and
ragged ends; postselection with early termination."""

import numpy as np
import pytest

from gen import circuits as gc
from oracle.dense import DenseSim
from oracle.factored import FactoredSim
from oracle.records import assemble

from parity import compare, gpu_records, near_tie

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_27058_gb300 import build
    build.build()
    import paper_2604_27058_gb300 as m
    return m


@pytest.mark.parametrize("precision,tune", [("fp32", "lw=1"), ("fp64_batched", "lw=1"), ("fp32", "lw=1,wn=1"),
                                            ("fp32", "lw=1,wn=3"), ("fp32", "lp=1")])
@pytest.mark.parametrize("seed", range(10))
def test_random_small_vs_dense(nc, seed, precision, tune):
    n = 3 + seed % 5
    text = gc.random_small(7000 + seed, n=n, n_ops=70, p_noise=0.04 if seed % 2 else 0.0,
                           t_frac=0.3, meas_frac=0.12)
    prog = nc.compile(text)
    sim = DenseSim(text)
    shots = 300
    g = gpu_records(prog, shots, 31, precision=precision, tune=tune)
    flagged = 0
    for s in range(shots):
        meas, p1, _ = sim.run_raw(31, s)
        if near_tie(p1, 31, s):
            flagged += 1
            continue
        r = assemble(sim.flat, meas, sim.ref_det, sim.ref_obs, False)
        assert [int(v) for v in g["meas"][:, s]] == r.meas, s
        assert [int(v) for v in g["det"][:, s]] == r.det, s
        assert [int(v) for v in g["obs"][:, s]] == r.obs, s
    assert flagged <= 3


@pytest.mark.parametrize("name,shots,postselect", [("tiny", 2500, False), ("lowmagic", 400, True),
                                                   ("coherent", 400, False), ("dense10", 300, False),
                                                   ("fig4", 777, False)])
@pytest.mark.parametrize("tune", ["lw=1", "lp=1", "mp=1,mg=1"])
def test_workloads_vs_oracle(nc, name, shots, postselect, tune):
    text = {"tiny": lambda: gc.tiny_random(seed=1), "lowmagic": gc.low_magic_gadgets,
            "coherent": lambda: gc.surface_code_memory(d=3, rounds=3, p=1e-3, theta=0.02),
            "dense10": lambda: gc.dense_random(seed=33, n=10, layers=12),
            "fig4": lambda: gc.fig4_example(0.05)}[name]()
    prog = nc.compile(text)
    assert prog.info.k_max > 0
    sim = FactoredSim(text)
    g = gpu_records(prog, shots, 77, tune=tune, postselect=postselect)
    n_ok, flagged = compare(sim, g, range(shots), 77, postselect=postselect)
    assert n_ok + flagged == shots and flagged <= 3
    assert g["shots_kept"] == int(g["kept"].sum())


@pytest.mark.parametrize("shots", [1, 31, 32, 33, 65, 1000, 70_001])
@pytest.mark.parametrize("tune", ["lw=1", "lp=1", "mp=1", "mp=1,mg=1"])
def test_equals_tile_layout(nc, shots, tune):
    """Ragged counts and many tiles: the warp layout's records equal the tile
    layout's on every shot whose draws are not near-ties (postselected
    low-magic workload)."""
    text = gc.low_magic_gadgets()
    prog = nc.compile(text)
    a = gpu_records(prog, shots, 4004, tune=tune, postselect=True)
    b = gpu_records(prog, shots, 4004, postselect=True)
    same = (a["meas"] == b["meas"]).all(axis=0) & (a["det"] == b["det"]).all(axis=0) & (a["kept"] == b["kept"])
    assert int((~same).sum()) <= max(2, shots // 20000)
    # padding bits beyond `shots` are zero
    raw = a["raw"]["kept"].cpu().numpy().view(np.uint64)
    if shots % 64:
        assert int(raw[0, -1] >> np.uint64(shots % 64)) == 0


@pytest.mark.parametrize("tune", ["lw=1", "lp=1", "mp=1,mg=2"])
def test_shot_offset(nc, tune):
    text = gc.tiny_random(seed=2)
    prog = nc.compile(text)
    full = gpu_records(prog, 512, 77, tune=tune)
    a = gpu_records(prog, 256, 77, tune=tune, shot_offset=0)
    b = gpu_records(prog, 256, 77, tune=tune, shot_offset=256)
    assert (np.concatenate([a["meas"], b["meas"]], axis=1) == full["meas"]).all()


def test_outputs_subset(nc):
    """Only detectors requested: the other rows are untouched."""
    import torch
    text = gc.low_magic_gadgets()
    prog = nc.compile(text)
    full = nc.sample(prog, 5000, 9, tune="lw=1")
    part = nc.sample(prog, 5000, 9, tune="lw=1", outputs=nc._nc.NC_OUT_DET)
    n = prog.info.n_det
    assert torch.equal(full["det"][:n], part["det"][:n])
