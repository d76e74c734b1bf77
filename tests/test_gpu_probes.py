"""GPU parity of expectation-value probes (EXPVAL, OP_EXPVAL) against the
factored oracle, shot by shot: FP32 batched within 1e-5, FP64 forms within
1e-10 (absolute; every value is in [-1, 1]). Shots with a flagged near-tie
measurement (|u - P| < 1e-6) are left out, as for records."""

import math

import numpy as np
import pytest

from gen import circuits as gc
from oracle.factored import FactoredSim
from oracle.records import probe_alive

from parity import near_tie

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-10, "fp64_batched": 1e-10}


@pytest.fixture(scope="module")
def nc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_27058_gb300 import build
    build.build()
    import paper_2604_27058_gb300 as m
    return m


def _check(nc, text, shots, seed, precision, tune=None, postselect=False, shot_idx=None, max_flag=3):
    prog = nc.compile(text)
    sim = FactoredSim(text)
    res = nc.sample(prog, shots, seed, precision=precision, tune=tune, postselect=postselect)
    ev = res["expval"].cpu().numpy()
    assert ev.shape == (prog.info.n_probes, shots)
    n = flagged = 0
    for s in (shot_idx if shot_idx is not None else range(shots)):
        tr = {}
        meas = sim.run_raw(seed, s, trace=tr)[0]
        if near_tie(tr.get("p1", {}), seed, s):
            flagged += 1
            continue
        alive = probe_alive(sim.flat, meas, sim.ref_det, postselect)
        want = np.array([tr["probe"][j] * alive[j] for j in range(prog.info.n_probes)])
        assert np.max(np.abs(ev[:, s] - want)) <= TOL[precision], (s, ev[:, s], want)
        n += 1
    assert flagged <= max_flag
    return n, ev


@pytest.mark.parametrize("precision,tune", [("fp32", None), ("fp32", "g=2,t=64"), ("fp64", None),
                                            ("fp64_batched", None), ("fp32", "lw=1"), ("fp64_batched", "lw=1")])
@pytest.mark.parametrize("seed", range(4))
def test_random_circuits_with_probes(nc, seed, precision, tune):
    text = gc.with_probes(gc.random_small(900 + seed, n=6, n_ops=90, p_noise=0.05, t_frac=0.3), seed, count=10)
    n, _ = _check(nc, text, 200, 41 + seed, precision, tune)
    assert n >= 190


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_closed_forms(nc, precision):
    text = ("H 0\nT 0\nEXPVAL X0 Y0 Z0\nH 1\nCX 1 2\nCX 2 3\nEXPVAL X1*X2*X3 Z1*Z2 Y1*Y2*X3\n"
            "R_X(0.3) 4\nEXPVAL Z4 Y4\nM 0 1 2 3 4\n")
    prog = nc.compile(text)
    res = nc.sample(prog, 1000, 3, precision=precision)
    ev = res["expval"].cpu().numpy()
    want = [math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0, 1.0, 1.0, -1.0, math.cos(0.3), -math.sin(0.3)]
    assert np.max(np.abs(ev - np.array(want)[:, None])) <= TOL[precision]


@pytest.mark.parametrize("precision,tune", [("fp32", None), ("fp64", None), ("fp32", "lw=1")])
def test_low_magic_postselected_probes(nc, precision, tune):
    """Probes in the postselected low-magic workload: a shot rejected before
    a probe reports 0 there."""
    text = gc.with_probes(gc.low_magic_gadgets(), 5, count=6, max_weight=4)
    n, ev = _check(nc, text, 150, 4004, precision, tune=tune, postselect=True)
    assert n >= 145


def test_clifford_program_probes(nc):
    """k_max = 0 with probes runs on the executor; values are 0 or +-1."""
    text = gc.with_probes(gc.surface_code_memory(d=3, rounds=2, p=0.01), 9, count=8, max_weight=3)
    n, ev = _check(nc, text, 500, 77, "fp32", shot_idx=range(0, 500, 5))
    assert set(np.unique(ev)) <= {-1.0, 0.0, 1.0}


def test_coherent_logical_probe(nc):
    """<Z_L> on a data row of the coherent-noise surface code before the
    final data measurement: the over-rotations pull it just below 1."""
    text = gc.surface_code_memory(d=3, rounds=3, p=1e-3, theta=0.02)
    lines = text.splitlines()
    last_m = max(i for i, ln in enumerate(lines) if ln.startswith("M"))
    data_row = lines[last_m].split()[1:4]
    lines.insert(last_m, "EXPVAL " + "*".join(f"Z{q}" for q in data_row))
    text = "\n".join(lines) + "\n"
    n, ev = _check(nc, text, 300, 6006, "fp32")
    assert n >= 295
    assert 0.5 < float(np.median(np.abs(ev))) <= 1.0


@pytest.mark.parametrize("precision", ["fp32", "fp64_batched"])
def test_dense_probes_through_fused_gathers(nc, precision):
    """Probes inside a dense circuit whose batched list uses the fused index
    map: a gather restores logical order before each probe."""
    text = gc.with_probes(gc.dense_random(seed=33, n=10, layers=12), 3, count=6, max_weight=4)
    prog = nc.compile(text)
    assert prog.info.k_max >= 8
    n, _ = _check(nc, text, 64, 19, precision)
    assert n >= 60


def test_host_and_graph_paths_equal_device(nc):
    import torch
    text = gc.with_probes(gc.random_small(950, n=6, n_ops=90, p_noise=0.05, t_frac=0.3), 1, count=5)
    prog = nc.compile(text)
    a = nc.sample(prog, 3000, 8)
    h = nc.sample_host(prog, 3000, 8)
    # the per-shot FP64 sums are shared-memory atomic adds: equal up to the
    # order of the additions
    d = float(np.max(np.abs(a["expval"].cpu().numpy() - h["expval"])))
    assert d <= 1e-12, d
    # staged host outputs: probe rows copied chunk by chunk (three chunks)
    h2 = nc.sample_host(prog, 3000, 8, tune="hd=0,hc=1024")
    assert h2["path"] & 4
    d = float(np.max(np.abs(a["expval"].cpu().numpy() - h2["expval"])))
    assert d <= 1e-12, d
    nc.prepare(prog)
    outs = [nc.alloc_records(prog, 3000)]
    kept = torch.zeros(1, dtype=torch.int64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        nc.sample_batch_async([prog], [3000], [8], outs, kept, err)
    g.replay()
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    d = float((outs[0]["expval"] - a["expval"]).abs().max())
    assert d <= 1e-12, d


def test_probe_outputs_optional(nc):
    text = "H 0\nEXPVAL X0\nM 0\n"
    prog = nc.compile(text)
    res = nc.sample(prog, 100, 1, outputs=nc.NC_OUT_MEAS | nc.NC_OUT_KEPT)
    assert res["expval"] is None
