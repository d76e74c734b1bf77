"""GPU parity of stratified importance sampling: every sampling path of the
CUDA library (record-level propagation with fault items, with in-kernel
sampling and after an item-list overflow; the batched executor with
per-shot fault lists and with bucketed faults; the plain FP64 executor)
against the oracle, shot by shot, with the fault sets drawn by the oracle's
own stratified sampler. Records are compared bit for bit (integer paths
without exclusion; paths with active amplitudes excluding flagged
near-ties). Full size: 10^8 shots, sampled shots recomputed by the oracle,
plus a property that holds on every shot (exactly K flipped records)."""

import numpy as np
import pytest

from gen import circuits as gc
from oracle.factored import FactoredSim
from oracle.stabilizer import FrameSim
from oracle.strata import build_strata, sample_stratum_faults

from parity import compare, gpu_records

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


def _faults(sim, seed, kk):
    t = build_strata(sim.flat.site_p, sim.flat.site_kind, max(kk, 1))
    return lambda s: sample_stratum_faults(t, seed, s, kk)


def _flip_circuit(n, p0=0.004, dp=0.003):
    """X_ERROR before M on n qubits with unequal probabilities: every fault
    flips exactly one measurement record."""
    lines = [f"X_ERROR({p0 + dp * q:.6f}) {q}" for q in range(n)]
    lines.append("M " + " ".join(map(str, range(n))))
    return "\n".join(lines)


@pytest.mark.parametrize("kk", [1, 3, 7])
@pytest.mark.parametrize("precision,tune", [("fp32", None), ("fp32", "ai=0"), ("fp32", "ac=64"),
                                            ("fp32", "aw=8"), ("fp32", "a=0"), ("fp32", "a=0,g=32,t=256"),
                                            ("fp64", None)])
def test_surface_code_strata_bit_exact(nc, kk, precision, tune):
    """k_max = 0 surface-code memory (d = 3, 3 rounds): records of stratum K
    equal the oracle's on shots spread over several tiles and the ragged
    last one, for every path (ac=64 overflows the item lists, so tiles
    sample in the tile kernel; a=0,g=32,t=256 takes the bucketed executor)."""
    text = gc.surface_code_memory(d=3, rounds=3, p=0.01)
    prog = nc.compile(text)
    sim = FrameSim(text)
    shots, seed, off = 5_000, 707, 128 * 3
    g = gpu_records(prog, shots, seed, precision=precision, tune=tune, stratum=kk, shot_offset=off)
    idx = sorted(set(range(0, shots, 37)) | {1023, 1024, 4095, 4096, shots - 1})
    n_ok, _ = compare(sim, g, [off + i for i in idx], seed, global_offset=off, exact=True,
                      faults=_faults(sim, seed, kk))
    assert n_ok == len(idx)
    assert g["shots_kept"] == shots


@pytest.mark.parametrize("kk", [0, 2, 5])
@pytest.mark.parametrize("precision,tune", [("fp32", None), ("fp32", "g=32,t=256"), ("fp32", "g=2,t=64"),
                                            ("fp64", None), ("fp64_batched", None), ("fp32", "lw=1")])
def test_tiny_workload_strata(nc, kk, precision, tune):
    """Active axes (k_max <= 6): the batched executor with per-shot fault
    lists (default), with bucketed faults (g=32,t=256), FP64 forms."""
    text = gc.tiny_random(seed=1)
    prog = nc.compile(text)
    assert prog.info.k_max > 0
    sim = FactoredSim(text)
    shots, seed = 700, 1001
    g = gpu_records(prog, shots, seed, precision=precision, tune=tune, stratum=kk)
    n_ok, flagged = compare(sim, g, range(0, shots, 3), seed, faults=_faults(sim, seed, kk))
    assert flagged <= 2
    assert n_ok + flagged == len(range(0, shots, 3))


@pytest.mark.parametrize("precision,tune", [("fp32", None), ("fp64", None), ("fp32", "lw=1")])
def test_low_magic_strata_postselected(nc, precision, tune):
    text = gc.low_magic_gadgets()
    prog = nc.compile(text)
    sim = FactoredSim(text)
    shots, seed, kk = 200, 4004, 2
    g = gpu_records(prog, shots, seed, precision=precision, tune=tune, postselect=True, stratum=kk)
    n_ok, flagged = compare(sim, g, range(shots), seed, postselect=True, faults=_faults(sim, seed, kk))
    assert flagged <= 3
    assert g["shots_kept"] == int(g["kept"].sum())
    assert g["shots_kept"] < shots  # two faults trip a detector in most shots


def test_stratum_zero_is_noiseless(nc):
    import torch
    prog = nc.compile(gc.surface_code_memory(d=3, rounds=3, p=0.01))
    a = nc.sample(prog, 3000, 5, stratum=0)
    b = nc.sample(prog, 3000, 5, noiseless=True)
    for key in ("meas", "det", "obs", "kept"):
        assert torch.equal(a[key], b[key]), key
    assert int(a["det"][: prog.info.n_det].count_nonzero()) == 0


def test_every_shot_has_exactly_k_flips_full_size(nc):
    """10^8 shots of stratum K = 3 on a 64-qubit flip circuit: the count of
    ones of every shot's 64 records is exactly 3 (checked on the device for
    all shots), and sampled shots equal the oracle's records."""
    import torch
    n, kk, shots, seed = 64, 3, 100_000_000, 31
    text = _flip_circuit(n)
    prog = nc.compile(text)
    res = nc.sample(prog, shots, seed, stratum=kk)
    rows = res["meas"][:n]
    for b in range(64):
        c = ((rows >> b) & 1).sum(dim=0)
        words = (shots - b + 63) // 64  # words holding a shot at bit b
        assert bool((c[:words] == kk).all()), b
    sim = FrameSim(text)
    rng = np.random.default_rng(1)
    idx = sorted(set(rng.integers(0, shots, 60).tolist()) | {0, 1, shots - 1})
    words = torch.tensor([i // 64 for i in idx], device="cuda")
    sub = rows.index_select(1, words).cpu().numpy()
    faults = _faults(sim, seed, kk)
    for j, s in enumerate(idx):
        got = [int((int(sub[r, j]) >> (s % 64)) & 1) for r in range(n)]
        assert got == sim.run_raw(seed, s, faults=faults(s))[0], s


def test_surface_code_strata_full_size_sampled(nc):
    """10^8 shots of the d = 5, 25-round surface code in stratum K = 4, the
    benchmark's stratified configuration; sampled shots recomputed by the
    oracle."""
    import torch
    text = gc.surface_code_memory(d=5, rounds=25, p=1e-3)
    prog = nc.compile(text)
    sim = FrameSim(text)
    shots, seed, kk = 100_000_000, 2002, 4
    res = nc.sample(prog, shots, seed, stratum=kk)
    rng = np.random.default_rng(2)
    idx = sorted(set(rng.integers(0, shots, 30).tolist()) | {0, shots - 1})
    words = torch.tensor([i // 64 for i in idx], device="cuda")
    info = prog.info
    faults = _faults(sim, seed, kk)
    from oracle.records import assemble
    sub = {k: res[k].index_select(1, words).cpu().numpy() for k in ("meas", "det", "obs")}
    for j, s in enumerate(idx):
        r = assemble(sim.flat, sim.run_raw(seed, s, faults=faults(s))[0], sim.ref_det, sim.ref_obs, False)
        bit = lambda k, row: int((int(sub[k][row, j]) >> (s % 64)) & 1)
        assert [bit("meas", q) for q in range(info.n_meas)] == r.meas, s
        assert [bit("det", q) for q in range(info.n_det)] == r.det, s
        assert [bit("obs", q) for q in range(info.n_obs)] == r.obs, s
    assert res["shots_kept"] == shots


def test_weighted_strata_recover_marginals(nc):
    """The stratified estimator sum_K P(K) mean_K(record) recovers each
    record's flip probability p_i (strata 0..10 carry all but ~2e-7 of the
    mass; stratum 0 flips nothing)."""
    n, seed = 16, 77
    text = _flip_circuit(n, p0=0.01, dp=0.01)
    prog = nc.compile(text)
    w, ok = nc.stratum_weights(prog, 10)
    assert all(ok)
    shots = 1 << 20
    est = np.zeros(n)
    for kk in range(1, 11):
        res = nc.sample(prog, shots, seed + kk, stratum=kk)
        bits = nc.unpack_rows(res["meas"], shots)[:n]
        est += w[kk] * bits.mean(axis=1)
    p = np.array([0.01 + 0.01 * q for q in range(n)])
    sigma = np.sqrt(sum(w[k] ** 2 * 0.25 / shots for k in range(1, 11)))
    assert np.all(np.abs(est - p) < 6 * sigma + 1e-6), (est - p) / sigma


def test_graph_captured_strata_equal_sample(nc):
    import torch
    progs = [nc.compile(gc.surface_code_memory(d=3, rounds=3, p=0.01)), nc.compile(gc.tiny_random(seed=1))]
    shots, seeds, kk = [4_000, 2_000], [11, 12], 3
    ref = [nc.sample(p, s, sd, stratum=kk) for p, s, sd in zip(progs, shots, seeds)]
    outs = [nc.alloc_records(p, s) for p, s in zip(progs, shots)]
    kept = torch.zeros(2, dtype=torch.int64, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for p in progs:
        nc.prepare(p)
    with pytest.raises(nc.NcError):  # tables not uploaded yet
        nc.sample_batch_async(progs, shots, seeds, outs, kept, err, stratum=kk + 20)
    for p in progs:
        nc.strata_prepare(p, kk)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        nc.sample_batch_async(progs, shots, seeds, outs, kept, err, stratum=kk)
    kept.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    for p, o, r in zip(progs, outs, ref):
        i = p.info
        for key, n in (("meas", i.n_meas), ("det", i.n_det), ("obs", i.n_obs), ("kept", 1)):
            assert torch.equal(o[key][:n], r[key][:n]), key


def test_strata_refusals(nc):
    prog = nc.compile("X_ERROR(0.1) 0 1\nM 0 1")
    with pytest.raises(nc.NcError) as e:
        nc.sample(prog, 100, 1, stratum=3)  # only two live sites
    assert e.value.name == "NC_E_ARG"
    with pytest.raises(nc.NcError) as e:
        nc.sample(prog, 100, 1, stratum=200)
    assert e.value.name == "NC_E_ARG"
