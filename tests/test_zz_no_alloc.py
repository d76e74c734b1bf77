"""nc_sample_noalloc: the sampling call for callers that cannot allocate
device memory while they run. It must give exactly the records nc_sample
gives (same executor, same draws), on consecutive calls that reuse its fixed
scratch array, and refuse work that does not fit that array.

This file is collected last (conftest orders test_zz_* after the rest)."""

import ctypes

import numpy as np
import pytest

from gen import circuits as gc

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


def _noalloc(nc, prog, shots, seed, postselect=False):
    import torch
    from paper_2604_27058_gb300 import _nc
    bufs = nc.alloc_records(prog, shots)
    rec = nc._records_struct(bufs, (shots + 63) // 64)
    opts = nc._opts("fp32", _nc.NC_OUT_ALL, postselect, 0, None, False)
    stream = torch.cuda.current_stream().cuda_stream
    code = _nc.lib().nc_sample_noalloc(prog.handle, shots, seed, ctypes.byref(opts), ctypes.byref(rec),
                                       ctypes.c_void_p(stream))
    return code, bufs, rec


CASES = {
    "surface_d5_r25": (lambda: gc.surface_code_memory(d=5, rounds=25, p=1e-3), 100_000, False),
    "tiny_k6": (lambda: gc.tiny_random(seed=1), 20_000, False),
    "low_magic_k10": (lambda: gc.low_magic_gadgets(), 9_000, True),
    # near-deterministic detectors: the reference trajectory must be nc_sample's
    "coherent_d3_r3": (lambda: gc.surface_code_memory(d=3, rounds=3, p=1e-3, theta=0.02), 6_000, False),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_noalloc_matches_nc_sample(nc, name):
    make, shots, postselect = CASES[name]
    prog = nc.compile(make())
    info = prog.info
    rows = {"meas": info.n_meas, "det": info.n_det, "obs": info.n_obs, "kept": 1}
    ref = nc.sample(prog, shots, 2002, postselect=postselect)
    for _ in range(2):  # two calls in a row reuse the same scratch array
        code, bufs, rec = _noalloc(nc, prog, shots, 2002, postselect=postselect)
        assert code == 0
        for key, n in rows.items():
            got = bufs[key][:n].cpu().numpy()
            want = ref[key][:n].cpu().numpy()
            assert np.array_equal(got, want), key
        assert rec.shots_run == shots
        assert rec.shots_kept == ref["shots_kept"]


def test_noalloc_rejects_oversized_workspace(nc):
    from paper_2604_27058_gb300 import _nc
    prog = nc.compile(gc.dense_random(seed=3, n=20, layers=12), peephole=False)  # every HIR pass off
    assert prog.info.k_max == 20  # one 32-shot tile needs 256 MiB of amplitudes
    code, _, _ = _noalloc(nc, prog, 64, 1)
    assert _nc.STATUS[code] == "NC_E_ARG"


def test_noalloc_matches_the_oracle(nc):
    """Records of the allocation-free call against the FP64 oracle, shot by
    shot (near-ties flagged), on the tiny workload."""
    from parity import compare
    from oracle.factored import FactoredSim
    text = gc.tiny_random(seed=1)
    prog = nc.compile(text)
    shots = 700
    code, bufs, _ = _noalloc(nc, prog, shots, 1001)
    assert code == 0
    info = prog.info
    g = {"meas": nc.unpack_rows(bufs["meas"], shots)[: info.n_meas],
         "det": nc.unpack_rows(bufs["det"], shots)[: info.n_det],
         "obs": nc.unpack_rows(bufs["obs"], shots)[: info.n_obs],
         "kept": nc.unpack_rows(bufs["kept"], shots)[0]}
    n_ok, flagged = compare(FactoredSim(text), g, range(shots), 1001)
    assert flagged <= 3 and n_ok + flagged == shots
