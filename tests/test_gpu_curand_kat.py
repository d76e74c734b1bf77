"""Known-answer check of the oracle's Philox4x32-10 against cuRAND's device
implementation (an independent implementation of the same published
generator). The counter (shot lo, shot hi, tag, index) that both sides use
is cuRAND's state after curand_init(seed, tag | index << 32, 4 * shot)."""

import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle.philox import philox4x32_10

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    d = tempfile.mkdtemp()
    so = os.path.join(d, "libcurand_philox.so")
    subprocess.check_call([nvcc, "-gencode=arch=compute_103a,code=sm_103a", "-O2", "-shared", "-Xcompiler", "-fPIC",
                           os.path.join(HERE, "helpers", "curand_philox.cu"), "-o", so])
    return ctypes.CDLL(so)


def test_oracle_philox_matches_curand(curand_lib):
    import torch
    rng = np.random.default_rng(11)
    n = 256
    seeds = rng.integers(0, 2**63, n, dtype=np.int64).astype(np.uint64)
    shots = rng.integers(0, 2**40, n, dtype=np.int64).astype(np.uint64)
    tags = rng.integers(1, 4, n).astype(np.uint64)
    idx = rng.integers(0, 2**32, n, dtype=np.int64).astype(np.uint64)
    seeds[:3] = [0, 2002, 2**64 - 1]
    shots[:3] = [0, 1, 2**62 - 1]  # curand_init's offset is 4 * shot, so shots stay below 2^62
    subseq = tags | (idx << np.uint64(32))
    dev = {k: torch.from_numpy(v.view(np.int64)).cuda() for k, v in
           (("seed", seeds), ("j", shots), ("sub", subseq))}
    out = torch.zeros((n, 4), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = curand_lib.curand_philox(ctypes.c_void_p(dev["seed"].data_ptr()), ctypes.c_void_p(dev["j"].data_ptr()),
                                  ctypes.c_void_p(dev["sub"].data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_int(n), ctypes.c_void_p(stream))
    assert rc == 0
    got = out.cpu().numpy().view(np.uint32)
    for i in range(n):
        s, j, sub = int(seeds[i]), int(shots[i]), int(subseq[i])
        ctr = (j & 0xFFFFFFFF, j >> 32, sub & 0xFFFFFFFF, sub >> 32)
        key = (s & 0xFFFFFFFF, s >> 32)
        assert tuple(int(x) for x in got[i]) == philox4x32_10(ctr, key), i
