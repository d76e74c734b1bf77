"""ctypes binding of libnc (include/nc.h): argument marshalling only.

Every step of compiling and sampling runs inside libnc; this module converts
Python arguments to the C ABI and wraps device buffers allocated with torch.
If libnc.so is missing it raises instead of falling back to anything else.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnc.so")

NC_FP32_BATCHED = 0
NC_FP64_PLAIN = 1
NC_FP64_BATCHED = 2
NC_OUT_MEAS = 1
NC_OUT_DET = 2
NC_OUT_OBS = 4
NC_OUT_KEPT = 8
NC_OUT_HOST = 16
NC_OUT_EXPVAL = 32
NC_NOALLOC_SCRATCH_BYTES = 64 << 20
NC_OUT_ALL = NC_OUT_MEAS | NC_OUT_DET | NC_OUT_OBS | NC_OUT_KEPT | NC_OUT_EXPVAL
NC_COMPILE_NO_PEEPHOLE = 1
NC_COMPILE_NO_REORDER = 2
NC_COMPILE_NO_FUSE = 4
NC_COMPILE_PLAIN = 7
NC_PS_NONE = 0
NC_PS_ALL_DETECTORS = 1

STATUS = {0: "NC_OK", 1: "NC_E_PARSE", 2: "NC_E_UNSUPPORTED", 3: "NC_E_KMAX",
          4: "NC_E_NONDET_DETECTOR", 5: "NC_E_ARG", 6: "NC_E_OOM", 7: "NC_E_CUDA",
          8: "NC_E_TIMEOUT", 9: "NC_E_INTERNAL"}

EXPORTS = ["nc_compile", "nc_compile_ex", "nc_program_info", "nc_program_serialize", "nc_program_deserialize",
           "nc_sample", "nc_sample_batch", "nc_program_free", "nc_status_str", "nc_debug_dump",
           "nc_abi_version", "nc_sample_noalloc", "nc_program_prepare", "nc_sample_batch_async",
           "nc_autotune", "nc_stratum_weights", "nc_strata_prepare"]


class NcError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        self.code = code
        self.name = STATUS.get(code, str(code))
        super().__init__(f"{self.name}: {msg}" if msg else self.name)


class Info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in (
        "n_qubits", "n_meas", "n_det", "n_obs", "k_max", "n_noise_sites", "n_ops",
        "n_events", "n_slots", "n_static", "n_random", "n_active_meas", "n_array_ops", "n_probes")] + [
        ("array_bytes_fp32", ctypes.c_double), ("prefix_ops", ctypes.c_uint32), ("prefix_k", ctypes.c_uint32),
        ("prefix_bytes_fp32", ctypes.c_double)]


class SampleOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("outputs", ctypes.c_uint32),
                ("postselect", ctypes.c_int), ("shot_offset", ctypes.c_uint64),
                ("tune", ctypes.c_char_p), ("noiseless", ctypes.c_int),
                ("stratified", ctypes.c_uint32), ("stratum", ctypes.c_uint32)]


class Records(ctypes.Structure):
    _fields_ = [("meas", ctypes.c_void_p), ("det", ctypes.c_void_p), ("obs", ctypes.c_void_p),
                ("kept", ctypes.c_void_p), ("words_per_record", ctypes.c_uint64),
                ("shots_run", ctypes.c_uint64), ("shots_kept", ctypes.c_uint64),
                ("kernel_ms", ctypes.c_double), ("exec_ms", ctypes.c_double),
                ("launches", ctypes.c_uint32), ("path", ctypes.c_uint32),
                ("expval", ctypes.c_void_p)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libnc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libnc.so not found at {LIB_PATH}: run paper_2604_27058_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, sz, u32, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint64
    L.nc_compile.argtypes = [ctypes.c_char_p, sz, ctypes.POINTER(vp), ctypes.c_char_p, sz]
    L.nc_compile_ex.argtypes = [ctypes.c_char_p, sz, u32, ctypes.POINTER(vp), ctypes.c_char_p, sz]
    L.nc_program_info.argtypes = [vp, ctypes.POINTER(Info)]
    L.nc_program_serialize.argtypes = [vp, vp, ctypes.POINTER(sz)]
    L.nc_program_deserialize.argtypes = [vp, sz, ctypes.POINTER(vp)]
    L.nc_sample.argtypes = [vp, u64, u64, ctypes.POINTER(SampleOpts), ctypes.POINTER(Records), vp]
    L.nc_sample_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(u64), ctypes.POINTER(u64), u32,
                                  ctypes.POINTER(SampleOpts), ctypes.POINTER(Records), vp]
    L.nc_program_free.argtypes = [vp]
    L.nc_program_free.restype = None
    L.nc_status_str.argtypes = [ctypes.c_int]
    L.nc_status_str.restype = ctypes.c_char_p
    L.nc_debug_dump.argtypes = [vp, u64, u64, u32, ctypes.c_int, ctypes.POINTER(u32),
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u32), vp]
    L.nc_sample_noalloc.argtypes = [vp, u64, u64, ctypes.POINTER(SampleOpts), ctypes.POINTER(Records), vp]
    L.nc_sample_noalloc.restype = ctypes.c_int
    L.nc_program_prepare.argtypes = [vp, vp]
    L.nc_sample_batch_async.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(u64), ctypes.POINTER(u64), u32,
                                        ctypes.POINTER(SampleOpts), ctypes.POINTER(Records), vp, vp, vp]
    L.nc_autotune.argtypes = [vp, u64, ctypes.POINTER(SampleOpts), vp, ctypes.c_char_p, sz]
    L.nc_stratum_weights.argtypes = [vp, u32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint8)]
    L.nc_strata_prepare.argtypes = [vp, u32, vp]
    L.nc_abi_version.argtypes = []
    L.nc_abi_version.restype = u32
    for name in ("nc_compile", "nc_compile_ex", "nc_program_info", "nc_program_serialize", "nc_program_deserialize",
                 "nc_sample", "nc_sample_batch", "nc_debug_dump", "nc_program_prepare", "nc_sample_batch_async",
                 "nc_autotune", "nc_stratum_weights", "nc_strata_prepare"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def check(code: int, msg: str = "") -> None:
    if code != 0:
        raise NcError(code, msg)


@dataclass
class ProgramInfo:
    n_qubits: int
    n_meas: int
    n_det: int
    n_obs: int
    k_max: int
    n_noise_sites: int
    n_ops: int
    n_events: int
    n_slots: int
    n_static: int
    n_random: int
    n_active_meas: int
    n_array_ops: int
    n_probes: int
    array_bytes_fp32: float
    prefix_ops: int
    prefix_k: int
    prefix_bytes_fp32: float
