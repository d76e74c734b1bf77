"""GB300-native near-Clifford shot sampler (frame-factored simulation,
Clifft, arXiv 2604.27058): compile once on the host, sample many shots on
one GPU.

    prog = compile(text)                       # nc_compile
    rec = sample(prog, shots, seed)            # nc_sample into torch tensors
    rec = sample_host(prog, shots, seed)       # nc_sample with host buffers
    rec = sample(prog, shots, seed, stratum=K) # exactly K faults per shot
    w, ok = stratum_weights(prog, k_max)       # P(K faults), K = 0..k_max

Record tensors are int64 views of the bit-packed uint64 rows of include/nc.h:
bit (s % 64) of word [r, s // 64] is record r of shot s.
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import _nc
from ._nc import (NC_FP32_BATCHED, NC_FP64_BATCHED, NC_FP64_PLAIN, NC_OUT_ALL, NC_OUT_DET, NC_OUT_EXPVAL,
                  NC_OUT_HOST, NC_OUT_KEPT, NC_OUT_MEAS, NC_OUT_OBS, NC_PS_ALL_DETECTORS, NC_PS_NONE,
                  NcError, ProgramInfo)

__all__ = ["Program", "compile", "sample", "sample_host", "sample_batch", "debug_dump",
           "stratum_weights", "strata_prepare", "unpack_rows", "NcError", "NC_FP32_BATCHED", "NC_FP64_PLAIN"]

PRECISION = {"fp32": NC_FP32_BATCHED, "fp64": NC_FP64_PLAIN, "fp64_batched": NC_FP64_BATCHED,
             NC_FP32_BATCHED: NC_FP32_BATCHED, NC_FP64_PLAIN: NC_FP64_PLAIN,
             NC_FP64_BATCHED: NC_FP64_BATCHED}


class Program:
    """A compiled program (owned by libnc)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        info = _nc.Info()
        _nc.check(_nc.lib().nc_program_info(self._h, ctypes.byref(info)))
        self.info = ProgramInfo(*[getattr(info, f) for f, _ in _nc.Info._fields_])

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def serialize(self) -> bytes:
        L = _nc.lib()
        n = ctypes.c_size_t(0)
        _nc.check(L.nc_program_serialize(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _nc.check(L.nc_program_serialize(self._h, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    @classmethod
    def deserialize(cls, blob: bytes) -> "Program":
        h = ctypes.c_void_p()
        _nc.check(_nc.lib().nc_program_deserialize(blob, len(blob), ctypes.byref(h)))
        return cls(h.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _nc.lib().nc_program_free(h)
            except Exception:
                pass
            self._h = None


def compile(text: str, peephole: bool = True, flags: int | None = None) -> Program:  # noqa: A001 - mirrors nc_compile
    """nc_compile_ex. peephole=False compiles the plain method
    (NC_COMPILE_PLAIN: no HIR pass, so the k-schedule and intermediate states
    are those of App. B); flags, when given, are the NC_COMPILE_* bits
    themselves."""
    data = text.encode()
    h = ctypes.c_void_p()
    err = ctypes.create_string_buffer(512)
    if flags is None:
        flags = 0 if peephole else _nc.NC_COMPILE_PLAIN
    code = _nc.lib().nc_compile_ex(data, len(data), flags, ctypes.byref(h), err, 512)
    _nc.check(code, err.value.decode(errors="replace"))
    return Program(h.value)


def _opts(precision, outputs, postselect, shot_offset, tune, noiseless, stratum=None):
    o = _nc.SampleOpts()
    o.precision = PRECISION[precision]
    o.outputs = outputs
    o.postselect = NC_PS_ALL_DETECTORS if postselect else NC_PS_NONE
    o.shot_offset = shot_offset
    o.tune = tune.encode() if tune else None
    o.noiseless = 1 if noiseless else 0
    o.stratified = 0 if stratum is None else 1
    o.stratum = 0 if stratum is None else int(stratum)
    return o


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def alloc_records(prog: Program, shots: int, device="cuda", outputs=NC_OUT_ALL):
    """Device record tensors (torch, int64 view of uint64 words) and, for a
    program with probes, an FP64 [n_probes, shots] expectation tensor."""
    import torch
    wpr = (shots + 63) // 64
    i = prog.info
    mk = lambda rows: torch.empty((max(rows, 1), max(wpr, 1)), dtype=torch.int64, device=device)
    ev = (outputs & NC_OUT_EXPVAL) and i.n_probes
    return {
        "meas": mk(i.n_meas) if outputs & NC_OUT_MEAS else None,
        "det": mk(i.n_det) if outputs & NC_OUT_DET else None,
        "obs": mk(i.n_obs) if outputs & NC_OUT_OBS else None,
        "kept": mk(1) if outputs & NC_OUT_KEPT else None,
        "expval": torch.empty((i.n_probes, max(shots, 1)), dtype=torch.float64, device=device) if ev else None,
        "words_per_record": wpr,
    }


def _records_struct(bufs, wpr, host=False):
    r = _nc.Records()
    for key in ("meas", "det", "obs", "kept", "expval"):
        t = bufs.get(key)
        if t is None:
            setattr(r, key, None)
        elif host:
            setattr(r, key, t.ctypes.data)
        else:
            setattr(r, key, t.data_ptr())
    r.words_per_record = wpr
    return r


def sample(prog: Program, shots: int, seed: int, precision="fp32", outputs=NC_OUT_ALL,
           postselect=False, shot_offset=0, tune=None, stream=None, out=None, noiseless=False, stratum=None):
    """nc_sample into device tensors; returns the buffer dict plus counts.
    stratum=K runs stratified importance sampling: exactly K faults per shot
    (weights from stratum_weights)."""
    bufs = out if out is not None else alloc_records(prog, shots, outputs=outputs)
    wpr = (shots + 63) // 64
    rec = _records_struct(bufs, wpr)
    opts = _opts(precision, outputs, postselect, shot_offset, tune, noiseless, stratum)
    _nc.check(_nc.lib().nc_sample(prog.handle, shots, seed, ctypes.byref(opts), ctypes.byref(rec),
                                  ctypes.c_void_p(_stream_ptr(stream))))
    res = dict(bufs)
    res["shots_run"] = rec.shots_run
    res["shots_kept"] = rec.shots_kept
    res["kernel_ms"] = rec.kernel_ms
    res["exec_ms"] = rec.exec_ms
    res["launches"] = rec.launches
    res["path"] = rec.path
    return res


def alloc_host_records(prog: Program, shots: int, outputs=NC_OUT_ALL, pinned=True):
    wpr = (shots + 63) // 64
    i = prog.info
    if pinned:
        import torch

        def mk(rows):
            return torch.empty((max(rows, 1), max(wpr, 1)), dtype=torch.int64, pin_memory=True).numpy()
    else:
        def mk(rows):
            return np.empty((max(rows, 1), max(wpr, 1)), dtype=np.int64)
    ev = (outputs & NC_OUT_EXPVAL) and i.n_probes
    return {
        "meas": mk(i.n_meas) if outputs & NC_OUT_MEAS else None,
        "det": mk(i.n_det) if outputs & NC_OUT_DET else None,
        "obs": mk(i.n_obs) if outputs & NC_OUT_OBS else None,
        "kept": mk(1) if outputs & NC_OUT_KEPT else None,
        "expval": _host_f64((i.n_probes, max(shots, 1)), pinned) if ev else None,
        "words_per_record": wpr,
    }


def _host_f64(shape, pinned):
    if pinned:
        import torch
        return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    return np.empty(shape, dtype=np.float64)


def sample_host(prog: Program, shots: int, seed: int, precision="fp32", outputs=NC_OUT_ALL,
                postselect=False, shot_offset=0, tune=None, stream=None, out=None, noiseless=False,
                stratum=None):
    """nc_sample with NC_OUT_HOST: records land in host (numpy) arrays."""
    bufs = out if out is not None else alloc_host_records(prog, shots, outputs)
    wpr = (shots + 63) // 64
    rec = _records_struct(bufs, wpr, host=True)
    opts = _opts(precision, outputs | NC_OUT_HOST, postselect, shot_offset, tune, noiseless, stratum)
    _nc.check(_nc.lib().nc_sample(prog.handle, shots, seed, ctypes.byref(opts), ctypes.byref(rec),
                                  ctypes.c_void_p(_stream_ptr(stream))))
    res = dict(bufs)
    res["shots_run"] = rec.shots_run
    res["shots_kept"] = rec.shots_kept
    res["kernel_ms"] = rec.kernel_ms
    res["exec_ms"] = rec.exec_ms
    res["launches"] = rec.launches
    res["path"] = rec.path
    return res


def sample_batch(progs, shots, seeds, precision="fp32", outputs=NC_OUT_ALL, postselect=False,
                 tune=None, stream=None, outs=None, stratum=None):
    n = len(progs)
    outs = outs if outs is not None else [alloc_records(p, s, outputs=outputs) for p, s in zip(progs, shots)]
    handles = (ctypes.c_void_p * n)(*[p.handle for p in progs])
    sh = (ctypes.c_uint64 * n)(*shots)
    sd = (ctypes.c_uint64 * n)(*seeds)
    recs = (_nc.Records * n)(*[_records_struct(b, (s + 63) // 64) for b, s in zip(outs, shots)])
    opts = _opts(precision, outputs, postselect, 0, tune, False, stratum)
    _nc.check(_nc.lib().nc_sample_batch(handles, sh, sd, n, ctypes.byref(opts), recs,
                                        ctypes.c_void_p(_stream_ptr(stream))))
    res = []
    for b, r in zip(outs, recs):
        d = dict(b)
        d["shots_run"] = r.shots_run
        d["shots_kept"] = r.shots_kept
        d["kernel_ms"] = r.kernel_ms
        d["exec_ms"] = r.exec_ms
        d["launches"] = r.launches
        d["path"] = r.path
        res.append(d)
    return res


def prepare(prog: Program, stream=None) -> None:
    """nc_program_prepare: upload and reference launch (synchronises)."""
    _nc.check(_nc.lib().nc_program_prepare(prog.handle, ctypes.c_void_p(_stream_ptr(stream))))


def sample_batch_async(progs, shots, seeds, outs, kept_dev, err_dev, precision="fp32", outputs=NC_OUT_ALL,
                       postselect=False, tune=None, stream=None, stratum=None):
    """nc_sample_batch_async: enqueue only (capturable in a CUDA graph).
    outs: record buffers from alloc_records; kept_dev: int64 device tensor
    of len(progs) and err_dev: int32 device tensor of 1, both zeroed by the
    caller."""
    n = len(progs)
    handles = (ctypes.c_void_p * n)(*[p.handle for p in progs])
    sh = (ctypes.c_uint64 * n)(*shots)
    sd = (ctypes.c_uint64 * n)(*seeds)
    recs = (_nc.Records * n)(*[_records_struct(b, (s + 63) // 64) for b, s in zip(outs, shots)])
    opts = _opts(precision, outputs, postselect, 0, tune, False, stratum)
    _nc.check(_nc.lib().nc_sample_batch_async(handles, sh, sd, n, ctypes.byref(opts), recs,
                                              ctypes.c_void_p(kept_dev.data_ptr()),
                                              ctypes.c_void_p(err_dev.data_ptr()),
                                              ctypes.c_void_p(_stream_ptr(stream))))


def autotune(prog: Program, shots: int, precision="fp32", outputs=NC_OUT_ALL, postselect=False,
             stream=None, stratum=None) -> str:
    """nc_autotune: returns the chosen launch shape (used by later calls
    with tune=None on this device)."""
    opts = _opts(precision, outputs, postselect, 0, None, False, stratum)
    buf = ctypes.create_string_buffer(128)
    _nc.check(_nc.lib().nc_autotune(prog.handle, shots, ctypes.byref(opts), ctypes.c_void_p(_stream_ptr(stream)),
                                    buf, 128))
    return buf.value.decode()


def stratum_weights(prog: Program, k_max: int):
    """nc_stratum_weights: (P(exactly K faults) for K = 0..k_max, and
    whether each stratum can be sampled). Host computation."""
    w = (ctypes.c_double * (k_max + 1))()
    v = (ctypes.c_uint8 * (k_max + 1))()
    _nc.check(_nc.lib().nc_stratum_weights(prog.handle, k_max, w, v))
    return list(w), [bool(x) for x in v]


def strata_prepare(prog: Program, k_max: int, stream=None) -> None:
    """nc_strata_prepare: upload the stratified tables up to k_max (needed
    before sample_batch_async with a stratum)."""
    _nc.check(_nc.lib().nc_strata_prepare(prog.handle, k_max, ctypes.c_void_p(_stream_ptr(stream))))


def debug_dump(prog: Program, seed: int, shot: int, event: int, precision="fp32", stream=None):
    """(frame x bits, frame z bits, amplitudes (complex128), k) just before
    measurement event ``event`` of global shot ``shot``."""
    nw = (max(prog.info.n_qubits, 1) + 31) // 32
    frame = (ctypes.c_uint32 * (2 * nw))()
    amps = (ctypes.c_double * (2 << prog.info.k_max))()
    k = ctypes.c_uint32(0)
    _nc.check(_nc.lib().nc_debug_dump(prog.handle, seed, shot, event, PRECISION[precision], frame, amps,
                                      ctypes.byref(k), ctypes.c_void_p(_stream_ptr(stream))))
    fw = list(frame)
    fx = sum(w << (32 * i) for i, w in enumerate(fw[:nw]))
    fz = sum(w << (32 * i) for i, w in enumerate(fw[nw:]))
    a = np.frombuffer(amps, dtype=np.float64).copy()
    kk = k.value
    phi = (a[0::2] + 1j * a[1::2])[: 1 << kk]
    return fx, fz, phi, kk


def unpack_rows(words, shots: int) -> np.ndarray:
    """[rows, words] int64/uint64 -> [rows, shots] uint8 bits."""
    if hasattr(words, "cpu"):
        words = words.cpu().numpy()
    w = np.ascontiguousarray(np.asarray(words)).view(np.uint8)
    bits = np.unpackbits(w.reshape(w.shape[0], -1), axis=1, bitorder="little")
    return bits[:, :shots]
