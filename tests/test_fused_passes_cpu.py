"""CPU check of the compiler's fused array-pass list (the batched executor's
second instruction list). For noiseless circuits whose frame stays zero up to
the first active measurement, the active vector built by the original array
instructions (logical order) must equal the one built by the fused list
(index map, deferred phases, pair passes, final gather), just before that
measurement. Both are emulated here with numpy from the serialized program;
no GPU is used."""

import struct

import numpy as np
import pytest

from gen import circuits as gc

HEAD = "<17If18I"
HEAD_BYTES = struct.calcsize(HEAD)
OFF_NAMES = ["ops", "masks", "q", "seg_start", "seg_end", "site_info", "site_eff", "slot_list", "det_ref",
             "obs_ref", "site_opt", "opt_tab", "plist", "orec", "site_blk", "aff_const", "aff_rowev_off",
             "aff_rowev", "aff_rand_ev", "aff_col_off", "aff_col", "aff_frec", "aff_parent", "aff_chain_off",
             "aff_chain", "srch", "guide", "fops", "fterm", "fperm", "site_p",
             "total_bytes"]
CODES = ["END", "FRAME_H", "FRAME_S", "FRAME_CX", "FRAME_CZ", "ARRAY_H", "ARRAY_S", "ARRAY_CX", "ARRAY_CZ",
         "EXPAND_ROT", "ROT_Z", "ROT_X", "MEAS_STATIC", "MEAS_RANDOM", "MEAS_ACTIVE_Z", "MEAS_ACTIVE_X",
         "NOISE_BLOCK", "FEEDFORWARD", "REC_OUT", "DETECTOR", "OBS_INCLUDE", "OBS_OUT", "KEPT_OUT", "BATCH",
         "DIAGF", "MIXF", "PERMF", "EXPVAL"]
RS = 1 / np.sqrt(2)


@pytest.fixture(scope="module")
def nc():
    from paper_2604_27058_gb300 import build
    build.build()
    import paper_2604_27058_gb300 as m
    return m


def _ops(blob, off, n):
    out = []
    for i in range(n):
        b = blob[off + 32 * i: off + 32 * (i + 1)]
        code, flags, a, bq, pa, pb = struct.unpack_from("<BBHHBB", b, 0)
        i0, i1, i2, i3 = struct.unpack_from("<4I", b, 8)
        cs, sn = struct.unpack_from("<2d", b, 8)
        out.append(dict(code=CODES[code], flags=flags, a=a, b=bq, pa=pa, pb=pb, i0=i0, i1=i1, i2=i2, i3=i3, cs=cs,
                        sn=sn))
    return out


def _par(x):
    return bin(x).count("1") & 1


def _phase(p, terms):
    ph = 1.0 + 0j
    for kind, r1, r2, cs, sn in terms:
        k, c1, c2 = kind & 255, (kind >> 8) & 1, (kind >> 9) & 1
        b1 = _par(p & r1) ^ c1
        if k == 1 and b1 and (_par(p & r2) ^ c2):
            ph = -ph
        elif k == 2 and b1:
            ph *= 1j
        elif k == 3 and b1:
            ph *= cs + 1j * sn  # frame planes stay zero here
    return ph


def _run_original(ops, probes=None):
    v = np.ones(1, dtype=complex)
    for o in ops:
        c = o["code"]
        if c == "EXPVAL" and probes is not None:
            probes.append(v.copy())
        k = int(np.log2(len(v)))
        idx = np.arange(len(v))
        if c == "EXPAND_ROT":
            v = np.concatenate([v * RS, v * RS * (o["cs"] + 1j * o["sn"])])
        elif c == "ROT_Z":
            v = np.where((idx >> o["pa"]) & 1, v * (o["cs"] + 1j * o["sn"]), v)
        elif c == "ARRAY_S":
            v = np.where((idx >> o["pa"]) & 1, v * 1j, v)
        elif c == "ARRAY_CZ":
            v = np.where(((idx >> o["pa"]) & 1) & ((idx >> o["pb"]) & 1), -v, v)
        elif c == "ARRAY_CX":
            v = v[idx ^ (((idx >> o["pa"]) & 1) << o["pb"])]
        elif c in ("ARRAY_H", "ROT_X"):
            i0 = idx[((idx >> o["pa"]) & 1) == 0]
            i1 = i0 | (1 << o["pa"])
            a, b = v[i0].copy(), v[i1].copy()
            if c == "ARRAY_H":
                v[i0], v[i1] = (a + b) * RS, (a - b) * RS
            else:
                cr, sr = o["cs"], o["sn"]
                v[i0] = cr * a - 1j * sr * b
                v[i1] = -1j * sr * a + cr * b
        elif c.startswith("MEAS_ACTIVE"):
            return v, k
    raise AssertionError("no active measurement")


def _run_fused(ops, terms, perm, probes=None):
    w = np.ones(1, dtype=complex)
    for o in ops:
        c = o["code"]
        if c == "EXPVAL" and probes is not None:
            probes.append(w.copy())
        k = int(np.log2(len(w)))
        if c == "EXPAND_ROT":
            w = np.concatenate([w * RS, w * RS * (o["cs"] + 1j * o["sn"])])
        elif c == "DIAGF":
            t = terms[o["i2"]: o["i2"] + o["i3"]]
            w = np.array([w[p] * _phase(p, t) for p in range(len(w))])
        elif c == "MIXF":
            lead = terms[o["i2"]]
            t = terms[o["i2"] + 1: o["i2"] + 1 + o["i3"]]
            m, r, rc, piv = o["i0"], o["i1"] & 0x7FFFFFFF, o["i1"] >> 31, o["pa"]
            assert (m >> piv) & 1
            for p in range(len(w)):
                if (p >> piv) & 1:
                    continue
                q = p ^ m
                p0, p1 = (p, q) if (_par(p & r) ^ rc) == 0 else (q, p)
                a, b = w[p0] * _phase(p0, t), w[p1] * _phase(p1, t)
                if o["pb"] == 0:
                    w[p0], w[p1] = (a + b) * RS, (a - b) * RS
                else:
                    cr, sr = lead[3], lead[4]
                    w[p0] = cr * a - 1j * sr * b
                    w[p1] = -1j * sr * a + cr * b
        elif c == "PERMF":
            kk = o["i1"]
            cols = perm[o["i0"]: o["i0"] + kk]
            cc = perm[o["i0"] + kk]
            t = terms[o["i2"]: o["i2"] + o["i3"]]
            nw = np.zeros_like(w)
            for i in range(len(w)):
                p = cc
                for b in range(kk):
                    if (i >> b) & 1:
                        p ^= cols[b]
                assert p < len(w)
                nw[i] = w[p] * _phase(p, t)
            w = nw
        elif c.startswith("MEAS_ACTIVE"):
            return w, k
    raise AssertionError("no active measurement")


@pytest.mark.parametrize("seed,n,layers", [(3, 8, 10), (4, 9, 12), (5, 10, 8)])
def test_fused_list_builds_the_same_vector(nc, seed, n, layers):
    blob = nc.compile(gc.dense_random(seed=seed, n=n, layers=layers), peephole=False).serialize()
    u = struct.unpack_from(HEAD, blob, 0)
    n_ops = u[4]
    n_fops, n_fterms, n_fperm = u[32], u[33], u[34]
    offs = dict(zip(OFF_NAMES, struct.unpack_from(f"<{len(OFF_NAMES)}Q", blob, HEAD_BYTES)))
    assert n_fops > 0
    ops = _ops(blob, offs["ops"], n_ops)
    fops = _ops(blob, offs["fops"], n_fops)
    terms = [struct.unpack_from("<4I2d", blob, offs["fterm"] + 32 * i) for i in range(n_fterms)]
    terms = [(t[0], t[2], t[3], t[4], t[5]) for t in terms]
    perm = list(struct.unpack_from(f"<{n_fperm}I", blob, offs["fperm"])) if n_fperm else []
    # fewer passes over the vector
    passes = sum(o["code"] in ("ARRAY_H", "ARRAY_S", "ARRAY_CX", "ARRAY_CZ", "ROT_Z", "ROT_X", "EXPAND_ROT")
                 for o in ops)
    fpasses = sum(o["code"] in ("DIAGF", "MIXF", "PERMF", "EXPAND_ROT") for o in fops)
    assert fpasses < passes
    v, k = _run_original(ops)
    w, kf = _run_fused(fops, terms, perm)
    assert k == kf
    assert np.allclose(v, w, atol=1e-12)


def test_dense_workload_passes_shrink(nc):
    """The k = 20 dense workload: its 3239 array instructions become at most
    a fifth as many passes."""
    blob = nc.compile(gc.dense_random(seed=3, n=20, layers=40)).serialize()
    u = struct.unpack_from(HEAD, blob, 0)
    offs = dict(zip(OFF_NAMES, struct.unpack_from(f"<{len(OFF_NAMES)}Q", blob, HEAD_BYTES)))
    ops = _ops(blob, offs["ops"], u[4])
    fops = _ops(blob, offs["fops"], u[32])
    passes = sum(o["code"] in ("ARRAY_H", "ARRAY_S", "ARRAY_CX", "ARRAY_CZ", "ROT_Z", "ROT_X", "EXPAND_ROT")
                 for o in ops)
    fpasses = sum(o["code"] in ("DIAGF", "MIXF", "PERMF", "EXPAND_ROT") for o in fops)
    assert fpasses * 5 <= passes, (fpasses, passes)


@pytest.mark.parametrize("seed", [1, 2])
def test_fused_list_in_logical_order_at_every_probe(nc, seed):
    """Probes (OP_EXPVAL) read the vector in logical order: at every probe the
    fused list's vector equals the original list's."""
    text = gc.with_probes(gc.dense_random(seed=seed, n=9, layers=10), seed, count=6, max_weight=3)
    # keep the probes before the final measurements
    lines = text.splitlines()
    body = [ln for ln in lines if not ln.startswith("M ")] + [ln for ln in lines if ln.startswith("M ")]
    blob = nc.compile("\n".join(body)).serialize()
    u = struct.unpack_from(HEAD, blob, 0)
    offs = dict(zip(OFF_NAMES, struct.unpack_from(f"<{len(OFF_NAMES)}Q", blob, HEAD_BYTES)))
    n_fops, n_fterms, n_fperm = u[32], u[33], u[34]
    assert n_fops > 0
    ops = _ops(blob, offs["ops"], u[4])
    fops = _ops(blob, offs["fops"], n_fops)
    terms = [struct.unpack_from("<4I2d", blob, offs["fterm"] + 32 * i) for i in range(n_fterms)]
    terms = [(t[0], t[2], t[3], t[4], t[5]) for t in terms]
    perm = list(struct.unpack_from(f"<{n_fperm}I", blob, offs["fperm"])) if n_fperm else []
    pa, pb = [], []
    _run_original(ops, pa)
    _run_fused(fops, terms, perm, pb)
    assert len(pa) == len(pb) == 6
    for a, b in zip(pa, pb):
        assert np.allclose(a, b, atol=1e-12)


@pytest.mark.parametrize("name", ["dense20", "dense10", "coherent"])
def test_gathers_that_form_measurement_sums(nc, name):
    """A gather flagged to form the next measurement's sums (FLAG_SUMS = 16)
    is followed directly by that active measurement, flagged as presummed
    (FLAG_PRESUMMED = 32), whose measured position and basis it names; every
    presummed measurement has such a gather; probes never do."""
    text = {"dense20": gc.dense_random(seed=3, n=20, layers=40), "dense10": gc.dense_random(seed=33, n=10, layers=12),
            "coherent": gc.surface_code_memory(d=3, rounds=3, p=1e-3, theta=0.02)}[name]
    blob = nc.compile(text).serialize()
    u = struct.unpack_from(HEAD, blob, 0)
    offs = dict(zip(OFF_NAMES, struct.unpack_from(f"<{len(OFF_NAMES)}Q", blob, HEAD_BYTES)))
    fops = _ops(blob, offs["fops"], u[32])
    n_sums = 0
    for i, o in enumerate(fops):
        if o["code"] == "PERMF" and o["flags"] & 16:
            n_sums += 1
            m = fops[i + 1]
            assert m["code"] in ("MEAS_ACTIVE_Z", "MEAS_ACTIVE_X") and m["flags"] & 32
            assert o["pa"] == m["pa"] and o["pb"] == (m["code"] == "MEAS_ACTIVE_X")
            assert m["pa"] < o["i1"]  # the measured position lies inside the gathered vector
        if o["flags"] & 32 and o["code"].startswith("MEAS_ACTIVE"):
            assert fops[i - 1]["code"] == "PERMF" and fops[i - 1]["flags"] & 16
        if o["code"] == "EXPVAL":
            assert not o["flags"] & 32
    assert n_sums >= (16 if name == "dense20" else 1)
