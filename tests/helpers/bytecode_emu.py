"""A slow Python interpreter of the compiled program's plain instruction list
(test infrastructure). It reads the serialized blob, runs one shot at a time
with the draw contract of ``oracle.philox`` and the fault sets of
``oracle.noise``, and returns the shot's records and probe values. It lets
the CPU tests check the compiler's output (instructions, masks, noise
tables, slot allocation, probes, the HIR peephole) against the oracle end to
end without a GPU. It shares no code with the library."""

from __future__ import annotations

import struct

import numpy as np

from oracle.noise import build_table, sample_faults
from oracle.philox import meas_top_bit, meas_u

HEAD = "<17If18I"
OFF_NAMES = ["ops", "masks", "q", "seg_start", "seg_end", "site_info", "site_eff", "slot_list", "det_ref",
             "obs_ref", "site_opt", "opt_tab", "plist", "orec", "site_blk", "aff_const", "aff_rowev_off",
             "aff_rowev", "aff_rand_ev", "aff_col_off", "aff_col", "aff_frec", "aff_parent", "aff_chain_off",
             "aff_chain", "srch", "guide", "fops", "fterm", "fperm", "site_p", "total_bytes"]
CODES = ["END", "FRAME_H", "FRAME_S", "FRAME_CX", "FRAME_CZ", "ARRAY_H", "ARRAY_S", "ARRAY_CX", "ARRAY_CZ",
         "EXPAND_ROT", "ROT_Z", "ROT_X", "MEAS_STATIC", "MEAS_RANDOM", "MEAS_ACTIVE_Z", "MEAS_ACTIVE_X",
         "NOISE_BLOCK", "FEEDFORWARD", "REC_OUT", "DETECTOR", "OBS_INCLUDE", "OBS_OUT", "KEPT_OUT", "BATCH",
         "DIAGF", "MIXF", "PERMF", "EXPVAL"]
F_SIGN, F_OUT, F_RESET = 1, 2, 4
SITE_FLIP = 5
RS = 1 / np.sqrt(2)


def _u32(blob, off, n):
    return list(struct.unpack_from(f"<{n}I", blob, off)) if n else []


class Program:
    def __init__(self, blob: bytes, site_p, site_kind):
        u = struct.unpack_from(HEAD, blob, 0)
        (self.n_qubits, self.nw, self.n_ops, self.n_sites, self.n_meas, self.n_det, self.n_obs,
         self.n_events, self.n_slots, self.k_max, self.kept_slot) = u[2:13]
        self.n_probes = u[27]
        offs = dict(zip(OFF_NAMES, struct.unpack_from(f"<{len(OFF_NAMES)}Q", blob, struct.calcsize(HEAD))))
        self.ops = []
        for i in range(self.n_ops):
            b = blob[offs["ops"] + 32 * i: offs["ops"] + 32 * (i + 1)]
            code, flags, a, bq, pa, pb = struct.unpack_from("<BBHHBB", b, 0)
            i0, i1, i2, i3 = struct.unpack_from("<4I", b, 8)
            cs, sn = struct.unpack_from("<2d", b, 8)
            self.ops.append(dict(code=CODES[code], flags=flags, a=a, b=bq, pa=pa, pb=pb, i0=i0, i1=i1, i2=i2,
                                 i3=i3, cs=cs, sn=sn))
        n_mask = u[13]
        self.masks = _u32(blob, offs["masks"], n_mask)
        self.site_info = _u32(blob, offs["site_info"], self.n_sites)
        self.site_eff = _u32(blob, offs["site_eff"], self.n_sites)
        self.slot_list = _u32(blob, offs["slot_list"], u[14])
        self.opt_tab = _u32(blob, offs["opt_tab"], 2 * u[15])
        # the survival table and draw contract come from the oracle (same
        # site list: the blob's site probabilities equal the oracle's)
        self.table = build_table(site_p, site_kind)
        self.ref_det = [0] * self.n_det
        self.ref_obs = [0] * self.n_obs
        ref = self.run(0, 0, noisy=False, argmax=True, raw=True)
        self.ref_det, self.ref_obs = ref["det"], ref["obs"]

    def _mask(self, off):
        return sum(w << (32 * j) for j, w in enumerate(self.masks[off: off + self.nw]))

    def run(self, seed, shot, noisy=True, argmax=False, postselect=False, raw=False, faults=None):
        N = self.n_qubits
        x = z = 0
        slots = [0] * (self.n_slots + 1)
        slots[self.kept_slot] = 1
        meas = [0] * self.n_meas
        det = [0] * self.n_det
        obs = [0] * self.n_obs
        probes = [0.0] * self.n_probes
        phi = np.ones(1, dtype=complex)
        k = 0
        if faults is None:
            faults = sample_faults(self.table, seed, shot) if (noisy and self.n_sites) else {}
        fault_sites = sorted(faults)
        nf = 0

        def bit(v, q):
            return (v >> q) & 1

        def par(v):
            return bin(v).count("1") & 1

        def insert0(j, p):
            return ((j >> p) << (p + 1)) | (j & ((1 << p) - 1))

        for op in self.ops:
            c = op["code"]
            kept = slots[self.kept_slot]
            if c in ("FRAME_H", "ARRAY_H"):
                xa, za = bit(x, op["a"]), bit(z, op["a"])
                x = (x & ~(1 << op["a"])) | (za << op["a"])
                z = (z & ~(1 << op["a"])) | (xa << op["a"])
                if c == "ARRAY_H":
                    idx = np.arange(1 << k)
                    i0 = idx[((idx >> op["pa"]) & 1) == 0]
                    i1 = i0 | (1 << op["pa"])
                    a, b = phi[i0].copy(), phi[i1].copy()
                    phi[i0], phi[i1] = (a + b) * RS, (a - b) * RS
            elif c in ("FRAME_S", "ARRAY_S"):
                z ^= bit(x, op["a"]) << op["a"]
                if c == "ARRAY_S":
                    idx = np.arange(1 << k)
                    i1 = idx[((idx >> op["pa"]) & 1) == 1]
                    phi[i1] *= 1j
            elif c in ("FRAME_CX", "ARRAY_CX"):
                x ^= bit(x, op["a"]) << op["b"]
                z ^= bit(z, op["b"]) << op["a"]
                if c == "ARRAY_CX":
                    idx = np.arange(1 << k)
                    phi = phi[idx ^ (((idx >> op["pa"]) & 1) << op["pb"])]
            elif c in ("FRAME_CZ", "ARRAY_CZ"):
                xa, xb = bit(x, op["a"]), bit(x, op["b"])
                z ^= (xb << op["a"]) ^ (xa << op["b"])
                if c == "ARRAY_CZ":
                    idx = np.arange(1 << k)
                    both = ((idx >> op["pa"]) & 1) & ((idx >> op["pb"]) & 1)
                    phi = np.where(both == 1, -phi, phi)
            elif c == "EXPAND_ROT":
                sn = -op["sn"] if bit(x, op["a"]) else op["sn"]
                phi = np.concatenate([phi * RS, phi * RS * (op["cs"] + 1j * sn)])
                k += 1
            elif c == "ROT_Z":
                sn = -op["sn"] if bit(x, op["a"]) else op["sn"]
                idx = np.arange(1 << k)
                phi = np.where(((idx >> op["pa"]) & 1) == 1, phi * (op["cs"] + 1j * sn), phi)
            elif c == "ROT_X":
                sn = -op["sn"] if bit(z, op["a"]) else op["sn"]
                cr = op["cs"]
                idx = np.arange(1 << k)
                i0 = idx[((idx >> op["pa"]) & 1) == 0]
                i1 = i0 | (1 << op["pa"])
                a, b = phi[i0].copy(), phi[i1].copy()
                phi[i0] = cr * a - 1j * sn * b
                phi[i1] = -1j * sn * a + cr * b
            elif c == "MEAS_STATIC":
                m = (1 if op["flags"] & F_SIGN else 0) ^ par(x & self._mask(op["i0"]))
                if op["flags"] & F_RESET:
                    for r in range(op["pb"]):
                        pl = ((op["i2"] if r < 2 else op["i3"]) >> (16 * (r & 1))) & 0xFFFF
                        if m:
                            if pl < N:
                                x ^= 1 << pl
                            else:
                                z ^= 1 << (pl - N)
                else:
                    slots[op["i2"]] = m
                    if op["flags"] & F_OUT:
                        meas[op["i3"]] = m & kept
            elif c == "MEAS_RANDOM":
                m = 0 if argmax else 1 - meas_top_bit(seed, shot, op["i0"])
                b = m ^ (1 if op["flags"] & F_SIGN else 0) ^ bit(z, op["a"])
                xa = bit(x, op["a"])
                x = (x & ~(1 << op["a"])) | ((bit(z, op["a"]) ^ b) << op["a"])
                z = (z & ~(1 << op["a"])) | (xa << op["a"])
                slots[op["i2"]] = m
                if op["flags"] & F_OUT:
                    meas[op["i3"]] = m & kept
            elif c in ("MEAS_ACTIVE_Z", "MEAS_ACTIVE_X"):
                xm = c == "MEAS_ACTIVE_X"
                pa = op["pa"]
                idx = np.arange(1 << k)
                lo = idx[((idx >> pa) & 1) == 0]
                hi = lo | (1 << pa)
                if xm:
                    b0, b1 = (phi[lo] + phi[hi]) * RS, (phi[lo] - phi[hi]) * RS
                else:
                    b0, b1 = phi[lo], phi[hi]
                s0, s1 = float(np.sum(np.abs(b0) ** 2)), float(np.sum(np.abs(b1) ** 2))
                pbit = bit(z, op["a"]) if xm else bit(x, op["a"])
                abit = 1 if op["flags"] & F_SIGN else 0
                tot = s0 + s1
                p1 = ((s1 if (1 ^ abit ^ pbit) else s0) / tot) if tot > 0 else 0.0
                if argmax:
                    m = 1 if p1 > 0.5 else 0
                elif p1 <= 0.0:
                    m = 0
                elif p1 >= 1.0:
                    m = 1
                elif p1 == 0.5:
                    m = 1 - meas_top_bit(seed, shot, op["i0"])
                else:
                    m = 1 if meas_u(seed, shot, op["i0"]) < p1 else 0
                b = m ^ abit ^ pbit
                keep = (b1 if b else b0) / np.sqrt(s1 if b else s0)
                # the kept half holds the other axes in order with pa removed;
                # the top axis then moves into position pa (demotion)
                top = k - 1
                if pa != top:
                    kk = np.arange(1 << (k - 1))
                    # index of the kept half: bits of positions != pa, in order
                    src = np.empty(1 << (k - 1), dtype=np.int64)
                    for j in kk:
                        full = insert0(int(j), pa)
                        # new index: old top bit goes to position pa
                        topbit = (full >> top) & 1
                        rest = full & ~(1 << top)
                        new = rest | (topbit << pa)
                        src[new] = j
                    keep = keep[src]
                phi = keep
                k -= 1
                slots[op["i2"]] = m
                if op["flags"] & F_OUT:
                    meas[op["i3"]] = m & kept
                if xm:
                    xa = bit(x, op["a"])
                    x = (x & ~(1 << op["a"])) | ((bit(z, op["a"]) ^ b) << op["a"])
                    z = (z & ~(1 << op["a"])) | (xa << op["a"])
                else:
                    x ^= b << op["a"]
            elif c == "NOISE_BLOCK":
                while nf < len(fault_sites) and fault_sites[nf] < op["i1"]:
                    site = fault_sites[nf]
                    opt = faults[site]
                    info, eff = self.site_info[site], self.site_eff[site]
                    if (info & 15) == SITE_FLIP:
                        slots[eff] ^= 1
                        if slots[self.kept_slot]:
                            meas[self.opt_tab[2 * (info >> 8) + 1]] ^= 1
                    else:
                        off = eff + opt * 2 * self.nw
                        x ^= self._mask(off)
                        z ^= self._mask(off + self.nw)
                    nf += 1
            elif c == "FEEDFORWARD":
                if slots[op["i2"]]:
                    x ^= self._mask(op["i0"])
                    z ^= self._mask(op["i0"] + self.nw)
            elif c == "REC_OUT":
                meas[op["i3"]] = slots[op["i2"]] & kept
            elif c == "DETECTOR":
                d = 0
                for j in range(op["i1"]):
                    d ^= slots[self.slot_list[op["i0"] + j]]
                if not raw:
                    d ^= self.ref_det[op["i3"]]
                det[op["i3"]] = d & kept
                if postselect and d:
                    slots[self.kept_slot] = 0
            elif c == "OBS_INCLUDE":
                d = 0
                for j in range(op["i1"]):
                    d ^= slots[self.slot_list[op["i0"] + j]]
                slots[op["i2"]] ^= d
            elif c == "OBS_OUT":
                v = slots[op["i2"]] ^ (0 if raw else self.ref_obs[op["i3"]])
                obs[op["i3"]] = v & kept
            elif c == "EXPVAL":
                v = 0.0
                if not op["pb"] and kept:
                    odd = op["pa"] & 1
                    idx = np.arange(1 << k)
                    sg = np.where(np.array([bin(int(j) & op["i2"]).count("1") & 1 for j in idx]) == 1, -1.0, 1.0)
                    acc = np.sum(np.conj(phi[idx ^ op["i1"]]) * phi * sg)
                    part = (acc.imag if odd else acc.real) / float(np.sum(np.abs(phi) ** 2))
                    om = par(x & self._mask(op["i0"] + self.nw)) ^ par(z & self._mask(op["i0"]))
                    sgn = -1.0 if op["pa"] in (1, 2) else 1.0
                    v = -sgn * part if om else sgn * part
                probes[op["i3"]] = v
        return dict(meas=meas, det=det, obs=obs, kept=slots[self.kept_slot], probes=probes)
