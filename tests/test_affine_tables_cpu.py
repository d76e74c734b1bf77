"""CPU check of the compiler's record-level propagation tables (programs with
k_max = 0): for sampled shots, const ^ A m ^ F f built from the serialized
tables must equal the oracle's records. The faults f and the random
measurement bits m come from the oracle's own sampler and Philox, and the
expected records come from the oracle's Pauli-frame simulator.
No GPU is used."""

import struct

import numpy as np
import pytest

from gen import circuits as gc
from oracle.noise import sample_faults
from oracle.philox import meas_u
from oracle.records import raw_parities
from oracle.stabilizer import FrameSim

HEAD = "<17If18I"  # 17 counts, mean_faults, n_blocks, aff_ok, aff_rows, aff_n_rand, aff_n_chunks,
                   # aff_chunks_per_shot (read as u32), n_guide, aff_n_chains, aff_n_chain_rows, pad,
                   # n_fops, n_fterms, n_fperm, f_perm
HEAD_BYTES = struct.calcsize(HEAD)
OFF_NAMES = ["ops", "masks", "q", "seg_start", "seg_end", "site_info", "site_eff", "slot_list", "det_ref",
             "obs_ref", "site_opt", "opt_tab", "plist", "orec", "site_blk", "aff_const", "aff_rowev_off",
             "aff_rowev", "aff_rand_ev", "aff_col_off", "aff_col", "aff_frec", "aff_parent", "aff_chain_off",
             "aff_chain", "srch", "guide", "fops", "fterm", "fperm", "site_p",
             "total_bytes"]
REC_PER_SITE = 15


@pytest.fixture(scope="module")
def nc():
    from paper_2604_27058_gb300 import build
    build.build()
    import paper_2604_27058_gb300 as m
    return m


def _tables(blob: bytes):
    u = struct.unpack_from(HEAD, blob, 0)
    n_sites, n_meas, n_det, n_obs = u[5], u[6], u[7], u[8]
    aff_ok, rows, n_rand = u[19], u[20], u[21]
    offs = dict(zip(OFF_NAMES, struct.unpack_from(f"<{len(OFF_NAMES)}Q", blob, HEAD_BYTES)))
    assert aff_ok == 1
    assert rows == n_meas + n_det + n_obs

    def arr(name, n):
        return np.frombuffer(blob, dtype=np.uint32, count=n, offset=offs[name])

    col_off = arr("aff_col_off", n_sites * REC_PER_SITE + 1)
    n_chunks = int(col_off[-1])
    assert n_chunks == u[22]
    chunks = np.frombuffer(blob, dtype=np.uint16, count=8 * n_chunks, offset=offs["aff_col"]).reshape(-1, 8)
    frec = np.frombuffer(blob, dtype=np.uint32, count=4 * n_sites, offset=offs["aff_frec"]).reshape(-1, 4)
    # per-site records: 4-bit chunk counts, K, first chunk (or the long-site mark)
    for s in range(n_sites):
        nib = int(frec[s, 0]) | (int(frec[s, 1]) << 32)
        kk = nib >> 60
        counts = [int(col_off[s * REC_PER_SITE + o + 1] - col_off[s * REC_PER_SITE + o]) for o in range(kk)]
        if int(frec[s, 2]) == 0xFFFFFFFF:
            assert max(counts) > 15
            continue
        assert int(frec[s, 2]) == int(col_off[s * REC_PER_SITE])
        assert [(nib >> (4 * o)) & 15 for o in range(kk)] == counts
    n_chains = u[25]
    chain_off = arr("aff_chain_off", n_chains + 1)
    assert u[26] == int(chain_off[-1])
    chains = [arr("aff_chain", int(chain_off[-1]))[chain_off[i]:chain_off[i + 1]] for i in range(n_chains)]
    parent = arr("aff_parent", rows)
    for ch in chains:  # chains follow parent links, head first
        assert parent[ch[0]] == 0xFFFFFFFF
        assert all(parent[ch[j]] == ch[j - 1] for j in range(1, len(ch)))
    # every row on exactly one chain, longest chains first
    assert sorted(int(r) for ch in chains for r in ch) == list(range(rows))
    assert all(len(chains[i]) >= len(chains[i + 1]) for i in range(len(chains) - 1))
    return {
        "chains": chains,
        "rows": rows, "n_meas": n_meas, "n_det": n_det,
        "const": arr("aff_const", rows),
        "rowev_off": arr("aff_rowev_off", rows + 1),
        "rowev": arr("aff_rowev", int(arr("aff_rowev_off", rows + 1)[-1])),
        "rand_ev": arr("aff_rand_ev", n_rand),
        "col_off": col_off,
        "chunks": chunks,
    }


def _rows(t, faults, m):
    v = t["const"].astype(np.uint8).copy()
    for r in range(t["rows"]):
        for e in t["rowev"][t["rowev_off"][r]:t["rowev_off"][r + 1]]:
            v[r] ^= m[e]
    pos_row = np.concatenate(t["chains"])  # chunk entries are chain positions
    for site, opt in faults.items():
        c = site * REC_PER_SITE + opt
        for ch in t["chunks"][t["col_off"][c]:t["col_off"][c + 1]]:
            for j in ch:
                if j != t["rows"]:  # padding entries
                    v[pos_row[j]] ^= 1
    for ch in t["chains"]:  # delta rows to record rows
        acc = 0
        for r in ch:
            acc ^= int(v[r])
            v[r] = acc
    return v


CIRCUITS = {
    "surface_d3_r3": lambda: gc.surface_code_memory(d=3, rounds=3, p=0.02),
    "surface_d5_r25": lambda: gc.surface_code_memory(d=5, rounds=25, p=1e-3),
    "random_clifford_ff_reset": lambda: gc.random_small(41, n=6, n_ops=120, p_noise=0.05, t_frac=0.0),
    "random_clifford_ff_reset_b": lambda: gc.random_small(42, n=8, n_ops=200, p_noise=0.03, t_frac=0.0),
}


@pytest.mark.parametrize("name", sorted(CIRCUITS))
def test_affine_tables_reproduce_oracle_records(nc, name):
    text = CIRCUITS[name]()
    prog = nc.compile(text)
    assert prog.info.k_max == 0
    t = _tables(prog.serialize())
    sim = FrameSim(text)
    flat = sim.flat
    seed = 777
    n_faulty = 0
    for shot in range(40):
        faults = sample_faults(sim.table, seed, shot)
        n_faulty += bool(faults)
        m = np.array([1 if meas_u(seed, shot, int(ev)) < 0.5 else 0 for ev in t["rand_ev"]], dtype=np.uint8)
        got = _rows(t, faults, m)
        meas, _ = sim.run_raw(seed, shot, faults=faults)
        det, obs = raw_parities(flat, meas)
        want = np.array(list(meas) + list(det) + list(obs), dtype=np.uint8)
        assert np.array_equal(got, want), f"shot {shot}"
    assert n_faulty > 0


def test_affine_tables_absent_with_active_axes(nc):
    prog = nc.compile(gc.tiny_random(seed=1))
    assert prog.info.k_max > 0
    blob = prog.serialize()
    assert struct.unpack_from(HEAD, blob, 0)[19] == 0


def _guide_key(t: int, shift: int) -> int:
    t = max(t, 1 << 16)
    e = t.bit_length() - 1
    lv = (e << 16) | ((t >> (e - 16)) & 0xFFFF)
    return (((63 << 16) | 0xFFFF) - lv) >> shift


@pytest.mark.parametrize("name", ["surface", "sweep_many_segments", "certain_fault"])
def test_guide_search_matches_bisection(nc, name):
    """The compiled survival search records and guide tables give, for any
    threshold t, the same first site with Q[i] <= t as plain bisection of
    the oracle's survival table."""
    from oracle.noise import _first_at_or_below, build_table
    from oracle.circuit import flatten
    text = {"surface": lambda: gc.surface_code_memory(d=5, rounds=25, p=1e-3),
            "sweep_many_segments": lambda: gc.sweep_mirror(1).text,
            "certain_fault": lambda: "X_ERROR(1) 0\nX_ERROR(0.5) 0 1\nDEPOLARIZE1(0.999999) 1\nM 0 1\n"}[name]()
    blob = nc.compile(text).serialize()
    u = struct.unpack_from(HEAD, blob, 0)
    n_sites, n_guide = u[5], u[24]
    offs = dict(zip(OFF_NAMES, struct.unpack_from(f"<{len(OFF_NAMES)}Q", blob, HEAD_BYTES)))
    srch = np.frombuffer(blob, dtype=np.uint32, count=8 * n_sites, offset=offs["srch"]).reshape(-1, 8)
    guide = np.frombuffer(blob, dtype=np.uint32, count=n_guide, offset=offs["guide"])
    f = flatten(text)
    table = build_table(f.site_p, f.site_kind)
    q = table.q
    rng = np.random.default_rng(5)
    sts = sorted(set(rng.integers(0, n_sites, 300).tolist()) | {0, n_sites - 1})
    checked = 0
    for st in sts:
        a, b, gbase, shift = (int(x) for x in srch[st][:4])
        q_end = int(srch[st][4]) | (int(srch[st][5]) << 32)
        q_l = int(srch[st][6]) | (int(srch[st][7]) << 32)
        assert (a, b) == (table.seg_start[st], table.seg_end[st])
        assert q_end == q[b - 1]
        assert q_l == ((1 << 64) - 1 if st == a else q[st - 1])
        ts = [(int(x) * q_l) >> 64 for x in rng.integers(0, 2**63, 40, dtype=np.int64) * 2]
        ts += [q_end, max(q_l - 1, 0)]
        for t in ts:
            if q_end > t:
                continue
            i = int(guide[gbase + _guide_key(t, shift)])
            assert i <= _first_at_or_below(q, st, b, t)
            while q[i] > t:
                i += 1
            assert i == _first_at_or_below(q, st, b, t)
            checked += 1
    assert checked >= min(100, 10 * n_sites)
