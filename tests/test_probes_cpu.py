"""Compiled expectation probes against the oracle's plan (CPU, no GPU): every
OP_EXPVAL instruction carries the Heisenberg image M(P) (x / z masks and the
i^ph phase), the active-position masks and the dormant-x flag that the
factored oracle derives for the same probe."""

import struct

import pytest

from gen import circuits as gc
from oracle.factored import FactoredSim

HEAD = "<17If18I"
HEAD_BYTES = struct.calcsize(HEAD)
OFF_NAMES = ["ops", "masks", "q", "seg_start", "seg_end", "site_info", "site_eff", "slot_list", "det_ref",
             "obs_ref", "site_opt", "opt_tab", "plist", "orec", "site_blk", "aff_const", "aff_rowev_off",
             "aff_rowev", "aff_rand_ev", "aff_col_off", "aff_col", "aff_frec", "aff_parent", "aff_chain_off",
             "aff_chain", "srch", "guide", "fops", "fterm", "fperm", "site_p", "total_bytes"]
OP_EXPVAL = 27


@pytest.fixture(scope="module")
def nc():
    from paper_2604_27058_gb300 import build
    build.build()
    import paper_2604_27058_gb300 as m
    return m


def _compiled_probes(prog):
    blob = prog.serialize()
    u = struct.unpack_from(HEAD, blob, 0)
    n_qubits, nw, n_ops = u[2], u[3], u[4]
    offs = dict(zip(OFF_NAMES, struct.unpack_from(f"<{len(OFF_NAMES)}Q", blob, HEAD_BYTES)))
    out = {}
    for i in range(n_ops):
        b = blob[offs["ops"] + 32 * i: offs["ops"] + 32 * (i + 1)]
        code, flags, a, bq, pa, pb = struct.unpack_from("<BBHHBB", b, 0)
        if code != OP_EXPVAL:
            continue
        i0, i1, i2, i3 = struct.unpack_from("<4I", b, 8)
        words = struct.unpack_from(f"<{2 * nw}I", blob, offs["masks"] + 4 * i0)
        x = sum(w << (32 * j) for j, w in enumerate(words[:nw]))
        z = sum(w << (32 * j) for j, w in enumerate(words[nw:]))
        out[i3] = dict(x=x, z=z, ph=pa, mx=i1, mz=i2, zero=bool(pb))
    return out


@pytest.mark.parametrize("seed", range(8))
def test_compiled_probes_match_the_oracle_plan(nc, seed):
    text = gc.with_probes(gc.random_small(800 + seed, n=6, n_ops=90, p_noise=0.05, t_frac=0.3), seed, count=10)
    prog = nc.compile(text, peephole=False)  # the plain method's plan, as the oracle's
    assert prog.info.n_probes == 10
    got = _compiled_probes(prog)
    sim = FactoredSim(text)
    want = {st.a["index"]: st.a for st in sim.steps if st.kind == "probe"}
    assert sorted(got) == sorted(want) == list(range(10))
    for j in range(10):
        w, g = want[j], got[j]
        assert g["zero"] == w["zero"], j
        assert (g["x"], g["z"], g["ph"]) == (w["x"], w["z"], w["ph"] % 4), j
        if not w["zero"]:
            assert (g["mx"], g["mz"]) == (w["mx"], w["mz"]), j


def test_probe_programs_use_the_executor_and_fused_gathers(nc):
    # k_max = 0 with probes: no record-level tables (the executors run probes)
    prog = nc.compile("H 0\nCX 0 1\nEXPVAL X0*X1 Z0\nM 0 1\n")
    blob = prog.serialize()
    u = struct.unpack_from(HEAD, blob, 0)
    assert u[19] == 0  # aff_ok
    assert prog.info.n_probes == 2


def test_parse_errors(nc):
    for bad in ("EXPVAL X0*X0", "EXPVAL Q1", "EXPVAL(1) X0", "EXPVAL", "EXPVAL X"):
        with pytest.raises(nc.NcError):
            nc.compile(bad)
