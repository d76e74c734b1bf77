"""Host side of stratified importance sampling (no GPU): the program blob
carries the oracle's site probabilities bit for bit, the library's stratum
weights and validity flags equal the oracle's, and the library refuses what
the contract refuses."""

import struct

import pytest

from gen import circuits as gc
from oracle.circuit import flatten
from oracle.strata import build_strata, stratum_valid, stratum_weights

HEAD = "<17If18I"
HEAD_BYTES = struct.calcsize(HEAD)
OFF_NAMES = ["ops", "masks", "q", "seg_start", "seg_end", "site_info", "site_eff", "slot_list", "det_ref",
             "obs_ref", "site_opt", "opt_tab", "plist", "orec", "site_blk", "aff_const", "aff_rowev_off",
             "aff_rowev", "aff_rand_ev", "aff_col_off", "aff_col", "aff_frec", "aff_parent", "aff_chain_off",
             "aff_chain", "srch", "guide", "fops", "fterm", "fperm", "site_p", "total_bytes"]

CIRCUITS = {
    "surface_d3": gc.surface_code_memory(d=3, rounds=3, p=0.01),
    "surface_d5": gc.surface_code_memory(d=5, rounds=25, p=1e-3),
    "tiny": gc.tiny_random(seed=1),
    "lowmagic": gc.low_magic_gadgets(),
    "mixed_p": "\n".join(["H 0 1 2", "DEPOLARIZE1(0.013) 0 1", "CX 0 1", "DEPOLARIZE2(0.002) 0 1",
                          "X_ERROR(0) 2", "Z_ERROR(0.3) 2", "M(0.07) 0 1 2"]),
}


@pytest.fixture(scope="module")
def nc():
    from paper_2604_27058_gb300 import build
    build.build()
    import paper_2604_27058_gb300 as m
    return m


def _blob_site_p(prog):
    blob = prog.serialize()
    u = struct.unpack_from(HEAD, blob, 0)
    n_sites = u[5]
    offs = dict(zip(OFF_NAMES, struct.unpack_from(f"<{len(OFF_NAMES)}Q", blob, HEAD_BYTES)))
    return list(struct.unpack_from(f"<{n_sites}d", blob, offs["site_p"])) if n_sites else []


@pytest.mark.parametrize("name", sorted(CIRCUITS))
def test_blob_site_probabilities_are_the_oracles(nc, name):
    text = CIRCUITS[name]
    prog = nc.compile(text)
    assert prog.info.n_noise_sites == len(flatten(text).site_p)
    assert _blob_site_p(prog) == flatten(text).site_p


@pytest.mark.parametrize("name", sorted(CIRCUITS))
def test_weights_and_validity_match_the_oracle(nc, name):
    text = CIRCUITS[name]
    prog = nc.compile(text)
    fl = flatten(text)
    k_max = 20
    w, ok = nc.stratum_weights(prog, k_max)
    assert w == stratum_weights(fl.site_p, k_max)  # same FP64 operations: equal bit for bit
    t = build_strata(fl.site_p, fl.site_kind, k_max)
    assert ok == [stratum_valid(t, k) for k in range(k_max + 1)]


def test_refusals(nc):
    prog = nc.compile(CIRCUITS["mixed_p"])  # 2 + 1 + 1 + 1 + 3 = 8 sites; X_ERROR(0) is not live
    w, ok = nc.stratum_weights(prog, 8)
    assert ok == [True] * 8 + [False]
    with pytest.raises(nc.NcError):
        nc.stratum_weights(prog, 128)  # above the per-shot list limit
    certain = nc.compile("X_ERROR(1) 0\nM 0")
    _, ok = nc.stratum_weights(certain, 1)
    assert ok == [False, False]
