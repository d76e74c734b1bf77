"""The compiled program, run by a plain Python interpreter of its instruction
list (tests/helpers/bytecode_emu.py), against the factored oracle, shot by
shot (CPU, no GPU). This checks the compiler's instructions, masks, noise
tables, record slots, probes and HIR peephole end to end. The oracle is the
plain method (no HIR pass), so the programs compiled with the peephole on
check that the rule changes no record. Records must be equal except flagged
near-ties; probes within 1e-10."""

import os
import sys

import pytest

from gen import circuits as gc
from oracle.circuit import flatten
from oracle.factored import FactoredSim
from oracle.records import assemble, probe_alive

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "helpers"))
from bytecode_emu import Program  # noqa: E402
from parity import near_tie  # noqa: E402


@pytest.fixture(scope="module")
def nc():
    from paper_2604_27058_gb300 import build
    build.build()
    import paper_2604_27058_gb300 as m
    return m


def _check(nc, text, shots, seed, postselect=False, max_flag=2, peephole=True):
    prog = nc.compile(text, peephole=peephole)
    fl = flatten(text)
    emu = Program(prog.serialize(), fl.site_p, fl.site_kind)
    sim = FactoredSim(text, k_limit=24)
    assert emu.ref_det == sim.ref_det and emu.ref_obs == sim.ref_obs
    n = flagged = 0
    for s in range(shots):
        tr = {}
        raw = sim.run_raw(seed, s, trace=tr)[0]
        if near_tie(tr.get("p1", {}), seed, s):
            flagged += 1
            continue
        want = assemble(sim.flat, raw, sim.ref_det, sim.ref_obs, postselect)
        got = emu.run(seed, s, postselect=postselect)
        assert got["meas"] == want.meas, s
        assert got["det"] == want.det, s
        assert got["obs"] == want.obs, s
        assert got["kept"] == want.kept, s
        if sim.flat.n_probes:
            alive = probe_alive(sim.flat, raw, sim.ref_det, postselect)
            for j in range(sim.flat.n_probes):
                assert abs(got["probes"][j] - tr["probe"][j] * alive[j]) <= 1e-10, (s, j)
        n += 1
    assert flagged <= max_flag
    return n


@pytest.mark.parametrize("peephole", [True, False])
@pytest.mark.parametrize("seed", range(8))
def test_random_circuits(nc, seed, peephole):
    text = gc.random_small(3100 + seed, n=6, n_ops=90, p_noise=0.06 if seed % 2 else 0.0, t_frac=0.3)
    assert _check(nc, text, 40, 17 + seed, peephole=peephole) >= 38


@pytest.mark.parametrize("seed", range(4))
def test_random_circuits_with_probes(nc, seed):
    text = gc.with_probes(gc.random_small(3200 + seed, n=6, n_ops=90, p_noise=0.05, t_frac=0.3), seed, count=8)
    assert _check(nc, text, 30, 5 + seed) >= 28


def test_coherent_surface_code(nc):
    assert _check(nc, gc.surface_code_memory(d=3, rounds=1, p=0.01, theta=0.05), 40, 6006) >= 38


def test_surface_code(nc):
    assert _check(nc, gc.surface_code_memory(d=3, rounds=2, p=0.02), 60, 2002, max_flag=0) == 60


def test_fig4_and_tiny(nc):
    assert _check(nc, gc.fig4_example(0.05), 60, 7) >= 58
    assert _check(nc, gc.tiny_random(seed=1), 20, 1001) >= 18


def test_low_magic_postselected(nc):
    assert _check(nc, gc.low_magic_gadgets(), 8, 4004, postselect=True) >= 7


def test_stratified_fault_sets_through_the_noise_tables(nc):
    """Shots of stratum K = 4 (the oracle's conditional fault sets) applied
    through the compiled noise tables give the oracle's records."""
    from oracle.strata import build_strata, sample_stratum_faults
    text = gc.surface_code_memory(d=3, rounds=3, p=0.01)
    prog = nc.compile(text)
    fl = flatten(text)
    emu = Program(prog.serialize(), fl.site_p, fl.site_kind)
    sim = FactoredSim(text)
    t = build_strata(fl.site_p, fl.site_kind, 4)
    for s in range(40):
        f = sample_stratum_faults(t, 9, s, 4)
        want = assemble(sim.flat, sim.run_raw(9, s, faults=f)[0], sim.ref_det, sim.ref_obs, False)
        got = emu.run(9, s, faults=f)
        assert (got["meas"], got["det"], got["obs"]) == (want.meas, want.det, want.obs), s


def test_sweep_mirror_circuits(nc):
    """Two of the sweep's mirror circuits with the most T gates (k_max up to
    14): every shot's records equal the oracle's."""
    circs = [gc.sweep_mirror(i) for i in range(64)]
    picks = sorted(range(64), key=lambda i: (-circs[i].t, circs[i].n * circs[i].depth))[:2]
    for i in picks:
        assert _check(nc, circs[i].text, 4, 5005 + i) >= 3


def test_coherent_d5_one_round(nc):
    """k_max = 12 after the HIR peephole; the plain oracle reaches 24 on the
    same circuit and gives the same records."""
    text = gc.surface_code_memory(d=5, rounds=1, p=1e-3, theta=0.02)
    assert nc.compile(text).info.k_max == 12
    assert FactoredSim(text, k_limit=24).k_max == 24
    assert _check(nc, text, 6, 31) >= 5


def test_peephole_fires_on_most_random_circuits(nc):
    """The random circuits above exercise the rule: it removes rotations
    (fewer array instructions) in at least a quarter of them."""
    fired = 0
    for seed in range(8):
        text = gc.random_small(3100 + seed, n=6, n_ops=90, p_noise=0.0, t_frac=0.3)
        fired += nc.compile(text).info.n_array_ops < nc.compile(text, peephole=False).info.n_array_ops
    assert fired >= 2
