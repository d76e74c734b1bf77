"""The compiled program, run by a plain Python interpreter of its instruction
list (tests/helpers/bytecode_emu.py), against the factored oracle, shot by
shot (CPU, no GPU). This checks the compiler's instructions, masks, noise
tables, record slots, probes and HIR passes end to end. The oracle is the
plain method (no HIR pass), so the programs compiled with the passes on
check that they change no record. Records must be equal except flagged
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


def _check(nc, text, shots, seed, postselect=False, max_flag=2, peephole=True, flags=None):
    prog = nc.compile(text, peephole=peephole, flags=flags)
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
    """k_max = 12 after the HIR passes; the plain oracle reaches 24 on the
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


# HIR passes one at a time (NC_COMPILE_* bits: 1 peephole, 2 reorder, 4
# fusion off), and all of them, against the plain oracle
HIR_FLAGS = {"all": 0, "fuse_only": 3, "reorder_only": 5, "peephole_only": 6}


def _clifford_t(seed, n=4, n_ops=70, noise=0.0):
    """Random circuits dense in T, T_DAG, S and R_Z, with mid-circuit
    measurements and resets, so that rotations about one axis often meet
    (fusion, cancellation, Clifford angles) and measurements can move."""
    import random
    rng = random.Random(seed)
    lines = []
    for _ in range(n_ops):
        r = rng.random()
        q = rng.randrange(n)
        if r < 0.35:
            lines.append(f"{rng.choice(['T', 'T', 'T_DAG', 'S'])} {q}")
        elif r < 0.45:
            lines.append(f"R_Z({rng.choice([0.3, -0.3, 0.7853981633974483, 1.5707963267948966])}) {q}")
        elif r < 0.6:
            lines.append(f"{rng.choice(['H', 'SQRT_X'])} {q}")
        elif r < 0.8:
            b = rng.randrange(n - 1)
            b += b >= q
            lines.append(f"{rng.choice(['CX', 'CZ'])} {q} {b}")
            if noise:
                lines.append(f"DEPOLARIZE2({noise}) {q} {b}")
        elif r < 0.9:
            lines.append(f"{rng.choice(['M', 'MX', 'MR'])} {q}")
        else:
            lines.append(f"X_ERROR({noise or 0.1}) {q}")
    lines.append("M " + " ".join(str(q) for q in range(n)))
    return "\n".join(lines) + "\n"


@pytest.mark.parametrize("which", sorted(HIR_FLAGS))
@pytest.mark.parametrize("seed", range(6))
def test_hir_passes_keep_records(nc, seed, which):
    text = _clifford_t(4100 + seed, noise=0.03 if seed % 3 == 2 else 0.0)
    assert _check(nc, text, 40, 23 + seed, flags=HIR_FLAGS[which]) >= 38


@pytest.mark.parametrize("which", sorted(HIR_FLAGS))
def test_hir_passes_on_random_circuits_with_probes(nc, which):
    text = gc.with_probes(gc.random_small(3210, n=6, n_ops=90, p_noise=0.05, t_frac=0.3), 3, count=8)
    assert _check(nc, text, 30, 8, flags=HIR_FLAGS[which]) >= 28


def test_hir_passes_fire(nc):
    """Each pass changes the bytecode of some of these circuits (fewer array
    instructions, or a lower k_max)."""
    fired = {w: 0 for w in HIR_FLAGS}
    for seed in range(6):
        text = _clifford_t(4100 + seed)
        plain = nc.compile(text, peephole=False).info
        for w, f in HIR_FLAGS.items():
            i = nc.compile(text, flags=f).info
            fired[w] += (i.n_array_ops, i.k_max) < (plain.n_array_ops, plain.k_max)
    assert all(v >= 2 for v in fired.values()), fired


def test_phase_fusion_and_clifford_reabsorption(nc):
    """T T is the Clifford S (pi/4): fused and re-absorbed, nothing reaches
    the active vector; T T_DAG and T^8 are the identity; T T T stays one
    3 pi/8 rotation."""
    for body, arrays in (("T 0\nT 0", 0), ("T 0\nT_DAG 0", 0), ("T 0\n" * 8, 0), ("T 0\nT 0\nT 0", 1)):
        text = f"H 0\n{body}\nH 0\nM 0\n"
        plain = nc.compile(text, peephole=False).info
        opt = nc.compile(text, flags=3).info  # fusion alone
        assert plain.k_max == 1 and plain.n_array_ops >= 1
        assert (opt.k_max > 0) == bool(arrays)
        assert opt.n_array_ops == (0 if not arrays else 2)  # expansion + active measurement
        assert _check(nc, text, 40, 3, flags=3) >= 39
    # a re-absorbed S conjugates what follows: H S H then MX differs from H H
    text = "H 0\nT 0\nT 0\nCX 0 1\nT 1\nH 0\nMX 0\nM 1\n"
    assert nc.compile(text, flags=3).info.n_array_ops < nc.compile(text, peephole=False).info.n_array_ops
    assert _check(nc, text, 60, 11, flags=3) >= 59


def test_noiseless_mirrors_collapse(nc):
    """A noiseless U U^dagger: every T meets its T_DAG through commuting
    operations, so the optimised program has no active axis; the plain one
    expands."""
    for seed in range(4):
        text = gc.mirror_small(seed)
        assert nc.compile(text, peephole=False).info.k_max > 0
        info = nc.compile(text).info
        assert info.k_max == 0 and info.n_array_ops == 0
        assert _check(nc, text, 8, seed) == 8


def test_reorder_measures_before_expanding(nc):
    """31 qubits in |+> rotated by T, then qubit 0 measured in X: qubit 0's
    measurement commutes with the other 30 rotations and moves ahead of
    them, so the active dimension peaks at 30 instead of 31 (two such
    measurements among 12 rotations: 10 instead of 12)."""
    text = "".join(f"H {q}\nT {q}\n" for q in range(31)) + "H 0\nM 0\n"
    assert nc.compile(text, flags=5).info.k_max == 30
    text20 = "".join(f"H {q}\nT {q}\n" for q in range(12)) + "H 0\nM 0\nH 5\nM 5\n"
    assert nc.compile(text20, peephole=False).info.k_max == 12
    assert nc.compile(text20, flags=5).info.k_max == 10  # both measured before T 6..11
    assert _check(nc, text20, 40, 5, flags=5) >= 39


def test_coherent_rows_kmax(nc):
    """The four coherent-noise rows (R_Z(0.02) beside every depolarising
    channel): k_max after the HIR passes, against the paper's own compiled
    5 / 8 / 13 / 24 (Table 1), and the plain method's."""
    rows = {(3, 1): (4, 8), (3, 3): (8, 8), (5, 1): (12, 24), (5, 5): (24, 24)}
    for (d, r), (opt, plain) in rows.items():
        text = gc.surface_code_memory(d=d, rounds=r, p=1e-3, theta=0.02)
        assert nc.compile(text).info.k_max == opt
        assert nc.compile(text, peephole=False).info.k_max == plain
