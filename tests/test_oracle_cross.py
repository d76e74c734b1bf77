"""Larger cross-checks between the oracle simulators, postselection semantics,
and planted-mistake tests: a plausible error planted in O-A (on the CPU) must
make its cross-check against O-B fail."""

import copy

import pytest

from gen import circuits as gc
from oracle.dense import DenseSim
from oracle.factored import FactoredSim
from oracle.stabilizer import FrameSim


def test_factored_equals_frame_sim_on_surface_code():
    text = gc.surface_code_memory(d=5, rounds=25, p=1e-3)
    a, b = FactoredSim(text), FrameSim(text)
    assert a.k_max == 0
    assert sum(a.ref_det) == 0 and a.ref_obs == [0]
    flips = 0
    for s in range(40):
        ra, rb = a.sample(2002, s), b.sample(2002, s)
        assert (ra.meas, ra.det, ra.obs) == (rb.meas, rb.det, rb.obs)
        flips += sum(ra.det)
    assert flips > 0


def test_factored_equals_frame_sim_on_large_random_clifford():
    text = gc.random_small(4242, n=30, n_ops=400, p_noise=0.01, rotations=False, meas_frac=0.15)
    a, b = FactoredSim(text), FrameSim(text)
    for s in range(20):
        assert a.run_raw(5, s)[0] == b.run_raw(5, s)[0]


def test_postselection_semantics():
    text = ("X_ERROR(0.5) 0\nM 0\nDETECTOR rec[-1]\nX 1\nM 1\nDETECTOR rec[-1]\n"
            "M 2\nOBSERVABLE_INCLUDE(0) rec[-2]\n")
    for cls in (DenseSim, FactoredSim, FrameSim):
        sim = cls(text)
        assert sim.ref_det == [0, 1] and sim.ref_obs == [1]
        seen = set()
        for s in range(64):
            r = sim.sample(3, s, postselect=True)
            raw = sim.sample(3, s, postselect=False)
            assert raw.kept == 1 and raw.det[1] == 0 and raw.obs == [0]
            if raw.meas[0] == 1:
                # rejected at detector 0: it reports 1, later records 0
                assert r.kept == 0 and r.det == [1, 0] and r.meas == [1, 0, 0] and r.obs == [0]
            else:
                assert r.kept == 1 and r.det == [0, 0] and r.meas == [0, 1, 0]
            seen.add(r.kept)
        assert seen == {0, 1}


def test_low_magic_gadgets_deterministic_and_kmax():
    text = gc.low_magic_gadgets()
    sim = FactoredSim(text)
    assert sim.k_max <= 10
    for s in range(3):
        meas = sim.run_raw(11, s, noisy=False)[0]
        from oracle.records import raw_parities
        det, obs = raw_parities(sim.flat, meas)
        assert det == sim.ref_det and obs == sim.ref_obs


# ---------------------------------------------------------------------------
# planted mistakes
# ---------------------------------------------------------------------------
def _mismatch_found(mutate, seeds=range(6)) -> bool:
    for seed in seeds:
        text = gc.random_small(5000 + seed, n=4, n_ops=70, p_noise=0.05, t_frac=0.3, meas_frac=0.12)
        d = DenseSim(text)
        f = FactoredSim(text)
        f.steps = mutate(copy.deepcopy(f.steps))
        for shot in range(8):
            md, pd, _ = d.run_raw(13, shot)
            tr = {}
            try:
                mf = f.run_raw(13, shot, trace=tr)[0]
            except Exception:
                return True
            if md != mf or any(abs(pd[e] - tr["p1"].get(e, -1)) > 1e-9 for e in pd):
                return True
    return False


def _flip_sign_bits(steps):
    for st in steps:
        if st.kind in ("mact", "mrand"):
            st.a["a"] ^= 1
    return steps


def _negate_angles(steps):
    for st in steps:
        if st.kind in ("rot", "expand"):
            st.a["theta"] = -st.a["theta"]
    return steps


def _drop_xflips(steps):
    return [st for st in steps if st.kind != "xflip"]


def _drop_cz(steps):
    return [st for st in steps if not (st.kind == "vg" and st.a["name"] == "CZ")]


def _swap_noise_xz(steps):
    for st in steps:
        if st.kind == "noise" and len(st.a["opts"]) == 3:
            o = st.a["opts"]
            st.a["opts"] = [o[2], o[1], o[0]]
    return steps


@pytest.mark.parametrize("mutate", [_flip_sign_bits, _negate_angles, _drop_xflips, _drop_cz,
                                    _swap_noise_xz])
def test_planted_mistake_is_caught(mutate):
    assert _mismatch_found(mutate)


def test_unmutated_passes_same_harness():
    assert not _mismatch_found(lambda s: s)


def test_reference_is_the_most_likely_trajectory():
    """Detector references come from the noiseless trajectory in which every
    measurement takes its more likely outcome: for the coherent-noise surface
    code that is the rotation-free circuit's reference, and a near-
    deterministic detector gets the likely value."""
    from gen import circuits as gc
    from oracle.factored import FactoredSim
    from oracle.stabilizer import FrameSim
    for d, r in ((3, 1), (3, 3)):
        coh = FactoredSim(gc.surface_code_memory(d=d, rounds=r, p=1e-3, theta=0.02))
        cliff = FrameSim(gc.surface_code_memory(d=d, rounds=r, p=1e-3))
        assert coh.ref_det == cliff.ref_det and coh.ref_obs == cliff.ref_obs
    assert FactoredSim("R_X(0.1) 0\nM 0\nDETECTOR rec[-1]").ref_det == [0]
    assert FactoredSim("R_X(3.0) 0\nM 0\nDETECTOR rec[-1]").ref_det == [1]
