"""Pins for the oracle's expectation-value probes (CPU only).

The factored oracle (O-A) computes <P> from the frame, the Heisenberg image
M(P) and the active vector; the dense oracle (O-B) from the physical state
vector. They are pinned by closed forms and by agreement with each other on
random noisy circuits with measurements, resets and feed-forward (a wrong
frame sign, a missed Y phase or a wrong position mask fails this)."""

import math

import pytest

from gen import circuits as gc
from oracle.dense import DenseSim
from oracle.factored import FactoredSim
from oracle.records import probe_alive


def _probes_factored(text, seed, shot):
    sim = FactoredSim(text)
    tr = {}
    sim.run_raw(seed, shot, trace=tr)
    return [tr["probe"][i] for i in range(sim.flat.n_probes)]


def _probes_dense(text, seed, shot):
    sim = DenseSim(text)
    pr = {}
    sim.run_raw(seed, shot, probes=pr)
    return [pr[i] for i in range(sim.flat.n_probes)]


@pytest.mark.parametrize("text,want", [
    ("H 0\nT 0\nEXPVAL X0 Y0 Z0", [math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0]),
    ("R_X(0.3) 0\nEXPVAL Z0 Y0 X0", [math.cos(0.3), -math.sin(0.3), 0.0]),
    ("R_Y(0.7) 0\nEXPVAL Z0 X0 Y0", [math.cos(0.7), math.sin(0.7), 0.0]),
    ("H 0\nCX 0 1\nCX 1 2\nEXPVAL X0*X1*X2 Z0*Z1 Z0 Y0*Y1*X2", [1.0, 1.0, 0.0, -1.0]),
    ("H 0\nT 0\nCX 0 1\nEXPVAL X0*X1 Y0*X1 Z0*Z1", [math.cos(math.pi / 4), math.sin(math.pi / 4), 1.0]),
    ("X 0\nEXPVAL Z0 Z1", [-1.0, 1.0]),
])
def test_closed_forms(text, want):
    for got in (_probes_factored(text, 1, 0), _probes_dense(text, 1, 0)):
        assert got == pytest.approx(want, abs=1e-12)


@pytest.mark.parametrize("seed", range(12))
def test_factored_equals_dense_on_random_noisy_circuits(seed):
    base = gc.random_small(700 + seed, n=5, n_ops=70, p_noise=0.08, t_frac=0.3)
    text = gc.with_probes(base, seed, count=8)
    fs, ds = FactoredSim(text), DenseSim(text)
    n = 0
    for shot in range(6):
        tr, pr = {}, {}
        mf = fs.run_raw(31, shot, trace=tr)[0]
        md = ds.run_raw(31, shot, probes=pr)[0]
        if mf != md:  # a near-tie measurement took different branches
            continue
        for i in range(fs.flat.n_probes):
            assert tr["probe"][i] == pytest.approx(pr[i], abs=1e-10), (seed, shot, i)
        n += 1
    assert n >= 4


def test_probes_after_postselection_rejection_are_masked():
    text = "X_ERROR(1) 0\nM 0\nDETECTOR rec[-1]\nEXPVAL Z1\nH 1\nEXPVAL X1"
    text_ref = "M 0\nDETECTOR rec[-1]\nEXPVAL Z1\nH 1\nEXPVAL X1"
    fs = FactoredSim(text_ref)
    sim = FactoredSim(text)
    meas = sim.run_raw(1, 0)[0]
    assert probe_alive(sim.flat, meas, fs.ref_det, postselect=True) == [0, 0]
    assert probe_alive(sim.flat, meas, fs.ref_det, postselect=False) == [1, 1]


def test_parse_errors():
    from oracle.circuit import CircuitError, flatten
    for bad in ("EXPVAL X0*X0", "EXPVAL Q1", "EXPVAL(1) X0", "EXPVAL"):
        with pytest.raises(CircuitError):
            flatten(bad)
    assert flatten("EXPVAL X3*Z1 Y0").n_probes == 2


def _planted(kind):
    import numpy as np
    from oracle import factored

    def bad(a, fx, fz, phi):
        if a["zero"]:
            return 0.0 if kind != "no_zero" else 1.0
        om = (bin(fx & a["z"]).count("1") + bin(fz & a["x"]).count("1")) & 1
        if kind == "no_frame_sign":
            om = 0
        if kind == "half_frame_sign":
            om = bin(fx & a["z"]).count("1") & 1
        idx = np.arange(len(phi))
        sg = 1 - 2 * (np.array([bin(int(i) & a["mz"]).count("1") & 1 for i in idx]))
        acc = np.sum(np.conj(phi[idx ^ a["mx"]]) * sg * phi)
        ph = 1 if kind == "no_phase" else 1j ** a["ph"]
        return float(((-1) ** om * ph * acc).real / np.sum(np.abs(phi) ** 2))
    return factored, bad


@pytest.mark.parametrize("kind", ["no_frame_sign", "half_frame_sign", "no_phase", "no_zero"])
def test_planted_mistakes_fail_a_pin(monkeypatch, kind):
    """A mistake planted in the oracle's probe (on the CPU) fails a pin."""
    mod, bad = _planted(kind)
    monkeypatch.setattr(mod, "probe_value", bad)
    failed = False
    for fn, args in ((test_closed_forms, None), (test_factored_equals_dense_on_random_noisy_circuits, None)):
        try:
            if fn is test_closed_forms:
                for text, want in [("H 0\nT 0\nEXPVAL X0 Y0 Z0", [math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0]),
                                   ("H 0\nCX 0 1\nCX 1 2\nEXPVAL X0*X1*X2 Z0*Z1 Z0 Y0*Y1*X2", [1.0, 1.0, 0.0, -1.0])]:
                    fn(text, want)
            else:
                for seed in range(12):
                    fn(seed)
        except AssertionError:
            failed = True
    assert failed
