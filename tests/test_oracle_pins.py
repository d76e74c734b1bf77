"""Pins of the three oracle simulators against closed forms, the paper's
worked example, invariants and each other (CPU only)."""

import itertools
import math
import os

import numpy as np
import pytest

from gen import circuits as gc
from oracle.dense import DenseSim
from oracle.factored import FactoredSim
from oracle.stabilizer import FrameSim

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _p1(sim_cls, text, event=0, seed=1, shot=0):
    sim = sim_cls(text)
    if sim_cls is DenseSim:
        return sim.run_raw(seed, shot)[1][event]
    tr = {}
    sim.run_raw(seed, shot, trace=tr)
    return tr["p1"][event]


@pytest.mark.parametrize("cls", [DenseSim, FactoredSim])
def test_t_on_plus_measured_in_x(cls):
    # P(m = 0) = cos^2(pi/8) for T|+> measured in X
    assert abs((1 - _p1(cls, "H 0\nT 0\nMX 0\n")) - math.cos(math.pi / 8) ** 2) < 1e-12


@pytest.mark.parametrize("cls", [DenseSim, FactoredSim])
def test_hth_measured_in_z(cls):
    assert abs(_p1(cls, "H 0\nT 0\nH 0\nM 0\n") - math.sin(math.pi / 8) ** 2) < 1e-12


@pytest.mark.parametrize("cls", [DenseSim, FactoredSim])
@pytest.mark.parametrize("theta", [0.3, -1.1, 2.5])
def test_rotation_closed_forms(cls, theta):
    s2 = math.sin(theta / 2) ** 2
    assert abs(_p1(cls, f"H 0\nR_Z({theta}) 0\nH 0\nM 0\n") - s2) < 1e-12
    assert abs(_p1(cls, f"R_X({theta}) 0\nM 0\n") - s2) < 1e-12
    assert abs(_p1(cls, f"R_Y({theta}) 0\nM 0\n") - s2) < 1e-12
    # R_Y about an entangled pair: measuring the partner after a CX
    assert abs(_p1(cls, f"R_Y({theta}) 0\nCX 0 1\nM 1\n") - s2) < 1e-12


@pytest.mark.parametrize("cls", [DenseSim, FactoredSim])
def test_t_powers(cls):
    assert _p1(cls, "H 0\n" + "T 0\n" * 8 + "H 0\nM 0\n") < 1e-12        # T^8 = I
    assert _p1(cls, "H 0\nT 0\nT 0\nS_DAG 0\nH 0\nM 0\n") < 1e-12       # T^2 = S
    assert _p1(cls, "H 0\nT 0\nT_DAG 0\nH 0\nM 0\n") < 1e-12             # T T^dag = I


def test_t_squared_equals_s_state():
    a = DenseSim("H 0\nT 0\nT 0\nM 0\n").run_raw(1, 0, stop_event=0)[2]
    b = DenseSim("H 0\nS 0\nM 0\n").run_raw(1, 0, stop_event=0)[2]
    assert abs(abs(np.vdot(a, b)) - 1) < 1e-12


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_ghz_t_parity_dense_exact(n):
    # GHZ_n with T on every qubit: P(X^n parity even) = (1 + cos(n pi/4)) / 2
    sim = DenseSim(gc.ghz_t_parity(n))
    psi = sim.run_raw(1, 0, stop_event=0)[2]
    h = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    t = psi.reshape([2] * n)
    for ax in range(n):
        t = np.moveaxis(np.tensordot(h, t, axes=([1], [ax])), 0, ax)
    probs = np.abs(t.reshape(-1)) ** 2
    even = sum(p for i, p in enumerate(probs) if bin(i).count("1") % 2 == 0)
    assert abs(even - (1 + math.cos(n * math.pi / 4)) / 2) < 1e-12


@pytest.mark.parametrize("n", [3, 5])
def test_ghz_t_parity_factored_statistics(n):
    sim = FactoredSim(gc.ghz_t_parity(n))
    shots = 3000
    even = sum(1 for s in range(shots) if sum(sim.sample(2, s).meas) % 2 == 0)
    p = (1 + math.cos(n * math.pi / 4)) / 2
    assert abs(even / shots - p) <= 5 * math.sqrt(p * (1 - p) / shots) + 1e-9


def _golden_circuit(name):
    lines = []
    for line in open(os.path.join(GOLDEN, name)):
        if not line.startswith("#"):
            lines.append(line)
    return "".join(lines)


@pytest.mark.parametrize("cls", [DenseSim, FactoredSim])
def test_fig4_example_noiseless(cls):
    assert _golden_circuit("fig4_example.txt") == gc.fig4_example(0.001)
    text = gc.fig4_example(0.0)
    for shot in range(20):
        sim = cls(text)
        if cls is DenseSim:
            m, p, _ = sim.run_raw(4, shot)
        else:
            tr = {}
            m = sim.run_raw(4, shot, trace=tr)[0]
            p = tr["p1"]
        assert abs(p[0] - 0.5) < 1e-12
        assert p[1] < 1e-12 and m[1] == 0


def test_fig4_example_shape_in_factored_plan():
    """Fig. 4's lowering: a dormant-static Z1 measurement, one expansion
    (OP_EXPAND_T) and an interfering active measurement on qubit 0."""
    sim = FactoredSim(gc.fig4_example())
    kinds = [st.kind for st in sim.steps]
    assert kinds.count("expand") == 1
    assert sim.k_max == 1
    assert [st.kind for st in sim.steps if st.kind.startswith("m")] == ["mact", "mstatic"]
    act = [st for st in sim.steps if st.kind == "mact"][0]
    assert act.a["kind"] == "X"


@pytest.mark.parametrize("seed", range(8))
def test_mirror_circuits_return_to_zero(seed):
    text = gc.mirror_small(seed, n=6, depth=10)
    fa = FactoredSim(text)
    fb = DenseSim(text)
    for shot in range(4):
        assert fa.sample(5, shot).meas == [0] * 6
        assert fb.sample(5, shot).meas == [0] * 6


def test_mirror_clifford_frame_sim():
    text = gc.mirror_small(3, n=7, depth=12).replace("T_DAG", "S_DAG").replace("T ", "S ")
    text = "\n".join(l for l in text.splitlines() if not l.startswith("R_Z")) + "\n"
    sim = FrameSim(text)
    for shot in range(5):
        assert sim.sample(1, shot).meas == [0] * 7


@pytest.mark.parametrize("cls", [DenseSim, FactoredSim, FrameSim])
@pytest.mark.parametrize("chan,p,expect", [
    ("X_ERROR", 0.3, 0.3), ("Y_ERROR", 0.3, 0.3), ("Z_ERROR", 0.3, 0.0),
    ("DEPOLARIZE1", 0.3, 0.2),
])
def test_noise_marginals(cls, chan, p, expect):
    sim = cls(f"{chan}({p}) 0\nM 0\n")
    n = 4000
    ones = sum(sim.sample(8, s).meas[0] for s in range(n))
    sd = math.sqrt(max(expect * (1 - expect), 1e-9) / n)
    assert abs(ones / n - expect) <= 5 * sd


@pytest.mark.parametrize("cls", [DenseSim, FactoredSim, FrameSim])
def test_depolarize2_marginal_and_flip(cls):
    sim = cls("DEPOLARIZE2(0.45) 0 1\nM 0\nM(0.2) 1\n")
    n = 4000
    a = b = 0
    for s in range(n):
        m = sim.sample(6, s).meas
        a += m[0]
        b += m[1]
    pa = 8 * 0.45 / 15
    pb = pa * 0.8 + (1 - pa) * 0.2
    assert abs(a / n - pa) <= 5 * math.sqrt(pa * (1 - pa) / n)
    assert abs(b / n - pb) <= 5 * math.sqrt(pb * (1 - pb) / n)


def test_factored_invariants_and_fixed_schedule():
    """Norm 1, k <= N, k <= number of rotations so far, and the runtime k
    trajectory equals the planned one for every shot (Thm. 1)."""
    text = gc.random_small(17, n=6, n_ops=120, p_noise=0.05, t_frac=0.35)
    sim = FactoredSim(text)
    n_rot_so_far = []
    cnt = 0
    for st in sim.steps:
        if st.kind in ("expand",):
            cnt += 1
        n_rot_so_far.append(cnt)
    traj = None
    for shot in range(8):
        tr = {}
        sim.run_raw(3, shot, trace=tr)
        assert max(abs(x - 1) for x in tr["norm"]) < 1e-10
        assert max(tr["k"]) <= 6
        assert all(k <= r for k, r in zip(tr["k"], n_rot_so_far))
        if traj is None:
            traj = tr["k"]
        assert tr["k"] == traj


@pytest.mark.parametrize("seed", range(12))
def test_frame_sim_equals_dense(seed):
    text = gc.random_small(1000 + seed, n=5, n_ops=60, p_noise=0.05, rotations=False)
    d, f = DenseSim(text), FrameSim(text)
    for shot in range(10):
        assert d.run_raw(21, shot)[0] == f.run_raw(21, shot)[0]


@pytest.mark.parametrize("seed", range(16))
def test_factored_equals_dense(seed):
    n = 3 + seed % 5
    text = gc.random_small(2000 + seed, n=n, n_ops=70, p_noise=0.04 if seed % 2 else 0.0,
                           t_frac=0.3, meas_frac=0.12)
    d, f = DenseSim(text), FactoredSim(text)
    for shot in range(6):
        md, pd, _ = d.run_raw(31, shot)
        tr = {}
        mf = f.run_raw(31, shot, trace=tr)[0]
        assert md == mf
        for e, p in pd.items():
            assert abs(p - tr["p1"][e]) < 1e-10


def _pauli_expectations_dense(psi, n):
    mats = {"I": np.eye(2), "X": np.array([[0, 1], [1, 0]]),
            "Y": np.array([[0, -1j], [1j, 0]]), "Z": np.diag([1, -1])}
    out = {}
    for word in itertools.product("IXYZ", repeat=n):
        m = np.array([[1]])
        for q in range(n - 1, -1, -1):
            m = np.kron(m, mats[word[q]])
        out[word] = float(np.real(np.vdot(psi, m @ psi)))
    return out


def _pauli_expectations_factored(sim, fx, fz, phi, act, n):
    """<psi|P|psi> with psi = U_C P~ (phi (x) 0_D):
    = (-1)^[M(P) anticommutes with P~] <phi (x) 0| M(P) |phi (x) 0>."""
    xm = np.array([[0, 1], [1, 0]])
    zm = np.diag([1, -1])
    out = {}
    for word in itertools.product("IXYZ", repeat=n):
        x, z, ph = sim._map({q: l for q, l in enumerate(word) if l != "I"})
        anti = (bin(x & fz).count("1") + bin(z & fx).count("1")) & 1
        if any((x >> q) & 1 and q not in act for q in range(n)):
            out[word] = 0.0
            continue
        mat = np.array([[1]])
        for pos in range(len(act) - 1, -1, -1):
            v = act[pos]
            mat = np.kron(mat, np.linalg.matrix_power(xm, (x >> v) & 1)
                          @ np.linalg.matrix_power(zm, (z >> v) & 1))
        val = (1j ** ph) * np.vdot(phi, mat @ phi) * (-1 if anti else 1)
        out[word] = float(np.real(val))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_factored_state_matches_dense_expansion(seed):
    """Dense-expansion check (Sec. 3.3): the physical state U_C P~ (phi (x) 0)
    equals O-B's state. Compared through all 4^n Pauli expectation values,
    which determine the density matrix, for random unitary Clifford+rotation
    circuits with noise fixed by the shot (n = 3, 4)."""
    n = 3 + seed % 2
    text = gc.random_small(3000 + seed, n=n, n_ops=50, p_noise=0.1, t_frac=0.35, meas_frac=0.0,
                           feedforward=False)
    text = "\n".join(l for l in text.splitlines() if not l.startswith("M ")) + "\n"
    d = DenseSim(text)
    f = FactoredSim(text)
    for shot in range(3):
        psi = d.run_raw(9, shot)[2]
        _, (fx, fz), phi, act = f.run_raw(9, shot)
        ed = _pauli_expectations_dense(psi, n)
        ef = _pauli_expectations_factored(f, fx, fz, phi, act, n)
        for w in ed:
            assert abs(ed[w] - ef[w]) < 1e-10, (w, ed[w], ef[w])


def _pair_probabilities(order_x=True):
    """Exact P(m = 1) of MX on qubit a, then on b given a's outcome, for the
    two-qubit block CZ (T|+>)^2, by brute force on its 4 amplitudes."""
    w = np.exp(1j * math.pi / 4)
    v = np.array([1, w, w, -w * w], dtype=complex) / 2  # index 2 * bit_a + bit_b
    h = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    vx = np.kron(h, h) @ v  # X basis of both qubits
    pa = abs(vx[2]) ** 2 + abs(vx[3]) ** 2
    pb = {0: abs(vx[1]) ** 2 / (abs(vx[0]) ** 2 + abs(vx[1]) ** 2),
          1: abs(vx[3]) ** 2 / (abs(vx[2]) ** 2 + abs(vx[3]) ** 2)}
    return pa, pb


@pytest.mark.parametrize("n", [16, 18])
def test_large_k_probabilities_closed_form(n):
    """Active dimension above the dense oracle's reach: H and T on n qubits
    (k = n), CZ on disjoint pairs, then MX on every qubit. The state is a
    product of identical two-qubit blocks, so every measurement probability
    along the cascade (k = n down to 1) is fixed by the block alone."""
    text = "".join(f"H {q}\nT {q}\n" for q in range(n))
    text += "".join(f"CZ {q} {q + 1}\n" for q in range(0, n, 2))
    text += "MX " + " ".join(map(str, range(n))) + "\n"
    sim = FactoredSim(text, k_limit=n)
    assert sim.k_max == n
    pa, pb = _pair_probabilities()
    for shot in range(3):
        tr = {}
        meas = sim.run_raw(5, shot, trace=tr)[0]
        for q in range(0, n, 2):
            assert tr["p1"][q] == pytest.approx(pa, abs=1e-12)
            assert tr["p1"][q + 1] == pytest.approx(pb[meas[q]], abs=1e-12)
