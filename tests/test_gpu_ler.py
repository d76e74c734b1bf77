"""Logical-error-rate agreement between the CUDA path and the FP64 oracle:
the rates of the same circuit, sampled with independent seeds (10^7 to 10^8
shots on the GPU, 4*10^4 to 10^5 on the oracle), pass a two-proportion test
at 99 %: |p_gpu - p_oracle| <= 2.576 sqrt(pbar (1 - pbar) (1/n_gpu + 1/n_oracle)).

Rates compared: for the postselected low-magic workload (n = 50, k_max = 10,
150 detectors), the kept fraction and the logical-error rate per kept shot
(observable flipped); for three sweep circuits (mirror circuits U U^dagger
with T gates, k_max 1 to 12, whose failure rate is well below 1), the
failure rate (any nonzero final record) and the observable flip rate. The
oracle runs in a spawn process pool over the host cores."""

import pytest

from gen import circuits as gc

from parity import gpu_rates, oracle_rates, two_proportion_ok

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_27058_gb300 import build
    build.build()
    import paper_2604_27058_gb300 as m
    return m


def test_low_magic_postselected_rates(nc):
    text = gc.low_magic_gadgets()
    n_o, kept_o, fail_o, _ = oracle_rates(text, 4104, 100_000, postselect=True)
    prog = nc.compile(text)
    n_g, kept_g, fail_g, _ = gpu_rates(prog, 100_000_000, 4004, postselect=True)
    assert 0.2 < kept_o / n_o < 0.8
    assert two_proportion_ok(kept_g, n_g, kept_o, n_o), (kept_g / n_g, kept_o / n_o)
    assert two_proportion_ok(fail_g, kept_g, fail_o, kept_o), (fail_g / kept_g, fail_o / kept_o)


@pytest.mark.parametrize("index", [45, 39, 46])
def test_sweep_circuit_rates(nc, index):
    c = gc.sweep_mirror(index)
    n_o, _, obs_o, fail_o = oracle_rates(c.text, 5105 + index, 40_000)
    prog = nc.compile(c.text)
    n_g, _, obs_g, fail_g = gpu_rates(prog, 10_000_000, 5005 + index)
    assert 0.05 < fail_o / n_o < 0.95
    assert two_proportion_ok(fail_g, n_g, fail_o, n_o), (fail_g / n_g, fail_o / n_o)
    assert two_proportion_ok(obs_g, n_g, obs_o, n_o), (obs_g / n_g, obs_o / n_o)
