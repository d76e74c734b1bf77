"""CPU-only checks of the C-ABI library: it builds, loads, exports every
symbol include/nc.h declares, and its host-side compiler behaves (no GPU
compute call is made here)."""

import ctypes
import os
import re

import pytest

from gen import circuits as gc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def nc():
    from paper_2604_27058_gb300 import build
    build.build()
    import paper_2604_27058_gb300 as m
    return m


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "nc.h")).read()
    return sorted(set(re.findall(r"\b(nc_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(nc):
    from paper_2604_27058_gb300 import _nc
    lib = _nc.lib()
    declared = _declared_symbols()
    assert set(declared) == set(_nc.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_status_strings(nc):
    from paper_2604_27058_gb300 import _nc
    lib = _nc.lib()
    for code in range(10):
        assert lib.nc_status_str(code)
    assert lib.nc_abi_version() >> 16 >= 1


@pytest.mark.parametrize("name,text,kmax", [
    ("tiny", gc.tiny_random(), 6),
    ("surface", gc.surface_code_memory(), 0),
    ("dense", gc.dense_random(), 20),
    ("lowmagic", gc.low_magic_gadgets(), 10),
    ("coherent_d3_r3", gc.surface_code_memory(d=3, rounds=3, p=1e-3, theta=0.02), 8),
    ("coherent_d5_r1", gc.surface_code_memory(d=5, rounds=1, p=1e-3, theta=0.02), 12),
])
def test_compile_matches_oracle_schedule(nc, name, text, kmax):
    from oracle.circuit import flatten
    p = nc.compile(text)
    f = flatten(text)
    assert p.info.k_max == kmax
    assert (p.info.n_qubits, p.info.n_meas, p.info.n_det, p.info.n_obs) == (
        f.n_qubits, f.n_records, f.n_detectors, f.n_observables)
    assert p.info.n_noise_sites == f.n_sites
    assert p.info.n_events == f.n_events


def test_k_schedule_matches_oracle_plan(nc):
    """With the HIR peephole off, the compiled k_max is the plain method's
    (the oracle's plan); with it on (the default) it can only be lower."""
    from oracle.factored import FactoredSim
    for seed in range(10):
        text = gc.random_small(900 + seed, n=6, n_ops=80, t_frac=0.3)
        plain = FactoredSim(text).k_max
        assert nc.compile(text, peephole=False).info.k_max == plain
        assert nc.compile(text).info.k_max <= plain
    for (d, r), (opt, plain) in zip(((3, 1), (3, 3), (5, 1)), ((4, 8), (8, 8), (12, 24))):
        text = gc.surface_code_memory(d=d, rounds=r, p=1e-3, theta=0.02)
        assert nc.compile(text, peephole=False).info.k_max == FactoredSim(text, k_limit=24).k_max == plain
        assert nc.compile(text).info.k_max == opt


def test_unknown_compile_flag_rejected(nc):
    import ctypes
    from paper_2604_27058_gb300 import _nc
    h = ctypes.c_void_p()
    code = _nc.lib().nc_compile_ex(b"H 0\nM 0\n", 8, 1 << 7, ctypes.byref(h), None, 0)
    assert _nc.STATUS[code] == "NC_E_ARG" and not h.value


def test_serialize_roundtrip(nc):
    p = nc.compile(gc.surface_code_memory(d=3, rounds=3))
    blob = p.serialize()
    q = nc.Program.deserialize(blob)
    assert q.serialize() == blob
    assert q.info == p.info
    with pytest.raises(nc.NcError) as e:
        nc.Program.deserialize(blob[:-8])
    assert e.value.name == "NC_E_ARG"
    bad = bytearray(blob)
    bad[0] ^= 0xFF
    with pytest.raises(nc.NcError):
        nc.Program.deserialize(bytes(bad))


@pytest.mark.parametrize("text,code", [
    ("FOO 1\n", "NC_E_UNSUPPORTED"),
    ("M 0\nDETECTOR rec[-2]\n", "NC_E_PARSE"),
    ("H 0\nREPEAT 2 {\nH 0\n", "NC_E_PARSE"),
    ("X_ERROR(1.5) 0\n", "NC_E_PARSE"),
    ("CX 0 0\n", "NC_E_PARSE"),
    ("CX 0\n", "NC_E_PARSE"),
    ("R_Z 0\n", "NC_E_PARSE"),
    ("}\n", "NC_E_PARSE"),
])
def test_compile_errors(nc, text, code):
    with pytest.raises(nc.NcError) as e:
        nc.compile(text)
    assert e.value.name == code


def test_kmax_limit(nc):
    text = "".join(f"H {q}\nT {q}\n" for q in range(31)) + "H 0\nM 0\n"
    with pytest.raises(nc.NcError) as e:
        nc.compile(text, peephole=False)
    assert e.value.name == "NC_E_KMAX"
    # the HIR reorder measures qubit 0 right after its own rotation (it
    # commutes with the other 30), so the optimised program stays at 30 axes
    assert nc.compile(text).info.k_max == 30
    with pytest.raises(nc.NcError) as e:
        nc.compile("".join(f"H {q}\nT {q}\n" for q in range(31)))
    assert e.value.name == "NC_E_KMAX"


def test_repeat_and_aliases(nc):
    a = nc.compile("REPEAT 3 {\nCNOT 0 1\nMZ 1\n}\n")
    b = nc.compile("CX 0 1\nM 1\nCX 0 1\nM 1\nCX 0 1\nM 1\n")
    assert a.info == b.info


def test_missing_library_fails_loudly(nc, monkeypatch):
    """No CPU fallback: without libnc.so the binding raises instead of
    sampling some other way."""
    from paper_2604_27058_gb300 import _nc
    monkeypatch.setattr(_nc, "LIB_PATH", "/nonexistent/libnc.so")
    monkeypatch.setattr(_nc, "_lib", None, raising=False)
    with pytest.raises(RuntimeError):
        _nc.lib()


def _plan_array_bytes(sim):
    """Array bytes per shot at FP32 from the oracle's plan (the same
    traversal count: expand 3 * 2^k, passes 2 * 2^k, active measurement
    2.5 * 2^k amplitudes of 8 bytes)."""
    k, b = 0, 0.0
    for st in sim.steps:
        if st.kind == "expand":
            b += 8 * 3 * 2 ** k
            k += 1
        elif st.kind == "rot" or (st.kind == "vg" and st.a["pos"] is not None):
            b += 8 * 2 * 2 ** k
        elif st.kind == "mact":
            b += 8 * 2.5 * 2 ** k
            k -= 1
    return b


@pytest.mark.parametrize("name", ["tiny", "lowmagic", "coherent", "small"])
def test_array_bytes_match_the_oracle_plan(nc, name):
    from oracle.factored import FactoredSim
    text = {"tiny": gc.tiny_random(), "lowmagic": gc.low_magic_gadgets(),
            "coherent": gc.surface_code_memory(d=3, rounds=3, p=1e-3, theta=0.02),
            "small": gc.random_small(77, n=6, n_ops=100, t_frac=0.3)}[name]
    got = nc.compile(text, peephole=False).info.array_bytes_fp32
    assert got == pytest.approx(_plan_array_bytes(FactoredSim(text)), rel=1e-12)
    assert nc.compile(text).info.array_bytes_fp32 <= got
    assert nc.compile(gc.surface_code_memory(d=3, rounds=2)).info.array_bytes_fp32 == 0.0


@pytest.mark.parametrize("name", ["dense", "dense_small", "tiny", "surface"])
def test_shared_prefix_matches_the_oracle_plan(nc, name):
    """The shared prefix ends at the first noise, measurement or record
    instruction; its active dimension is the number of expansions the
    oracle's plan makes before its first such step."""
    from oracle.factored import FactoredSim
    text = {"dense": gc.dense_random(), "dense_small": gc.dense_random(seed=33, n=10, layers=12),
            "tiny": gc.tiny_random(), "surface": gc.surface_code_memory(d=3, rounds=2)}[name]
    info = nc.compile(text, peephole=False).info  # the plain method, as the oracle's plan
    sim = FactoredSim(text)
    k = 0
    for st in sim.steps:
        if st.kind == "expand":
            k += 1
        elif st.kind not in ("vg", "rot"):
            break
    assert info.prefix_k == k
    assert 0.0 <= info.prefix_bytes_fp32 <= info.array_bytes_fp32
    if name == "dense":
        assert info.prefix_k == 20 and info.prefix_bytes_fp32 > 0.99 * info.array_bytes_fp32 - 6e7


def _per_shot_cost(info):
    """The compiler's selection cost: unfused traversal bytes per shot, less a
    shared prefix of at least 6 axes plus one copy of its vector."""
    b = info.array_bytes_fp32
    if info.prefix_ops > 0 and info.prefix_k >= 6:
        b -= info.prefix_bytes_fp32 - 8.0 * 2 ** info.prefix_k
    return b


@pytest.mark.parametrize("name", ["dense20", "dense12", "coherent_d3r1", "coherent_d3r3", "lowmagic", "tiny",
                                  "random"])
def test_pass_search_never_costs_more(nc, name):
    """nc_compile keeps the cheapest of the pass subsets it tries, so the
    kept program costs at most what the plain program (every HIR pass off)
    and the all-passes program would cost; compiling twice gives the same
    bytes."""
    text = {"dense20": lambda: gc.dense_random(seed=3, n=20, layers=40),
            "dense12": lambda: gc.dense_random(seed=3, n=20, layers=12),
            "coherent_d3r1": lambda: gc.surface_code_memory(d=3, rounds=1, p=1e-3, theta=0.02),
            "coherent_d3r3": lambda: gc.surface_code_memory(d=3, rounds=3, p=1e-3, theta=0.02),
            "lowmagic": gc.low_magic_gadgets, "tiny": lambda: gc.tiny_random(seed=1),
            "random": lambda: gc.random_small(77, n=6, n_ops=100, t_frac=0.3)}[name]()
    kept = nc.compile(text)
    plain = nc.compile(text, peephole=False)
    assert _per_shot_cost(kept.info) <= _per_shot_cost(plain.info) + 1e-6
    assert kept.info.k_max <= plain.info.k_max or _per_shot_cost(kept.info) < _per_shot_cost(plain.info)
    assert nc.compile(text).serialize() == kept.serialize()
