"""bench.py helpers on CPU: workload names and sizes, the record bytes of
the roofline, the committed traffic figure, and the reference arm (the
oracle on the host cores) producing its JSON line."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_workloads_and_names():
    for name in ("surface", "tiny", "dense", "lowmagic", "coherent"):
        wname, text, shots, ps = bench.workload(name)
        assert wname and text and shots > 0 and ps == (name == "lowmagic")

    class A:
        workload = "surface"
        stratum = None
    assert bench.workload_name(A) == "surface_code_d5_r25_p1e-3"
    A.stratum = 4
    assert bench.workload_name(A) == "surface_code_d5_r25_p1e-3_stratum4"


def test_record_bytes_of_the_surface_code():
    class I:
        n_meas, n_det, n_obs = 625, 600, 1
    assert bench.record_bytes_per_shot(I) == pytest.approx(1227 / 8)


def test_traffic_figure_is_per_shot():
    t = bench.ncu_traffic("surface_code_d5_r25_p1e-3")
    if t is not None:  # present while the kernel sources match the capture
        assert 153.4 <= t < 200


def test_reference_arm_prints_one_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--ref-budget", "0.5", "--workload", "tiny"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
