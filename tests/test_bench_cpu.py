"""Host logic of bench.py on the CPU: the reference arm (the oracle on a bounded sample)
prints one JSON line with the contract's keys, for the 2D and the 3D set-up; the byte
models and the uneven-batch sizes are what their docstrings state."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _reference_line(*extra):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", *extra], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


@pytest.mark.parametrize("extra", [("--cpu-n", "64"),
                                   ("--dim", "3", "--cpu-cells3", "24,24,16", "--pad3", "4", "--cycle", "W")])
def test_reference_arm_json_line(extra):
    d = _reference_line(*extra)
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "iterations"):
        assert key in d, key
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["iterations"] >= 1
    assert "workload" in d["config"]


def test_byte_models():
    sys.path.insert(0, ROOT)
    import bench

    info = {"coarse_entries": 1000, "nodes2": 100, "radius2": 2, "nodes3": 10}
    m = bench.kernel_model(info, its=18, restart=10, n1=400, n3=10, dim=2, elem=8)
    assert m["coarse"]["bytes"] == 16.0 * 1000 + 6 * 16.0 * 10
    # level-2 row operation averaged over a (1,1) visit: two of three read all 25 planes
    assert m["stencil"]["bytes"] == pytest.approx(8 * (25 * 2 / 3 + 3) * 100)
    # mean Arnoldi basis size over 18 iterations with restart 10: (1+...+10 + 1+...+8) / 18
    nv = (55 + 36) / 18
    assert m["arnoldi_norm"]["bytes"] == pytest.approx((32 + 16 * nv) * 400)
    m3 = bench.kernel_model(info, its=1, restart=10, n1=400, n3=10, dim=3, elem=16)
    assert m3["stencil"]["bytes"] == pytest.approx(16 * (125 * 2 / 3 + 3) * 100)


def test_uneven_sizes_and_3d_workload():
    sys.path.insert(0, ROOT)
    import bench

    ns = type("A", (), {})()
    ns.uneven = 16
    sizes = bench.uneven_sizes(ns)
    assert sizes == sorted(sizes) and len(sizes) == 16
    assert all(256 <= s <= 1536 and s % 4 == 0 for s in sizes)
    assert sizes == bench.uneven_sizes(ns)   # seeded
    ns3 = type("A", (), {})()
    ns3.cells3, ns3.pad3, ns3.ppw, ns3.jacobi = "24,16,12", 4, 12, None
    wl = bench.workload3(ns3)
    assert wl["kappa2"].shape == (13, 17, 25)
    assert wl["widths6"] == [4, 4, 4, 4, 0, 4] and wl["owidths"] == [(4, 4), (4, 4), (0, 4)]
    assert wl["q"][0, 8, 12] != 0 and np.count_nonzero(wl["q"]) == 1   # centre of the top face
    assert bench.n_nodes(wl) == 13 * 17 * 25


def test_cpu_baseline_repeats_solves_to_its_budget(monkeypatch):
    """The GPU arm's cpu_baseline repeats the sample solve until --cpu-seconds of solve
    time are spent and reports nodes x solves / total time."""
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setattr(bench, "oracle_solve", lambda smp, args: (0.3, 8))
    args = type("A", (), {"cpu_seconds": 10.0})()
    smp = dict(solver="fgmres", cells="576x576", nodes=332929, n=512)
    c = bench.cpu_baseline(smp, args)
    assert c["value"] == pytest.approx(332929 * 34 / 1e6 / (0.3 * 34))
    assert c["sample"].count("34 full FGMRES solves") == 1 and c["kind"] == "oracle"
    args.cpu_seconds = 0.0
    assert "full FGMRES solve to" in bench.cpu_baseline(smp, args)["sample"]
