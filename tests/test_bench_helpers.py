"""CPU tests of bench.py's bookkeeping: the algorithmic bytes behind the
roofline fraction, and the rule that a recorded DRAM figure is reported only
while the kernel source it was measured on is unchanged (comments aside)."""
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_per_step():
    # 5 stages x (read K0 + write K0 + write K1 + read K1 except on stage 1),
    # 8 B each per DOF, plus the per-element records of every stage
    K, Np = 1000, bench.NP
    dof = 4 * K * Np
    expect = dof * 8 * (3 + 4 * 4) + 5 * K * bench.GEO_BYTES_MIXED
    assert bench.algorithmic_bytes_per_step(K, bench.GEO_BYTES_MIXED) == expect
    # per DOF-stage at p = 4, mixed path: 32 + 80/60 B on stages 2..5,
    # 24 + 80/60 B on stage 1, 31.73 B on average over a step
    per = bench.algorithmic_bytes_per_step(K, bench.GEO_BYTES_MIXED) / (5 * dof)
    assert abs(per - (152.0 / 5 + 80.0 / 60)) < 1e-12


def test_code_only_ignores_comments_and_spacing():
    a = "int f(int x) {  // doubles x\n    return 2 * x; /* twice\n x */ }\n"
    b = "int f(int x)\n{\n return 2 * x;\n}"
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(b.replace("2 *", "3 *"))


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    """A copy of the tensor-core kernel's sources and a traffic record whose
    hash matches them."""
    import json
    src = os.path.join(ROOT, "paper_2508_17917_gb300", "csrc")
    dst = tmp_path / "paper_2508_17917_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.KERNEL_FILES[3]:
        shutil.copy(os.path.join(src, f), dst / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_hash(3)
    rec = {"3": {"kernel_hash": h, "dram_bytes_per_dof_stage": 40.25}}
    (tmp_path / "profiles" / "stage_kernel_traffic.json").write_text(json.dumps(rec))
    return dst


def test_recorded_traffic_follows_the_kernel_source(fake_root):
    assert bench.recorded_traffic(3) == 40.25
    f = fake_root / "dg_stage_tc.cuh"
    # a comment edit keeps the figure
    f.write_text(f.read_text() + "\n// a note\n")
    assert bench.recorded_traffic(3) == 40.25
    # a code edit drops it
    f.write_text(f.read_text() + "\nstatic const int unused_constant = 1;\n")
    assert bench.recorded_traffic(3) is None


def test_record_traffic_from_ncu_csv(fake_root, tmp_path):
    """An ncu raw-page CSV (header, units row, one row per launch) becomes a
    record keyed by the kernel hash; units are honoured."""
    import argparse
    csv = tmp_path / "raw.csv"
    csv.write_text(
        '"ID","Kernel Name","dram__bytes_read.sum","dram__bytes_write.sum"\n'
        '"","","Mbyte","Gbyte"\n'
        '"0","void dg::make_shadow_kernel<4>(...)","1.0","1.0"\n'
        '"1","void dg::stage_tc_kernel<4, false, false, false>(dg::StageParams, dg::Phys<float>)",'
        '"600.5","0.75"\n')
    assert bench.ncu_dram_bytes(str(csv), "stage_tc_kernel") == [600.5e6 + 0.75e9]
    args = argparse.Namespace(variant=3, record_traffic=str(csv), record_k=1000)
    bench.record_traffic(args)
    per = (600.5e6 + 0.75e9) / (4 * 1000 * bench.NP)
    assert abs(bench.recorded_traffic(3) - per) < 1e-9 * per


def test_algorithmic_flops_per_dof_stage():
    # by phase at p = 4 (per element): gradient 3960, volume flux 1440,
    # divergence 3600, faces 3750, lift 1800, update 240 over 60 DOFs
    assert abs(bench.algorithmic_flops_per_dof_stage(4) - 14790 / 60) < 1e-12


def test_recorded_traffic_without_a_record(fake_root):
    os.remove(os.path.join(bench.ROOT, "profiles", "stage_kernel_traffic.json"))
    assert bench.recorded_traffic(3) is None
    assert bench.recorded_traffic(7) is None


def test_strouhal_from_zero_crossings():
    import numpy as np
    t = np.linspace(0.0, 40.0, 8001)
    cl = 0.3 * np.sin(2 * np.pi * 0.165 * t + 0.4) + 0.02
    assert abs(bench.strouhal(t, cl) - 0.165) < 1e-6
    # fewer than three crossings: no frequency
    assert bench.strouhal(t[:600], cl[:600]) is None
