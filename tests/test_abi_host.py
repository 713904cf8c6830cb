"""CPU tests of the C-ABI library: it loads, exports every symbol declared in
include/*.h, and its host-only entry points agree with the oracle.  No GPU
call is made here; a context cannot be created without a device and must say
so with DG_ECUDA rather than fall back to the CPU."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_2508_17917_gb300 import build as dgbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dg():
    dgbuild.build()
    import paper_2508_17917_gb300 as dg
    dg.lib()
    return dg


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(dg):
    names = declared_functions()
    assert len(names) >= 28
    out = subprocess.run(["nm", "-D", "--defined-only", dg.library_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(dg_[a-z0-9_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert set(names) == set(dg.EXPORTED)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_reference_operators_match_oracle(dg, p):
    lib_ops = dg.dg_reference_operators(p)
    o = oracle.refelem.operators(p)
    assert np.abs(lib_ops["r"] - o["r"]).max() < 1e-14
    assert np.abs(lib_ops["s"] - o["s"]).max() < 1e-14
    assert np.abs(lib_ops["Dr"] - o["Dr"]).max() < 1e-12
    assert np.abs(lib_ops["Ds"] - o["Ds"]).max() < 1e-12
    # LIFT columns are ordered counter-clockwise per face in the library;
    # compare through the face node identity of each column
    Nfp = p + 1
    for f in range(3):
        lf = lib_ops["Fmask"][f]
        of = list(o["Fmask"][f])
        assert sorted(lf) == sorted(of)
        for i in range(Nfp):
            j = of.index(lf[i])
            assert np.abs(lib_ops["LIFT"][:, f * Nfp + i] - o["LIFT"][:, f * Nfp + j]).max() < 1e-12


def test_rigid_step_matches_oracle(dg):
    rng = np.random.default_rng(0)
    for _ in range(50):
        coeff = (rng.uniform(0.5, 2), rng.uniform(0, 0.5), rng.uniform(1, 50))
        st = rng.normal(size=3)
        F, dt = rng.normal(), rng.uniform(1e-4, 0.1)
        a, va = dg.dg_rigid_step(coeff, F, dt, st)
        b, vb = oracle.newmark_step(coeff, F, dt, st)
        assert np.allclose(a, b, rtol=1e-13, atol=1e-15) and abs(va - vb) <= 1e-13 * max(1, abs(vb))


def test_rigid_step_rejects_bad_input(dg):
    with pytest.raises(dg.DGError):
        dg.dg_rigid_step((1.0, 0.0, 1.0), 0.0, 0.0, np.zeros(3))


def test_create_rejects_bad_params(dg):
    bad = dg.DgParams(9, 0, 1.4, 0.72, 1e-3, 0.0, 0.01, 1, 1, 0, 1, 1)
    with pytest.raises(dg.DGError) as e:
        dg.dg_create(bad)
    assert e.value.status == -1
    for theta in (1.5, -1.01, float("nan")):
        bad_theta = dg.DgParams(2, 0, 1.4, 0.72, 1e-3, theta, 0.01, 1, 1, 0, 1, 1)
        with pytest.raises(dg.DGError) as e:
            dg.dg_create(bad_theta)
        assert e.value.status == -1


def test_no_cpu_fallback_without_gpu(dg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ok = dg.DgParams(2, 0, 1.4, 0.72, 1e-3, 0.0, 0.01, 1, 1, 0, 1, 1)
    with pytest.raises(dg.DGError) as e:
        dg.dg_create(ok)
    assert e.value.status == -3


def test_batch_create_rejects_bad_input_without_gpu(dg):
    import dg_inputs
    m = dg_inputs.ogrid_cylinder(12, 3, 0.5, 3.0, seed=0)
    ok = dict(mesh=m, p=3, mu=0.01, M_r=1.0, C_r=0.01, K_r=1.6, mass=7.85)
    common = dict(p_inf=17.857142857142858)
    for bad in (dict(ok, p=7), dict(ok, mass=0.0), dict(ok, mu=-1.0)):
        with pytest.raises(dg.DGError) as e:
            dg.BatchSolver([bad], **common)
        assert e.value.status == -1
    import torch
    if not torch.cuda.is_available():
        with pytest.raises(dg.DGError) as e:
            dg.BatchSolver([ok], **common)
        assert e.value.status == -3 and "device" in str(e.value)
