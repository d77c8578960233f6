"""The bounds-checked build (-DLBM_CHECKED) over every kernel variant, on the
GPU. compute-sanitizer is not available here; this build tests every
population, wall-hit accumulator, geometry-index, node-table and
plane-cache access of the step and state-reading kernels against its
buffer's extent, and records the first violation.

A child process loads the checked library (LBM_LIBRARY) and runs small
cases of every path: default, random matrix, barycentric, channel (inert
solid, body force, species tau), species bounce-back, velocity inlet, both
addressings and parities, both batched modes, observables, site map, field
and population export. No access may fall outside its buffer, and the
results must equal the default build's to FP32 rounding (the checked build
optimises device code less, so the order of a few roundings may differ),
so the checks change nothing else.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_cases(lbm):
    """Every variant on a small case; returns {name: array}."""
    out = {}
    c = workloads.ragged_case()

    def geom(mask=None, bc=lbm.BC_PRESSURE):
        return lbm.Geometry(c["nx"], c["ny"], c["nz"], slab=c["slab"], porosity=c["porosity"],
                            corr_len=c["corr_len"], seed=c["seed"], mask=mask, bc=bc)

    g = geom()
    m = g.export()["mask"]
    z = np.arange(m.size) // (c["nx"] * c["ny"])
    mixed = np.where((m == 1) & (z >= 25), 2, m).astype(np.uint8)
    gm = geom(mask=mixed)
    cases = {
        "default-dense": (g, dict(layout=lbm.LAYOUT_DENSE)),
        "default-fluid-fp16": (g, dict(layout=lbm.LAYOUT_FLUID, storage=lbm.FP16_DEV)),
        "random-bf16": (g, dict(layout=lbm.LAYOUT_FLUID, storage=lbm.BF16_DEV, sputter=lbm.SPUTTER_RANDOM,
                                sputter_seed=3)),
        "bary": (g, dict(layout=lbm.LAYOUT_FLUID, velocity=lbm.VELOCITY_BARYCENTRIC, c_in=0.05)),
        "bary-random-dense": (g, dict(layout=lbm.LAYOUT_DENSE, velocity=lbm.VELOCITY_BARYCENTRIC, c_in=0.05,
                                      sputter=lbm.SPUTTER_RANDOM, sputter_seed=4)),
        "channel-inert": (gm, dict(layout=lbm.LAYOUT_FLUID, tau_s=0.6)),
        "channel-inert-random-dense": (gm, dict(layout=lbm.LAYOUT_DENSE, sputter=lbm.SPUTTER_RANDOM, sputter_seed=5)),
        "bounceback": (g, dict(layout=lbm.LAYOUT_FLUID, sputter=lbm.SPUTTER_BOUNCEBACK, desorb=True)),
        "velocity-inlet-force": (g, dict(layout=lbm.LAYOUT_FLUID, u_in=0.02, g_z=1e-5)),
    }
    for name, (gg, kw) in cases.items():
        s = lbm.Simulation(gg, n_species=2, p=0.45, pS_P=0.1, deterministic=True, **kw)
        s.step(37)
        o = s.observables(site_map=True)
        out[name + "/rho_R"] = s.field("rho_R")
        out[name + "/uz"] = s.field("uz")
        out[name + "/site"] = o["site_map"]
        out[name + "/pops"] = s.populations()
        out[name + "/scal"] = np.array([o[k] for k in ("M_C", "M_R", "M_P", "hits_R", "in_R", "eta")])
        s.close()
    for mode in (0, 1):
        sims = [lbm.Simulation(gg, n_species=2, p=0.3, deterministic=True, layout=lbm.LAYOUT_FLUID, **kw)
                for gg, kw in ((g, {}), (gm, {}), (g, dict(sputter=lbm.SPUTTER_RANDOM)))]
        sims[1].step(1)
        lbm.step_batch(sims, 24, mode=mode)
        for k, s in enumerate(sims):
            out[f"batch{mode}-{k}/rho_P"] = s.field("rho_P")
            s.close()
    out["status"] = np.array([lbm.check_status()], np.uint64) if lbm.LIB_PATH.endswith(
        os.path.join("_lib_checked", "liblbm.so")) else np.zeros(1, np.uint64)
    return out


def child_main(path):
    from paper_1607_02874_gb300 import lbm

    np.savez(path, **run_cases(lbm))


def test_checked_build_finds_nothing_and_changes_nothing(tmp_path):
    from paper_1607_02874_gb300 import build, lbm

    lib = build.build(checked=True)
    out = tmp_path / "checked.npz"
    env = dict(os.environ, LBM_LIBRARY=lib)
    code = f"import sys; sys.path.insert(0, {ROOT!r}); import tests.test_gpu_checked as t; t.child_main({str(out)!r})"
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    got = np.load(out)
    word = int(got["status"][0])
    assert word == 0, f"out-of-bounds access: kind {word >> 56}, element {word & ((1 << 56) - 1)}"
    ref = run_cases(lbm)
    with pytest.raises(lbm.LbmError):
        lbm.check_status()  # the default build has no checks
    for k, v in ref.items():
        if k == "status":
            continue
        v = np.asarray(v, np.float64)
        # 16-bit storage rounds stochastically from the FP32 value: a last-bit
        # FP32 difference may flip one rounding, one unit of the format
        tol = 5e-2 if "bf16" in k else (4e-3 if "fp16" in k else 1e-5)
        np.testing.assert_allclose(got[k], v, rtol=tol, atol=tol * max(np.abs(v).max(), 1e-30), err_msg=k)
