"""Parameter studies of the hot path on the GPU (JSON to stdout).

``precision``: the 256x256x512 sample (porosity 0.70, correlation length 14,
Da = 1, C+R+P) stepped in FP32, FP16 and BF16 deviation storage from the same
start. Reports MLUPS, the speed ratio to FP32, the field errors against the
FP32 run, and two conversion measures against the FP32 run:
- eta (Sec. 3, Eq. eff), which stays ~0 until product reaches the outlet;
- the flux conversion X = reacted R / inflowing R, which is meaningful from
  the first steps.

``da_sweep``: the 128x128x256 sample (porosity 0.60, correlation length 10,
C+R+P) for each Da, run until eta changes by less than 1e-8 (relative) over
1000 steps or to the step cap, in dense and fluid-only addressing. Reports eta,
X, p, the steps taken and MLUPS.

Usage::

    python -m paper_1607_02874_gb300.studies precision [--steps 10000]
    python -m paper_1607_02874_gb300.studies da_sweep [--cap 20000]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

from . import lbm  # noqa: E402

FIELDS = ("drho_C", "ux", "uy", "uz", "rho_R", "rho_P")


def _timed_steps(sim, torch, n, chunk=500):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(sim.stream)
    left = n
    while left > 0:
        k = min(chunk, left)
        sim.step(k)
        left -= k
    ev1.record(sim.stream)
    sim.stream.synchronize()
    return ev0.elapsed_time(ev1) / 1e3


def _interior(geom, mask):
    plane = geom.nx * geom.ny
    z = np.arange(mask.size) // plane
    return (mask == 0) & (z > 0) & (z < geom.nz - 1)


def _conversion(o):
    return o["reacted"] / o["in_R"] if o["in_R"] > 0 else 0.0


def precision(steps=10000, storages=("fp32", "fp16", "bf16")):
    import torch

    cfg = workloads.CFG3
    codes = {"fp32": lbm.FP32, "fp16": lbm.FP16_DEV, "bf16": lbm.BF16_DEV}
    stream = torch.cuda.Stream()
    g = lbm.Geometry(cfg["nx"], cfg["ny"], cfg["nz"], slab=cfg["slab"], porosity=cfg["porosity"],
                     corr_len=cfg["corr_len"], seed=cfg["seed"], stream=stream)
    nf = g.info()["n_fluid"]
    sel = _interior(g, g.export()["mask"])
    runs = {}
    for st in storages:
        s = lbm.Simulation(g, tau=cfg["tau"], rho_in=cfg["rho_in"], rho_out=cfg["rho_out"], c_in=cfg["c_in"],
                           Da=cfg["Da"], n_species=2, storage=codes[st], layout=lbm.LAYOUT_FLUID, stream=stream)
        secs = _timed_steps(s, torch, steps)
        o = s.observables(profiles=False)
        runs[st] = {"MLUPS": nf * steps / secs / 1e6, "obs": o,
                    "fields": {k: s.field(k)[sel].astype(np.float64) for k in FIELDS}}
        s.close()
    ref = runs["fp32"]
    out = {"workload": cfg["name"], "steps": steps, "n_fluid": nf, "p": ref["obs"]["p"], "results": {}}
    for st, r in runs.items():
        errs = {}
        for k in FIELDS:
            den = np.abs(ref["fields"][k]).max()
            errs[k] = float(np.abs(r["fields"][k] - ref["fields"][k]).max() / den) if den > 0 else 0.0
        X, X32 = _conversion(r["obs"]), _conversion(ref["obs"])
        out["results"][st] = {
            "MLUPS": round(r["MLUPS"], 1), "speedup_vs_fp32": round(r["MLUPS"] / ref["MLUPS"], 3),
            "eta": r["obs"]["eta"], "conversion_X": X,
            "eta_rel_err_vs_fp32": abs(r["obs"]["eta"] - ref["obs"]["eta"]) / abs(ref["obs"]["eta"])
            if ref["obs"]["eta"] else None,
            "X_rel_err_vs_fp32": abs(X - X32) / abs(X32) if X32 else None,
            "field_err_vs_fp32": errs,
            "M_R_rel_err_vs_fp32": abs(r["obs"]["M_R"] - ref["obs"]["M_R"]) / ref["obs"]["M_R"],
            "M_P_rel_err_vs_fp32": abs(r["obs"]["M_P"] - ref["obs"]["M_P"]) / max(ref["obs"]["M_P"], 1e-300),
        }
    return out


def da_sweep(cap=20000, check=1000, tol=1e-8, das=None, layouts=("dense", "fluid")):
    import torch

    cfg = workloads.CFG2
    das = das or cfg["Da_list"]
    codes = {"dense": lbm.LAYOUT_DENSE, "fluid": lbm.LAYOUT_FLUID}
    stream = torch.cuda.Stream()
    g = lbm.Geometry(cfg["nx"], cfg["ny"], cfg["nz"], slab=cfg["slab"], porosity=cfg["porosity"],
                     corr_len=cfg["corr_len"], seed=cfg["seed"], stream=stream)
    info = g.info()
    out = {"workload": cfg["name"], "n_fluid": info["n_fluid"], "delta": info["delta"], "cap": cap,
           "criterion": f"|eta(t) - eta(t-{check})| <= {tol} eta(t), eta > 0", "runs": []}
    for ly in layouts:
        for Da in das:
            s = lbm.Simulation(g, tau=cfg["tau"], rho_in=cfg["rho_in"], rho_out=cfg["rho_out"], c_in=cfg["c_in"],
                               Da=Da, n_species=2, storage=lbm.FP32, layout=codes[ly], stream=stream)
            prev, steps, secs, conv = None, 0, 0.0, False
            while steps < cap:
                secs += _timed_steps(s, torch, check)
                steps += check
                eta = s.observables_noalloc()["eta"]
                if prev is not None and eta > 0 and abs(eta - prev) <= tol * eta:
                    conv = True
                    break
                prev = eta
            o = s.observables(profiles=True)
            front = o["react_z"][cfg["slab"][0]:cfg["slab"][0] + 8].sum() / max(o["react_z"].sum(), 1e-300)
            out["runs"].append({
                "layout": ly, "Da": Da, "p": o["p"], "steps": steps, "converged": conv,
                "eta": o["eta"], "conversion_X": _conversion(o), "front8_reaction_share": front,
                "MLUPS": round(info["n_fluid"] * steps / secs / 1e6, 1),
            })
            s.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["precision", "da_sweep"])
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--cap", type=int, default=20000)
    args = ap.parse_args()
    t0 = time.time()
    res = precision(args.steps) if args.study == "precision" else da_sweep(args.cap)
    res["wall_s"] = round(time.time() - t0, 1)
    print(json.dumps(res, default=float))


if __name__ == "__main__":
    main()
