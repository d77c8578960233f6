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

``replica``: the paper's two-dimensional reactor (Sec. 2.1, Sec. 3, Table 1)
as a one-cell-thick 500 x 1 x 250 box: disk-grown ingots of h = 200 and
w = 6, 10, 20, 30 across the flow (perpendicular) for p = 0.35 .. 0.65, the
w = 10 ingot along the flow (parallel), and w = 10 ingots of other lengths h
at p = 0.45 (the scaling eta ~ h/H of Sec. 3); velocity inlet U_in = 0.08 with
rho_C = 0.8, rho_R = 0.2, the barycentric velocity, tau = 4, pS_R = 0.95,
pS_P = 0. All simulations advance together in batched launches. Reports eta
(Eq. eff) at two times, the product flux Phi_P(z) (Eq. Phi_P) for w/h = 0.1
and at z = 150 for every w (Fig. 5), the share of the reaction in the first
three ingot layers facing the flow, and the paper's trends (Fig. 6 and the
orientation study) as checks.

The replica also reports Fig. 3 as numbers (replica_fig3): after 10,000
steps, how deep the reactant gets into the w = 10 ingot and through which
faces the product leaves it, in both orientations.

``leveque``: the Appendix's validation channel (150 lattice units of
reactive plate, L_y = 50, Pe = 253, p = 1, body-force-driven carrier). The
per-node wall hits of the developed flow give the reactive plate's
concentration gradient, compared with Lévêque's solution. Reports both
profiles and the mean absolute error.

``serving``: the request stream (256 requests, Poisson arrivals at 20 per
second, cubic boxes of side 48..192, porosity U[0.55, 0.75], correlation
length U[4, 16], Da log-uniform in [1e-3, 10]) through the continuous-batching
loop of ``serving``, once in FP16 and once in FP32 storage with fluid-only
addressing. A request is steady when eta changes by less than 1e-8
(relative) over 1000 steps, else it stops at the step cap (20,000). Reports
p50/p99 time-to-steady (arrival to retirement), the service time, MLUPS,
the largest batch, and how many requests converged or were capped.

Usage::

    python -m paper_1607_02874_gb300.studies precision [--steps 10000]
    python -m paper_1607_02874_gb300.studies da_sweep [--cap 20000]
    python -m paper_1607_02874_gb300.studies replica [--steps 30000]
    python -m paper_1607_02874_gb300.studies leveque [--steps 30000]
    python -m paper_1607_02874_gb300.studies serving [--cap 20000] [--requests 256] [--storages fp16,fp32]
"""
from __future__ import annotations

import argparse
import json
import math
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


# D3Q19 directions of the library (include/lbm.h): x and z components
_CX = np.array([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0])
_CZ = np.array([0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1])


def replica_fig3(steps=10000, save=None):
    """Fig. 3 of the paper as numbers: the w = 10 ingot at p = 0.45 after
    `steps` steps, perpendicular and parallel. Reports the reactant's mean
    density per ingot layer from the face that meets the flow (how deep it
    gets), and where the product leaves the ingot's rectangle: the net
    product flux (sum over the fluid cells just outside each face of the
    component of j_P = sum_i c_i f_P,i pointing away from the ingot)
    through the face meeting the flow, the opposite face and the two sides.
    With save, the rho_R and rho_P fields go to an .npz file."""
    import torch

    R = workloads.REPLICA
    nx, nz, w, p = R["nx"], R["nz"], 10, 0.45
    stream = torch.cuda.Stream()
    out, arrays = {}, {}
    for orient in ("perpendicular", "parallel"):
        box = workloads.ingot_box(nx, nz, R["h"], w, orient)
        mask = workloads.disk_ingot(nx, nz, box, porosity=R["porosity"], diameter=R["pore_diameter"],
                                    seed=R["seed"] + w)
        g = lbm.Geometry(nx, 1, nz, slab=(box[2], box[3]), mask=mask, stream=stream)
        s = lbm.Simulation(g, tau=R["tau"], rho_in=R["rho_C"], rho_out=R["rho_C"], c_in=R["c_in"], p=p,
                           pS_R=R["pS_R"], pS_P=R["pS_P"], n_species=2, layout=lbm.LAYOUT_FLUID, u_in=R["u_in"],
                           velocity=lbm.VELOCITY_BARYCENTRIC, stream=stream)
        s.step(steps)
        rho_R = s.field("rho_R").reshape(nz, nx).astype(np.float64)
        rho_P = s.field("rho_P").reshape(nz, nx).astype(np.float64)
        f = s.populations()[2].astype(np.float64)  # product populations [19][n]
        jx = (_CX[:, None] * f).sum(0).reshape(nz, nx)
        jz = (_CZ[:, None] * f).sum(0).reshape(nz, nx)
        x0, x1, z0, z1 = box
        m = mask.reshape(nz, nx)
        # the face that meets the flow is z = z0 in both orientations (the
        # flow runs along +z)
        faces = {"upstream": float(-jz[z0 - 1, x0:x1].sum()), "downstream": float(jz[z1, x0:x1].sum()),
                 "sides": float(-jx[z0:z1, x0 - 1].sum() + jx[z0:z1, x1].sum())}
        tot = sum(faces.values())
        depth = []
        for k in range(min(z1 - z0, 12)):
            pore = m[z0 + k, x0:x1] == 0
            depth.append(float(rho_R[z0 + k, x0:x1][pore].mean()) if pore.any() else 0.0)
        o = s.observables(profiles=False)
        out[orient] = {"box": list(box), "product_out": faces,
                       "product_out_share": {k: v / tot for k, v in faces.items()} if tot > 0 else None,
                       "rhoR_by_layer_from_upstream_face": depth, "rhoR_upstream_of_ingot": float(
                           rho_R[z0 - 3, x0:x1].mean()), "eta": o["eta"], "reacted": o["reacted"]}
        arrays[orient + "_rho_R"], arrays[orient + "_rho_P"] = rho_R.astype(np.float32), rho_P.astype(np.float32)
        s.close()
    if save:
        np.savez_compressed(save, **arrays)
    return {"workload": R["name"], "steps": steps, "w": w, "p": p, "runs": out}


def replica(steps=None, storage=lbm.FP32):
    import torch

    R = workloads.REPLICA
    steps = steps or R["steps"]
    nx, nz, h = R["nx"], R["nz"], R["h"]
    stream = torch.cuda.Stream()
    runs = [("perpendicular", w, p, h) for w in R["w_list"] for p in R["p_list"]]
    runs += [("parallel", 10, p, h) for p in R["p_list"]]
    # the efficiency scaling law eta = (h/H) phi(...): other ingot lengths at
    # w = 10, p = 0.45
    runs += [("perpendicular", 10, 0.45, hh) for hh in R["h_list"] if hh != h]
    geoms, sims = {}, []
    for orient, w, p, hh in runs:
        if (orient, w, hh) not in geoms:
            box = workloads.ingot_box(nx, nz, hh, w, orient)
            mask = workloads.disk_ingot(nx, nz, box, porosity=R["porosity"], diameter=R["pore_diameter"],
                                        seed=R["seed"] + w)
            g = lbm.Geometry(nx, 1, nz, slab=(box[2], box[3]), mask=mask, stream=stream)
            sub = mask.reshape(nz, nx)[box[2]:box[3], box[0]:box[1]]
            geoms[(orient, w, hh)] = (g, box, float(1.0 - sub.mean()))
        g = geoms[(orient, w, hh)][0]
        sims.append(lbm.Simulation(g, tau=R["tau"], rho_in=R["rho_C"], rho_out=R["rho_C"], c_in=R["c_in"], p=p,
                                   pS_R=R["pS_R"], pS_P=R["pS_P"], n_species=2, storage=storage,
                                   layout=lbm.LAYOUT_FLUID, u_in=R["u_in"], velocity=lbm.VELOCITY_BARYCENTRIC,
                                   stream=stream))
    cells = sum(s.geom.info()["n_fluid"] for s in sims)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    first = steps * 2 // 3
    ev0.record(stream)
    for k in range(0, first, 1000):
        lbm.step_batch(sims, min(1000, first - k), stream=stream)
    ev1.record(stream)
    stream.synchronize()
    secs = ev0.elapsed_time(ev1) / 1e3
    eta_mid = [s.observables(profiles=False)["eta"] for s in sims]
    ev0.record(stream)
    for k in range(first, steps, 1000):
        lbm.step_batch(sims, min(1000, steps - k), stream=stream)
    ev1.record(stream)
    stream.synchronize()
    secs += ev0.elapsed_time(ev1) / 1e3
    nu = (R["tau"] - 0.5) / 3.0  # = D: the species share tau
    cs = 3.0 ** -0.5
    out = {"workload": R["name"], "steps": steps, "sims": len(sims), "fluid_cells": cells,
           "MLUPS": round(cells * steps / secs / 1e6, 1), "runs": [],
           # Sec. 2.3 with this reading's tau: Re = U_in h / nu, Pe = U_in h / D,
           # Kn = cs (tau - 1/2) / delta with the 3-unit pore diameter, Ma = U_in / cs
           "dimensionless": {"Re": R["u_in"] * h / nu, "Pe": R["u_in"] * h / nu,
                             "Kn": cs * (R["tau"] - 0.5) / R["pore_diameter"], "Ma": R["u_in"] / cs}}
    for (orient, w, p, hh), s, em in zip(runs, sims, eta_mid):
        o = s.observables(profiles=True)
        g, box, phi = geoms[(orient, w, hh)]
        react = o["react_z"]
        if orient == "perpendicular":
            front = react[box[2]:box[2] + 3].sum() / max(react.sum(), 1e-300)
        else:
            front = None
        r = {"orientation": orient, "w": w, "h": hh, "w_over_h": w / hh, "p": p, "porosity": round(phi, 4),
             "eta": o["eta"], f"eta_at_{first}": em, "phiP_z150": o["phiP_z"][150], "front3_reaction_share": front,
             "conversion_X": _conversion(o)}
        if orient == "perpendicular" and w == 20 and hh == h:
            r["phiP_z"] = [float(v) for v in o["phiP_z"]]
        out["runs"].append(r)
        s.close()
    # the paper's trends (Fig. 6, orientation study)
    perp = {(r["w"], r["p"]): r["eta"] for r in out["runs"] if r["orientation"] == "perpendicular" and r["h"] == h}
    par = {r["p"]: r["eta"] for r in out["runs"] if r["orientation"] == "parallel"}
    by_h = {r["h"]: r["eta"] for r in out["runs"] if r["orientation"] == "perpendicular" and r["w"] == 10
            and r["p"] == 0.45}
    ws, ps = R["w_list"], R["p_list"]
    intercepts = {}
    for p in ps:
        y = np.array([perp[(w, p)] for w in ws])
        slope, icpt = np.polyfit(np.array(ws) / h, y, 1)
        intercepts[p] = float(icpt)
    out["trends"] = {
        "eta_increases_with_p_at_every_w": all(perp[(w, a)] < perp[(w, b)] for w in ws for a, b in zip(ps, ps[1:])),
        "eta_nonzero_as_w_over_h_to_0": {str(p): v for p, v in intercepts.items()},
        "eta_w30_over_w6": {str(p): perp[(30, p)] / perp[(6, p)] if perp[(6, p)] > 0 else None for p in ps},
        "parallel_below_perpendicular_w10": all(par[p] < perp[(10, p)] for p in ps),
        "eta_w10_p045": perp[(10, 0.45)],
        "eta_over_h_over_H_w10_p045": {str(hh): e / (hh / nx) for hh, e in sorted(by_h.items())},
        "paper_eta_w10_p045": 0.2,
    }
    return out


# nodes compared with Lévêque's solution: away from the leading-edge
# singularity (first 5) and from the outlet end (last 20), where the open
# outlet and the gap in the plates (the inlet/outlet planes and their
# neighbours must be fluid) disturb the profile
LEVEQUE_WINDOW = (5, workloads.LEVEQUE["L"] - 20)


def leveque_gradients(site_map):
    """(G, G_L) per node of the reactive plate, from the upstream end: G the
    dimensionless wall gradient d(c/c_in)/d(y/L_y) = q L_y / (D c_in), q the
    reactant reaching the node per step (p = pS_R = 1: the site map); G_L
    Lévêque's (9^(1/3) Gamma(4/3))^-1 (4 Pe / (x / L_y))^(1/3) at the node's
    distance x = k + 1/2 from the plate's leading edge."""
    c = workloads.LEVEQUE
    D = (c["tau_s"] - 0.5) / 3.0
    q = np.asarray(site_map, np.float64)[: c["L"]]
    G = q * c["L_y"] / D
    x = np.arange(c["L"]) + 0.5
    GL = (4.0 * c["Pe"] * c["L_y"] / x) ** (1.0 / 3.0) / (9.0 ** (1.0 / 3.0) * math.gamma(4.0 / 3.0))
    return G, GL


def leveque(steps=None):
    import torch

    c = workloads.LEVEQUE
    steps = steps or c["steps"]
    nx, nz = c["L_y"] + 2, c["L"] + 4
    stream = torch.cuda.Stream()
    g = lbm.Geometry(nx, 1, nz, slab=(2, nz - 2), mask=workloads.leveque_mask(), stream=stream)
    s = lbm.Simulation(g, n_species=2, tau=c["tau"], tau_s=c["tau_s"], rho_in=1.0, rho_out=1.0, c_in=1.0, p=1.0,
                       pS_R=1.0, pS_P=0.0, g_z=workloads.leveque_force(), layout=lbm.LAYOUT_FLUID, stream=stream)
    secs = _timed_steps(s, torch, steps)
    G, GL = leveque_gradients(s.observables(site_map=True)["site_map"])
    uz = s.field("uz").reshape(nz, nx)[nz // 2, 1:nx - 1]
    rel = np.abs(G - GL) / GL
    a, b = LEVEQUE_WINDOW
    out = {"workload": c["name"], "steps": steps, "MLUPS": round(g.info()["n_fluid"] * steps / secs / 1e6, 1),
           "g_z": workloads.leveque_force(), "u_max": float(uz.max()),
           "u_max_expected": c["Pe"] * (c["tau_s"] - 0.5) / 3.0 / c["L_y"], "window": [a, b],
           "mae_window": float(rel[a:b].mean()), "max_rel_window": float(rel[a:b].max()),
           "mae_all_nodes": float(rel.mean()), "paper_mae": 0.04,
           "x": [k + 0.5 for k in range(c["L"])], "G": [float(v) for v in G], "G_leveque": [float(v) for v in GL]}
    s.close()
    return out


def serving(cap=20000, n_requests=256, storages=("fp16", "fp32"), check=1000, tol=1e-8, budget_frac=0.8):
    import torch

    from .serving import LbmBackend, ServingLoop, requests_from_workload

    reqs = requests_from_workload(workloads.serving_requests(n=n_requests))
    out = {"requests": n_requests, "rate_per_s": 20.0, "cap": cap, "check_every": check, "tol": tol}
    for name in storages:
        storage = {"fp32": lbm.FP32, "fp16": lbm.FP16_DEV, "bf16": lbm.BF16_DEV}[name]
        torch.cuda.empty_cache()
        budget = int(budget_frac * torch.cuda.mem_get_info()[0])
        be = LbmBackend(storage=storage, layout=lbm.LAYOUT_FLUID)
        loop = ServingLoop(be, budget_bytes=budget, steps_per_tick=100, check_every=check, max_steps=cap, tol=tol,
                           workers=4)
        res = loop.run(reqs)
        recs = res.pop("records")
        res["budget_bytes"] = budget
        res["max_batch"] = max((e[2] for e in loop.trace if e[1] == "tick"), default=0)
        ok = [r for r in recs if r["status"] in ("converged", "capped")]
        steps = np.array([r["steps"] for r in ok], float)
        res["steps_p50"] = float(np.median(steps)) if steps.size else float("nan")
        res["eta"] = {str(r["id"]): r["eta"] for r in ok}
        out[name] = res
        torch.cuda.synchronize()
    if "fp16" in out and "fp32" in out:
        a, b = out["fp16"]["eta"], out["fp32"]["eta"]
        rel = [abs(a[k] - b[k]) / abs(b[k]) for k in a if k in b and b[k] > 0]
        out["eta_rel_fp16_vs_fp32"] = {"median": float(np.median(rel)), "max": float(np.max(rel))} if rel else None
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["precision", "da_sweep", "replica", "leveque", "serving"])
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--cap", type=int, default=20000)
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--storages", default="fp16,fp32", help="serving: storages to run, comma-separated")
    ap.add_argument("--save", default=None, help="replica: write the Fig. 3 fields to this .npz file")
    args = ap.parse_args()
    t0 = time.time()
    if args.study == "precision":
        res = precision(args.steps or 10000)
    elif args.study == "da_sweep":
        res = da_sweep(args.cap)
    elif args.study == "replica":
        res = replica(args.steps)
        res["fig3"] = replica_fig3(save=args.save)
    elif args.study == "serving":
        res = serving(args.cap, args.requests, storages=tuple(args.storages.split(",")))
    else:
        res = leveque(args.steps)
    res["wall_s"] = round(time.time() - t0, 1)
    print(json.dumps(res, default=float))


if __name__ == "__main__":
    main()
