#!/usr/bin/env python
"""Benchmark: fused reactive LB step on the large synthetic np-Au sample.

One "step" = one time step of the whole hot path (collision of carrier,
reactant and product, streaming, bounce-back, catalytic sputtering,
inlet/outlet planes, wall-hit bookkeeping) over every fluid cell: four
launches (the catalytic nodes' emission, the fused collide-stream kernel
over the warps away from the inlet/outlet planes, the one over the rest,
the nodes' wall hits), five on odd steps, whose fast kernel takes the
all-fluid region warps in a launch of their own. After the warm-up, --windows windows
of --steps steps are timed; the line reports the median window.

Prints one JSON line (rank 0). With --impl reference it times the FP64 CPU
oracle instead, on a bounded sub-box of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "fluid+species MLUPS and % HBM roofline (FP32 vs FP16-storage); serving p50/p99 latency"
STORAGES = {"fp32": 0, "fp16": 1, "bf16": 2}
LAYOUTS = {"auto": 0, "dense": 1, "fluid": 2}
Q = 19
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100, help="steps per timed window")
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--windows", type=int, default=5, help="timed windows of --steps steps each")
    ap.add_argument("--c-init", type=float, default=1.0,
                    help="initial reactant density in the fluid (1.0: the catalytic boundary is live from the "
                         "first step; 0: the paper's start with no reactant inside)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=workloads.CFG5["name"], choices=sorted(workloads.CONFIGS))
    ap.add_argument("--storage", default=None, choices=sorted(STORAGES))
    ap.add_argument("--layout", default=None, choices=sorted(LAYOUTS))
    ap.add_argument("--no-companion", action="store_true", help="skip the FP32 companion measurement")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=24,
                    help="requests of the serving stream to run (0 skips the serving measurement)")
    ap.add_argument("--serving-max-steps", type=int, default=2000)
    ap.add_argument("--cpu-child", default=None, help=argparse.SUPPRESS)
    return ap.parse_args()


def default_storage_layout(cfg):
    if cfg is workloads.CFG5:
        return "fp16", "fluid"
    return "fp32", "auto"


# --------------------------------------------------------------------------
# CPU side: the oracle on a bounded sub-box (spawned child process so that
# its OpenMP pool starts clean and no CUDA context is forked)
# --------------------------------------------------------------------------
def cpu_sample(cfg):
    """Sub-box of the workload: same porosity, correlation length, seed,
    species and boundary types, 64 x 64 x 128 with the slab covering the
    same fraction of z."""
    nz = 128
    frac0, frac1 = cfg["slab"][0] / cfg["nz"], cfg["slab"][1] / cfg["nz"]
    z0 = max(2, int(round(frac0 * nz)))
    z1 = min(nz - 2, int(round(frac1 * nz)))
    return dict(nx=64, ny=64, nz=nz, slab=(z0, z1))


def cpu_child(spec_json):
    spec = json.loads(spec_json)
    from oracle import oracle

    oracle.build()
    cfg = workloads.CONFIGS[spec["workload"]]
    sb = cpu_sample(cfg)
    mask = oracle.geometry(sb["nx"], sb["ny"], sb["nz"], sb["slab"][0], sb["slab"][1], cfg["porosity"],
                           cfg["corr_len"], cfg["seed"])
    sim = oracle.Sim(sb["nx"], sb["ny"], sb["nz"], mask, n_species=cfg["n_species"], tau=cfg["tau"],
                     rho_in=cfg["rho_in"], rho_out=cfg["rho_out"], c_in=cfg["c_in"], p=spec["p"])
    nf = int((mask == 0).sum())
    for _ in range(spec["warmup"]):
        sim.step(1)
    steps = spec["steps"]
    if steps <= 0:  # fill about target_s seconds
        t0 = time.perf_counter()
        sim.step(2)
        per = (time.perf_counter() - t0) / 2
        steps = max(2, int(spec.get("target_s", 12.0) / max(per, 1e-6)))
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    print(json.dumps({"value": nf * steps / dt / 1e6, "steps": steps, "seconds": dt, "n_fluid": nf,
                      "cores": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count())),
                      "box": [sb["nx"], sb["ny"], sb["nz"]], "slab": list(sb["slab"])}))


def run_cpu(workload, p, steps, warmup, target_s=12.0):
    env = dict(os.environ)
    env["OMP_NUM_THREADS"] = str(os.cpu_count())
    env.pop("CUDA_VISIBLE_DEVICES", None)
    spec = json.dumps({"workload": workload, "p": p, "steps": steps, "warmup": warmup, "target_s": target_s})
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-child", spec], env=env,
                         capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = workloads.CONFIGS[args.workload]
    from oracle import oracle

    oracle.build()
    sb = cpu_sample(cfg)
    mask = oracle.geometry(sb["nx"], sb["ny"], sb["nz"], sb["slab"][0], sb["slab"][1], cfg["porosity"],
                           cfg["corr_len"], cfg["seed"])
    delta = oracle.chord_length(sb["nx"], sb["ny"], sb["nz"], sb["slab"][0], sb["slab"][1], mask)
    p = oracle.reaction_probability(cfg["Da"], delta)
    r = run_cpu(args.workload, p, args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": r["value"], "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * r["seconds"] / r["steps"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg["name"], "sample": f"{sb['nx']}x{sb['ny']}x{sb['nz']} sub-box, slab {sb['slab']}",
                   "n_fluid": r["n_fluid"]},
        "cpu_baseline": {"value": r["value"], "unit": "MLUPS", "cores": r["cores"], "kind": "oracle",
                         "sample": f"{sb['nx']}x{sb['ny']}x{sb['nz']} sub-box of {cfg['name']} "
                                   f"(same porosity, correlation length, seed, species, BCs), {r['steps']} steps"},
        "e2e": {"value": r["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# --------------------------------------------------------------------------
# GPU side
# --------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampled during the timed region."""

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def code_only(text):
    """C++ source with its comments removed and whitespace runs collapsed
    (string and character literals kept), so that the kernel hash changes
    with the code but not with its comments."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash(read=None):
    """Hash of the step kernels' code (comments and layout excluded): the
    committed DRAM traffic per entry holds for this code only."""
    read = read or (lambda f: open(os.path.join(ROOT, "paper_1607_02874_gb300", "csrc", f)).read())
    h = hashlib.sha256()
    for f in ("step_impl.cuh", "lbm_internal.h"):
        h.update(code_only(read(f)).encode())
        h.update(b"\0")
    return h.hexdigest()[:16]


def recorded_traffic(key, entries):
    """DRAM bytes per launch of the fast step kernel from a committed ncu
    summary, if it was taken on the current kernel source: bytes per lattice
    entry (measured on a smaller case, both parities averaged) times the
    entries one launch updates."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    e = d.get(key)
    if not e or e.get("kernel_hash") != kernel_source_hash():
        return None
    return int(round(e["fast_bytes_per_entry"] * entries))


def max_over_ranks(x, dist, device):
    """The largest value of x over all ranks (x itself on one rank): every
    rank times the same work, and the job takes as long as its slowest."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world, cells_per_rank, steps, seconds):
    """Whole-job throughput of `world` replicas that each update
    cells_per_rank cells `steps` times within `seconds` (the slowest rank's
    time)."""
    return world * cells_per_rank * steps / seconds / 1e6


def time_steps(sim, torch, K, stream):
    """CUDA events on the simulation's stream around every launch."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    ev[0].record(stream)
    for k in range(K):
        sim.step(1)
        ev[k + 1].record(stream)
    stream.synchronize()
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(K)]
    return ev[0].elapsed_time(ev[K]), per


def main():
    args = parse()
    if args.cpu_child:
        cpu_child(args.cpu_child)
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    import numpy as np
    import torch

    from paper_1607_02874_gb300 import build as lbuild
    from paper_1607_02874_gb300 import lbm

    lbuild.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    cfg = workloads.CONFIGS[args.workload]
    st_name, ly_name = default_storage_layout(cfg)
    st_name = args.storage or st_name
    ly_name = args.layout or ly_name
    stream = torch.cuda.Stream()
    S = 1 + cfg["n_species"]

    with torch.cuda.stream(stream):
        g = lbm.Geometry(cfg["nx"], cfg["ny"], cfg["nz"], slab=cfg["slab"], porosity=cfg["porosity"],
                         corr_len=cfg["corr_len"], seed=cfg["seed"], stream=stream)
    ginfo = g.info()
    nf = ginfo["n_fluid"]

    def measure(storage_name, layout_name, K, W, windows, clocks=False):
        sim = lbm.Simulation(g, tau=cfg["tau"], rho_in=cfg["rho_in"], rho_out=cfg["rho_out"], c_in=cfg["c_in"],
                             Da=cfg["Da"], n_species=cfg["n_species"], storage=STORAGES[storage_name],
                             layout=LAYOUTS[layout_name], c_init=args.c_init, stream=stream)
        sim.step(W)
        stream.synchronize()
        torch.cuda.synchronize()
        clk = Clocks(local) if clocks else None
        if clk:
            clk.__enter__()
        win = []
        for _ in range(windows):
            barrier()
            torch.cuda.synchronize()
            total_ms, _per = time_steps(sim, torch, K, stream)
            torch.cuda.synchronize()
            barrier()
            win.append(max_over_ranks(total_ms, dist, "cuda"))
        if clk:
            clk.__exit__(None, None, None)
        # the launches of a step timed apart (CUDA events on the stream
        # the library launches on), over both parities
        t_split = sim.info()["step"]
        split = [sim.step_timed() for _ in range(8)]
        ms_fast = statistics.mean(x[0][0] for x in split)
        # the fast kernel by the parity of the step it advances (t -> t + 1)
        by_par = [statistics.mean(x[0][0] for j, x in enumerate(split) if (t_split + j) % 2 == par) for par in (0, 1)]
        ms_gen = statistics.mean(x[0][1] for x in split)
        ms_node = statistics.mean(x[0][2] for x in split)
        ent = split[0][1]
        obs = sim.observables()
        info = sim.info()
        warps = sim.warp_counts()
        sim.close()
        return {"win_ms": win, "obs": obs, "info": info, "ms_fast": ms_fast, "ms_gen": ms_gen, "ms_node": ms_node,
                "ms_fast_par": by_par, "entries": ent, "warps": warps, "clocks": clk.summary() if clk else None}

    res = measure(st_name, ly_name, args.steps, args.warmup, args.windows, clocks=True)
    bpv = 4 if st_name == "fp32" else 2
    B_alg = 2 * Q * S * bpv
    win_sorted = sorted(res["win_ms"])
    med_ms = statistics.median(res["win_ms"])
    ms_step = med_ms / args.steps
    value = job_mlups(world, nf, args.steps, med_ms / 1e3)
    peak, peak_kind = measured_peaks()
    layout_used = {1: "dense", 2: "fluid"}[res["info"]["layout"]]
    e_fast, e_gen = res["entries"]
    achieved = B_alg * e_fast / (res["ms_fast"] / 1e3) / 1e9
    step_gbs = B_alg * nf / (ms_step / 1e3) / 1e9
    traffic = recorded_traffic(f"{cfg['name']}/{st_name}/{layout_used}", e_fast)
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
            "bytes_per_cell_update": B_alg, "units_per_launch": e_fast,
            "kernel": "fast_step_kernel (fused collide/stream of every warp away from the inlet/outlet planes, "
                      f"with the bounce-back redirection for cells touching a solid; {e_fast} of {e_fast + e_gen} "
                      "lattice entries; on odd steps two launches, the all-fluid region warps and the rest, "
                      "timed together)",
            "launch_ms": round(res["ms_fast"], 4),
            "launch_ms_even_odd": [round(x, 4) for x in res["ms_fast_par"]],
            "odd_even_ratio": round(res["ms_fast_par"][1] / res["ms_fast_par"][0], 3),
            "warps": res["warps"],
            "general_kernel": {"entries": e_gen, "launch_ms": round(res["ms_gen"], 4),
                               "achieved": round(B_alg * e_gen / (res["ms_gen"] / 1e3) / 1e9, 1)},
            "node_kernels": {"nodes": ginfo["n_nodes"], "launch_ms": round(res["ms_node"], 4),
                             "what": "catalytic-node emission and wall-hit kernels of one step together"},
            "step": {"achieved": round(step_gbs, 1), "frac": round(step_gbs / peak, 4),
                     "what": "algorithmic bytes of every fluid cell / median-window step time (every launch of the step)"}}

    variants = {}
    if not args.no_companion and st_name != "fp32":
        kc = max(args.steps // 2, 10)
        comp = measure("fp32", ly_name, kc, min(args.warmup, 20), max(args.windows // 2, 1) + 1)
        med32 = statistics.median(comp["win_ms"])
        v32 = job_mlups(world, nf, kc, med32 / 1e3)
        a32 = 2 * Q * S * 4 * comp["entries"][0] / (comp["ms_fast"] / 1e3) / 1e9
        s32 = 2 * Q * S * 4 * nf / (med32 / kc / 1e3) / 1e9
        variants["fp32"] = {"value": round(v32, 1), "unit": "MLUPS", "roofline_frac": round(a32 / peak, 4),
                            "achieved_gbs": round(a32, 1), "step_frac": round(s32 / peak, 4),
                            "odd_even_ratio": round(comp["ms_fast_par"][1] / comp["ms_fast_par"][0], 3),
                            "storage_speedup": round(value / v32, 3)}

    e2e = None
    if not args.no_e2e:
        # the input: the sample's mask in pinned host memory, filled before
        # the timed region
        exported = g.export()["mask"]
        pinned = torch.empty(exported.size, dtype=torch.uint8, pin_memory=True)
        host_mask = pinned.numpy()
        host_mask[:] = exported
        del exported
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        g2 = lbm.Geometry(cfg["nx"], cfg["ny"], cfg["nz"], slab=cfg["slab"], mask=host_mask, stream=stream)
        sim2 = lbm.Simulation(g2, tau=cfg["tau"], rho_in=cfg["rho_in"], rho_out=cfg["rho_out"], c_in=cfg["c_in"],
                              Da=cfg["Da"], n_species=cfg["n_species"], storage=STORAGES[st_name],
                              layout=LAYOUTS[ly_name], c_init=args.c_init, stream=stream)
        sim2.step(args.steps)
        o2 = sim2.observables(profiles=True)
        t1 = time.perf_counter()
        dt = max_over_ranks(t1 - t0, dist, "cuda")
        d2h = 8 * 20 + 5 * 8 * cfg["nz"]
        e2e = {"value": round(job_mlups(world, nf, args.steps, dt), 1), "unit": "MLUPS",
               "h2d_bytes_per_step": int(host_mask.nbytes / args.steps), "d2h_bytes_per_step": int(d2h / args.steps),
               "what": "lbm_create_geometry from the mask in pinned host memory + lbm_init + lbm_step x steps + "
                       "lbm_observables"}
        sim2.close()
        g2.close()

    serving = None
    if args.serving_requests > 0:
        from paper_1607_02874_gb300.serving import LbmBackend, ServingLoop, requests_from_workload

        reqs = requests_from_workload(workloads.serving_requests(n=args.serving_requests))
        be = LbmBackend(storage=lbm.FP16_DEV, layout=lbm.LAYOUT_FLUID)
        budget = int(0.5 * torch.cuda.mem_get_info()[0])
        loop = ServingLoop(be, budget_bytes=budget, steps_per_tick=100, check_every=500,
                           max_steps=args.serving_max_steps, tol=1e-8)
        out = loop.run(reqs)
        serving = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in out.items() if k != "records"}
        serving.update({"stream": f"scaled-down smoke run of the serving loop: the first {len(reqs)} of the 256 "
                                  f"requests (Poisson arrivals 20/s, cubic L in [48,192], phi U[0.55,0.75], "
                                  f"l U[4,16], Da log-U[1e-3,10]), FP16 fluid-only, steady when eta changes < 1e-8 "
                                  f"over 500 steps, cap {args.serving_max_steps} steps (the full stream with the "
                                  f"20k-step cap is studies.py serving)",
                        "budget_bytes": budget,
                        "max_batch": max((e[2] for e in loop.trace if e[1] == "tick"), default=0)})

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = run_cpu(cfg["name"], res["info"]["p"], 0, 2)
        cpu = {"value": round(r["value"], 3), "unit": "MLUPS", "cores": r["cores"], "kind": "oracle",
               "sample": f"{r['box'][0]}x{r['box'][1]}x{r['box'][2]} sub-box of {cfg['name']} (same porosity, "
                         f"correlation length, seed, species, BCs, p), {r['steps']} steps, FP64, "
                         f"{r['n_fluid']} fluid cells"}

    obs = res["obs"]
    # launches in the timed windows: odd steps run the region warps' fast
    # launch besides the one over the other fast warps
    wc = res["warps"]
    other = int(e_gen > 0) + 2 * int(ginfo["n_nodes"] > 0)
    n_timed = args.steps * args.windows
    n_odd = (args.warmup + n_timed) // 2 - args.warmup // 2
    fast_even = int(wc["plain"] + wc["region"] + wc["wall"] > 0)
    fast_odd = int(wc["region"] > 0) + int(wc["plain"] + wc["wall"] > 0)
    gpu_launches = (n_timed - n_odd) * (fast_even + other) + n_odd * (fast_odd + other)
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
        "windows": {"n": args.windows, "steps_each": args.steps,
                    "ms_per_step": [round(w / args.steps, 4) for w in res["win_ms"]],
                    "best_ms_per_step": round(win_sorted[0] / args.steps, 4),
                    "median_ms_per_step": round(ms_step, 4),
                    "mean_ms_per_step": round(statistics.mean(res["win_ms"]) / args.steps, 4),
                    "best_value": round(job_mlups(world, nf, args.steps, win_sorted[0] / 1e3), 1)},
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": cfg["name"], "box": [cfg["nx"], cfg["ny"], cfg["nz"]], "slab": list(cfg["slab"]),
                   "porosity": cfg["porosity"], "corr_len": cfg["corr_len"], "Da": cfg["Da"],
                   "species": "C+R+P" if S == 3 else "C+R", "storage": st_name, "layout": layout_used,
                   "n_fluid": nf, "n_nodes": ginfo["n_nodes"], "p": res["info"]["p"], "delta": ginfo["delta"],
                   "l2": f"inputs larger than L2: {B_alg * nf / 2 / 1e9:.1f} GB of populations per step vs "
                         f"{L2_BYTES / 1e6:.0f} MB L2",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "initial_reactant": args.c_init,
                   "catalysis": ("live in the timed region: reactant at rest in every fluid cell at t = 0, so "
                                 "every gas-solid link carries wall hits from the first step")
                   if args.c_init > 0 else "paper's start: no reactant inside at t = 0"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": res["clocks"], "variants": variants, "serving": serving,
        "check": {"eta": obs["eta"], "M_R": obs["M_R"], "M_P": obs["M_P"], "hits_R": obs["hits_R"],
                  "reacted": obs["reacted"], "resid_C_rel": obs["resid_C"] / obs["M_C"],
                  "resid_RP_rel": obs["resid_RP"] / max(obs["reacted"], 1e-300), "status": obs["status"]},
    }
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
