"""Benchmark of the D2Q9 pseudopotential step on GB300.

Default workload: one 8192 x 8192 FP32 droplet lattice (R = 2048, T_r = 0.8,
BGK tau = 1, eps = 1.73, sigma = 1), the roofline configuration.  A "step"
is one time step of the whole hot path over that lattice: pull, density,
psi, force, collision and store, by default in one kernel launch (the
single pass).  The working set (two population buffers, 4.8 GB) is far
larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload roofline|batched|served]

Prints one JSON line (rank 0).  On one GPU the default line also carries
"batched" (the 512-lattice batch of configuration 4, 100 timed steps, against
one handle per lattice) and "served" (configuration 5's Poisson stream of
1000 requests, step counts divided by 100, against one plain handle per
request), measured after the roofline lattice's timed region, and in
"config" the same lattice's step rate with psi in native FP64 (20 steps).
``--impl reference`` times the FP64 CPU
oracle (the only reference this method has) on a bounded crop of the same
workload, on the host cores.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("MLUPS and % of HBM peak per step; batched/served p50/p99 vs plain FP32 at "
                   "1e-5")
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="roofline", choices=["roofline", "batched", "served"])
    ap.add_argument("--requests", type=int, default=1000,
                    help="served workload: number of requests of the Poisson stream")
    ap.add_argument("--step-scale", type=int, default=100,
                    help="served workload: divide each request's step count by this")
    ap.add_argument("--target-sites", type=int, default=0,
                    help="served workload: resident-site target of the server (0: default)")
    ap.add_argument("--chunk", type=int, default=100,
                    help="served workload: most steps per server chunk")
    ap.add_argument("--chunk-ms", type=float, default=4.0,
                    help="served workload: GPU time a server chunk aims at (< 0: fixed --chunk)")
    ap.add_argument("--eos", default="df", choices=["f64", "df", "f32"],
                    help="arithmetic of psi/EOS: float-float (default), native FP64 or FP32")
    ap.add_argument("--variant", default="auto", choices=["auto", "tma", "plain"])
    ap.add_argument("--schedule", default="fused", choices=["two_pass", "fused"],
                    help="fused: one pass per step (default); two_pass: psi pass + collision pass")
    ap.add_argument("--storage", default="f32dev", choices=["f32", "f32dev", "f16dev"])
    ap.add_argument("--collision", default="bgk", choices=["bgk", "mrt"],
                    help="collision operator: BGK (default) or MRT with the rates of the "
                         "paper's oscillation test (s = 1 for the non-hydrodynamic moments, "
                         "1/tau for the stress)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--roofline-only", action="store_true",
                    help="default workload: skip the batched and served measurements that the "
                         "JSON line otherwise carries beside the roofline lattice")
    ap.add_argument("--tile", type=int, nargs=3, metavar=("TX", "TY", "SPT"), default=None,
                    help="fixed tile and sites per thread for both passes (no autotune)")
    ap.add_argument("--grid", type=int, default=0,
                    help="with --tile: CTAs of the launches (0: persistent, SMs x occupancy; "
                         "at least the tile count: one CTA per tile)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip lbm_autotune (tile shapes, sites per thread, grid) before timing")
    ap.add_argument("--lattices", type=int, default=512,
                    help="batched workload: the first N lattices of the 512-lattice recipe "
                         "(512 is the benchmark; fewer are for profiler captures)")
    ap.add_argument("--no-sequential", dest="sequential", action="store_false",
                    help="batched workload: skip the one-handle-per-lattice comparison")
    ap.add_argument("--size", type=int, default=8192,
                    help="lattice side of the droplet workload (8192 is the benchmark; "
                         "smaller sides are for profiler captures)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def job_rate(dist, units, seconds, device=None):
    """Whole-job rate of replicas: the units every rank processed divided by
    the slowest rank's time.  Returns (rate, slowest seconds); one process
    without a process group: units / seconds."""
    if dist is None:
        return units / seconds, seconds
    import torch

    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (6.8 TB/s)"


KERNEL_SOURCES = ("lbm_device.cuh", "lbm_async.cuh", "lbm_copy_plan.h", "lbm_layout.h",
                  "lbm_kernels.h", "lbm_fused_tma.cuh")


def _code_only(text):
    """C++ source without its comments and blank space, so that an edit of a
    comment leaves the hash of the code unchanged."""
    import re

    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash():
    """Hash of the code (comments left out) of the files that define the
    single-pass step kernel (not the host runtime)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2003_07968_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(d, f), encoding="utf-8") as fh:
            h.update(f.encode() + _code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload_key):
    """DRAM bytes per launch from a committed ncu summary, only while the
    kernel sources are unchanged since the capture (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as fh:
            tab = json.load(fh)
    except Exception:
        return None
    ent = tab.get(workload_key, {}).get(kernel)
    if not ent or ent.get("source_hash") != kernel_source_hash():
        return None
    return ent.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix=f"clocks_rank{self.index}_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.readlines()
        try:
            os.remove(self.path)
        except OSError:
            pass
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ workloads
def roofline_workload(n=8192):
    import synth

    R, T = n / 4.0, 0.8
    return dict(key=f"droplet_{n}", nx=n, ny=n, R=R, T=T, tau=1.0,
                field=lambda: synth.droplet(n, n, R, T),
                name=f"droplet {n}x{n} FP32, R={int(R)}, T_r={T}, BGK tau=1.0, eps=1.73, sigma=1")


def cpu_baseline(seconds=12.0):
    """The FP64 oracle, as it stands, on a bounded crop of the roofline
    workload: a 1024 x 1024 periodic window across the droplet edge."""
    import oracle
    import synth

    n, R, T = 8192, 2048.0, 0.8
    full_x0 = n // 2 + int(R) - 512
    y, x = np.mgrid[0:1024, 0:1024].astype(float)
    y += n // 2 - 512
    x += full_x0
    rg, rl = synth.coexistence(T)
    r = np.sqrt((x - n // 2) ** 2 + (y - n // 2) ** 2)
    rho = 0.5 * (rl + rg) - 0.5 * (rl - rg) * np.tanh(2.0 * (r - R) / 5.0)
    p = oracle.params(T=T, tau=1.0)
    f = oracle.init_equilibrium(rho)
    t0 = time.perf_counter()
    oracle.step(p, f, 1)
    one = time.perf_counter() - t0
    k = max(1, min(200, int(seconds / max(one, 1e-6))))
    t0 = time.perf_counter()
    oracle.step(p, f, k)
    dt = time.perf_counter() - t0
    return {"value": round(1024 * 1024 * k / dt / 1e6, 3), "unit": "MLUPS",
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"1024x1024 crop of the 8192^2 droplet across its interface, {k} steps, "
                      f"FP64 C oracle with OpenMP ({dt:.1f} s)"}


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle

    wl = roofline_workload()
    n = 512  # crop per step: bounded so the whole run ends within minutes
    import synth

    T, R = wl["T"], wl["R"]
    y, x = np.mgrid[0:n, 0:n].astype(float)
    y += wl["ny"] // 2 - n // 2
    x += wl["nx"] // 2 + int(R) - n // 2
    rg, rl = synth.coexistence(T)
    r = np.sqrt((x - wl["nx"] // 2) ** 2 + (y - wl["ny"] // 2) ** 2)
    rho = 0.5 * (rl + rg) - 0.5 * (rl - rg) * np.tanh(2.0 * (r - R) / 5.0)
    p = oracle.params(T=T, tau=wl["tau"])
    f = oracle.init_equilibrium(rho)
    oracle.step(p, f, args.warmup)
    t0 = time.perf_counter()
    oracle.step(p, f, args.steps)
    dt = time.perf_counter() - t0
    v = n * n * args.steps / dt / 1e6
    sample = (f"{n}x{n} periodic crop of the 8192^2 droplet across its interface per step, "
              f"FP64 C oracle with OpenMP")
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(dt / args.steps * 1e3, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": wl["name"] + " (oracle crop)"},
           "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": oracle.num_threads(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0},
           "gpu_launches": 0}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2003_07968_gb300 import build, capi as P

    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    P.load()
    eos = {"f64": P.LBM_EOS_F64, "df": P.LBM_EOS_DF, "f32": P.LBM_EOS_F32}[args.eos]
    storage = {"f32": P.LBM_STORE_F32, "f32dev": P.LBM_STORE_F32_DEV,
               "f16dev": P.LBM_STORE_F16_DEV}[args.storage]
    wl = roofline_workload(args.size)
    rho = wl["field"]()
    coll = {}
    if args.collision == "mrt":
        coll = dict(collision=P.LBM_COLL_MRT, mrt_rates=[1.0] * 7 + [1.0 / wl["tau"]] * 2)
    d = P.lbm_desc_default(wl["nx"], wl["ny"], T=wl["T"], tau=wl["tau"], eos_precision=eos,
                           storage=storage, **coll)
    h = P.lbm_create(d, kernel_variant={"auto": P.LBM_KERNEL_AUTO, "tma": P.LBM_KERNEL_TMA,
                                        "plain": P.LBM_KERNEL_PLAIN}[args.variant],
                     schedule={"two_pass": P.LBM_SCHED_TWO_PASS,
                               "fused": P.LBM_SCHED_FUSED}[args.schedule],
                     tile=tuple(args.tile[:2]) if args.tile else None,
                     sites_per_thread=args.tile[2] if args.tile else 0,
                     grid_ctas=args.grid if args.tile else 0)
    st = h.stream
    P.lbm_init(h, 0, rho)
    if args.autotune and not args.tile:
        P.lbm_autotune(h, 10)
    info = P.lbm_info(h)
    sites = info["sites"]
    P.lbm_step(h, args.warmup)
    P.lbm_sync(h)

    # ---- device-resident timed region (kernels profiled with events on h.stream)
    P.lbm_profile(h, True)
    P.lbm_profile_read(h)  # reset pending records
    l0 = P.lbm_launch_count(h)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(st)
        P.lbm_step(h, args.steps)
        e1.record(st)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches = P.lbm_launch_count(h) - l0
    ms = e0.elapsed_time(e1)
    stats = {s["name"]: s for s in P.lbm_profile_read(h)}
    P.lbm_profile(h, False)
    P.lbm_sync(h)
    rate, s_max = job_rate(dist, sites * args.steps, ms * 1e-3, device="cuda")
    ms_max = s_max * 1e3
    value = rate / 1e6

    # ---- end-to-end through the C ABI with host buffers (pinned)
    host_rho = torch.from_numpy(rho).pin_memory().numpy()
    host_out = torch.empty(rho.shape, dtype=torch.float64).pin_memory().numpy()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    P.lbm_init(h, 0, host_rho)
    P.lbm_step(h, args.steps)
    m = P.lbm_moments(h, 0, rho=True, u=False, mass=True, out={"rho": host_out})
    e2e_rate, _ = job_rate(dist, sites * args.steps, time.perf_counter() - t0, device="cuda")
    e2e = {"value": round(e2e_rate / 1e6, 3), "unit": "MLUPS",
           "h2d_bytes_per_step": round(host_rho.nbytes / args.steps, 1),
           "d2h_bytes_per_step": round((host_out.nbytes + 8) / args.steps, 1),
           "mass_rel_drift": abs(m["mass"] - float(rho.sum())) / float(rho.sum())}
    P.lbm_destroy(h)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    peak, peak_src = measured_hbm_peak()
    ks = [s for s in stats.values() if s["launches"] > 0]
    dom = max(ks, key=lambda s: s["total_ms"])
    avg_ms = dom["total_ms"] / max(dom["launches"], 1)
    achieved = dom["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9
    tot = sum(s["total_ms"] for s in ks)
    kernels = {s["name"]: {"launches": s["launches"], "avg_ms": round(s["total_ms"] / max(s["launches"], 1), 5),
                           "share": round(s["total_ms"] / max(tot, 1e-9), 4),
                           "algorithmic_GBps": round(s["bytes_per_launch"] / (s["total_ms"] / max(s["launches"], 1) * 1e-3) / 1e9, 1)}
               for s in ks}
    es = 2 if args.storage == "f16dev" else 4
    step_bytes = 18 * es  # read 9 and write 9 populations: the method's minimum per site
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_max / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["name"] if args.collision == "bgk"
                   else wl["name"].replace("BGK", "MRT"), "storage": args.storage, "eos": args.eos,
                   "eos_arithmetic": EOS_ARITH[args.eos],
                   "collision": args.collision,
                   "schedule": args.schedule, "kernel_variant": args.variant,
                   "psi_pass": {"variant": ["auto", "plain", "tma"][info["psi_variant"]],
                                "tile": [info["psi_tile_x"], info["psi_tile_y"]],
                                "sites_per_thread": info["psi_spt"],
                                "grid_ctas": info["psi_grid_ctas"]},
                   "collide_pass": {"variant": ["auto", "plain", "tma"][info["collide_variant"]],
                                    "tile": [info["tile_x"], info["tile_y"]],
                                    "sites_per_thread": info["spt"],
                                    "tensor_map": bool(info["tensor_map"]),
                                    "grid_ctas": info["grid_ctas"]},
                   "sites": sites,
                   "l2": f"working set {info['device_bytes'] / 1e9:.2f} GB vs 129 MB L2: "
                         "inputs larger than L2, no flush",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     # the committed capture is of one kernel instance: the TMA single
                     # pass, 32x16 tiles, FP32 deviations, float-float EOS, BGK
                     "traffic": (ncu_traffic(dom["name"], wl["key"])
                                 if (args.collision, args.storage, args.eos, args.schedule,
                                     info["collide_variant"], info["tile_x"], info["tile_y"])
                                 == ("bgk", "f32dev", "df", "fused", P.LBM_KERNEL_TMA, 32, 16)
                                 else None),
                     "peak_source": peak_src,
                     "bytes_per_launch": dom["bytes_per_launch"]},
        "step_roofline": {"algorithmic_bytes_per_site": step_bytes,
                          "effective_GBps": round(value * 1e6 * step_bytes / 1e9 / world, 1),
                          "frac": round(value * 1e6 * step_bytes / 1e9 / world / peak, 4)},
        "kernels": kernels,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
    }
    if world == 1 and not args.roofline_only and args.eos == "df":
        out["config"]["native_f64_eos"] = measure_native_f64_eos(P, wl, rho, storage, coll)
    if world == 1 and not args.roofline_only:
        # the metric's other two parts, measured after the timed region above
        # and outside it: the 512-lattice batch and the served stream, each
        # against sequential plain handles on this GPU
        b = measure_batched(P, storage, steps=100, warmup=5)
        b.pop("_info")
        out["batched"] = b
        sv = measure_served(P, storage, requests=1000, step_scale=100)
        sv.pop("_target")
        out["served"] = sv
    if not args.no_cpu_baseline and world == 1:
        out["cpu_baseline"] = cpu_baseline()
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------------ batched workload
EOS_ARITH = {
    "df": "float-float radicand (about 43 bits, FP64-equivalent at physical densities), "
          "FP32 square root",
    "f64": "native FP64 radicand and square root",
    "f32": "FP32 radicand and square root",
}


def measure_native_f64_eos(P, wl, rho, storage, coll, steps=20):
    """The same lattice with psi evaluated in native FP64 (LBM_EOS_F64), the
    tile autotuned for it: context beside the float-float default, whose
    radicand keeps about 43 bits.  FP64 runs at a small fraction of the FP32
    rate on this GPU."""
    import torch

    d = P.lbm_desc_default(wl["nx"], wl["ny"], T=wl["T"], tau=wl["tau"],
                           eos_precision=P.LBM_EOS_F64, storage=storage, **coll)
    h = P.lbm_create(d, schedule=P.LBM_SCHED_FUSED)
    P.lbm_init(h, 0, rho)
    P.lbm_autotune(h, 5)
    P.lbm_step(h, 3)
    P.lbm_sync(h)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(h.stream)
    P.lbm_step(h, steps)
    e1.record(h.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sites = P.lbm_info(h)["sites"]
    P.lbm_destroy(h)
    return {"MLUPS": round(sites * steps / (ms * 1e-3) / 1e6, 1), "steps": steps,
            "ms_per_step": round(ms / steps, 5)}


def measure_batched(P, storage, steps, warmup, autotune=True, sequential=True, lattices=512):
    """512 independent droplet lattices of uneven sizes (sides U{64..512},
    R = side x U(0.15, 0.35), T_r U(0.6, 0.9), tau = 1) stepped together by
    one batch handle (persistent launches over one tile list, CUDA graphs),
    against the same lattices stepped one handle after another on one stream.
    Three lattices (the first, the middle one, the largest) must come out of
    the batch bitwise equal to their own handles' runs."""
    import torch

    import synth

    rec = synth.batch_recipe()[:max(1, min(lattices, 512))]
    descs = [P.lbm_desc_default(r["nx"], r["ny"], T=r["T"], storage=storage) for r in rec]
    fields = [synth.droplet(r["nx"], r["ny"], r["R"], r["T"]) for r in rec]
    sites = sum(r["nx"] * r["ny"] for r in rec)
    h = P.lbm_create(descs)
    for i, f in enumerate(fields):
        P.lbm_init(h, i, f)
    if autotune:
        P.lbm_autotune(h, 10)
    P.lbm_step(h, warmup)
    P.lbm_sync(h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    P.lbm_profile(h, True)
    P.lbm_profile_read(h)
    l0 = P.lbm_launch_count(h)
    torch.cuda.synchronize()
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(h.stream)
        P.lbm_step(h, steps)
        e1.record(h.stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    stats = {st["name"]: st for st in P.lbm_profile_read(h)}
    P.lbm_profile(h, False)
    launches = P.lbm_launch_count(h) - l0
    P.lbm_sync(h)
    info = P.lbm_info(h)
    batched = sites * steps / (ms * 1e-3) / 1e6
    seq, same = None, None
    if sequential:
        stream = torch.cuda.Stream()
        hs = []
        for d, f in zip(descs, fields):
            hh = P.lbm_create(d, stream=stream)
            P.lbm_init(hh, 0, f)
            P.lbm_step(hh, warmup)
            hs.append(hh)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for hh in hs:
            P.lbm_step(hh, steps)
        s1.record(stream)
        torch.cuda.synchronize()
        seq = sites * steps / (s0.elapsed_time(s1) * 1e-3) / 1e6
        big = int(np.argmax([r["nx"] * r["ny"] for r in rec]))
        same = True
        for i in sorted({0, len(rec) // 2, big}):
            a_ = P.lbm_moments(h, i, u=False, mass=False)["rho"]
            b_ = P.lbm_moments(hs[i], 0, u=False, mass=False)["rho"]
            same = same and bool(np.array_equal(a_, b_))
        for hh in hs:
            P.lbm_destroy(hh)
    P.lbm_destroy(h)
    peak, peak_src = measured_hbm_peak()
    es = 2 if storage == P.LBM_STORE_F16_DEV else 4
    kname, k2 = max(stats.items(), key=lambda kv: kv[1]["total_ms"])  # dominant kernel
    avg = k2["total_ms"] / max(k2["launches"], 1)
    achieved = k2["bytes_per_launch"] / (avg * 1e-3) / 1e9
    return {
        "MLUPS": round(batched, 1),
        "sequential_MLUPS": round(seq, 1) if seq else None,
        "speedup": round(batched / seq, 3) if seq else None,
        "batch_equals_alone": same,
        "lattices": len(rec), "sites": sites, "steps": steps, "ms_per_step": round(ms / steps, 5),
        "sequential": "one handle per lattice, lbm_step one after another on one stream",
        "kernel": {"name": kname, "tile": [info["tile_x"], info["tile_y"]],
                   "sites_per_thread": info["spt"], "achieved_GBps": round(achieved, 1),
                   "frac": round(achieved / peak, 4), "peak_source": peak_src},
        "algorithmic_bytes_per_site": 18 * es,
        "gpu_launches": int(launches), "clocks": clk.summary(),
        "_info": info,
    }


def run_batched(args):
    """The batched workload alone, as its own JSON line."""
    import torch

    from paper_2003_07968_gb300 import build, capi as P

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    P.load()
    storage = {"f32": P.LBM_STORE_F32, "f32dev": P.LBM_STORE_F32_DEV,
               "f16dev": P.LBM_STORE_F16_DEV}[args.storage]
    b = measure_batched(P, storage, args.steps, args.warmup, args.autotune, args.sequential,
                        args.lattices)
    info = b.pop("_info")
    peak, peak_src = measured_hbm_peak()
    out = {"metric": METRIC, "value": b["MLUPS"], "unit": "MLUPS",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": b["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"batched: {b['lattices']} droplet lattices, sides U{{64..512}}, "
                                  f"{b['sites']} sites",
                      "storage": args.storage, "eos": args.eos,
                      "psi_pass": [info["psi_variant"], info["psi_tile_x"], info["psi_tile_y"],
                                   info["psi_spt"], info["psi_grid_ctas"]],
                      "collide_pass": [info["collide_variant"], info["tile_x"], info["tile_y"],
                                       info["spt"], info["grid_ctas"]],
                      "schedule": ["auto", "two_pass", "fused"][info["schedule"]]},
           "batched": b,
           "roofline": {"bound": "hbm", "kernel": b["kernel"]["name"],
                        "achieved": b["kernel"]["achieved_GBps"], "peak": peak, "unit": "GB/s",
                        "frac": b["kernel"]["frac"], "traffic": None, "peak_source": peak_src},
           "gpu_launches": b["gpu_launches"], "clocks": b["clocks"]}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ served workload
def measure_served(P, storage, requests, step_scale, chunk=100, chunk_ms=4.0, target_sites=0):
    """Poisson stream (200/s) of droplet / flat-band solves with sides
    U{128..2048} and steps U{1000..50000} / step_scale, submitted in real time
    to one continuous-batching server; against the same requests served one
    at a time by plain handles (first come first served, same arrivals).
    Three served results must equal the same lattice stepped alone, bitwise."""
    import threading

    import torch

    import synth

    reqs = synth.serving_stream(n=requests)
    for r in reqs:
        r["steps"] = max(1, r["steps"] // step_scale)
    fields = [synth.request_field(r) for r in reqs]
    descs = [P.lbm_desc_default(r["nx"], r["ny"], T=r["T"], storage=storage) for r in reqs]
    work = sum(r["nx"] * r["ny"] * r["steps"] for r in reqs)
    # warm the kernels once
    h = P.lbm_create(P.lbm_desc_default(256, 256, storage=storage))
    P.lbm_init(h, 0, synth.droplet(256, 256, 60.0, 0.8))
    P.lbm_step(h, 20)
    P.lbm_sync(h)
    P.lbm_destroy(h)

    # results carry rho only, as the sequential runs below read rho only
    opts = P.lbm_server_opts_default(arena_bytes=64 << 30, chunk_steps=chunk,
                                     chunk_ms=chunk_ms, storage=storage,
                                     max_resident=1024, with_velocity=0)
    if target_sites:
        opts.target_resident_sites = target_sites
    srv = P.lbm_server_create(opts)
    tickets = [None] * len(reqs)
    t_start = time.perf_counter()

    def submitter():
        for i, r in enumerate(reqs):
            dt = r["t_arrival"] - (time.perf_counter() - t_start)
            if dt > 0:
                time.sleep(dt)
            tickets[i] = P.lbm_submit(srv, descs[i], fields[i], r["steps"])

    th = threading.Thread(target=submitter)
    with ClockSampler(torch.cuda.current_device()) as clk:
        th.start()
        results, lat, failed = {}, [], 0
        while len(results) < len(reqs):
            for i, t in enumerate(tickets):
                if t is not None and i not in results:
                    try:
                        out = P.lbm_poll(srv, t, u=False)
                    except P.LbmError:
                        out = {"rho": None, "latency_s": float("nan")}
                        failed += 1
                    if out is not None:
                        results[i] = out
                        lat.append(out["latency_s"])
            time.sleep(0.0005)
        t_end = time.perf_counter()
        th.join()
    stats = P.lbm_server_get_stats(srv)
    P.lbm_server_destroy(srv)
    wall = t_end - t_start
    served = work / wall / 1e6
    # sequential: one plain handle per request, first come first served
    stream = torch.cuda.Stream()
    service = []
    for d, f, r in zip(descs, fields, reqs):
        t0 = time.perf_counter()
        hh = P.lbm_create(d, stream=stream)
        P.lbm_init(hh, 0, f)
        P.lbm_step(hh, r["steps"])
        P.lbm_moments(hh, 0, u=False, mass=False)
        P.lbm_destroy(hh)
        service.append(time.perf_counter() - t0)
    fin, seq_lat = 0.0, []
    for r, sv in zip(reqs, service):
        fin = max(fin, r["t_arrival"]) + sv
        seq_lat.append(fin - r["t_arrival"])
    seq_wall = fin - reqs[0]["t_arrival"]
    # a few served results must equal the same lattice stepped alone
    same = True
    for i in (0, len(reqs) // 2, len(reqs) - 1):
        hh = P.lbm_create(descs[i])
        P.lbm_init(hh, 0, fields[i])
        P.lbm_step(hh, reqs[i]["steps"])
        a = P.lbm_moments(hh, 0, u=False, mass=False)["rho"]
        P.lbm_destroy(hh)
        same = same and results[i]["rho"] is not None and bool(np.array_equal(a, results[i]["rho"]))
    pct = lambda v, q: float(np.percentile(np.array(v), q))
    return {"MLUPS": round(served, 1), "p50_s": round(pct(lat, 50), 4),
            "p99_s": round(pct(lat, 99), 4), "wall_s": round(wall, 3),
            "gpu_busy_s": round(stats["busy_s"], 3),
            "sequential_MLUPS": round(work / seq_wall / 1e6, 1),
            "sequential_p50_s": round(pct(seq_lat, 50), 4),
            "sequential_p99_s": round(pct(seq_lat, 99), 4),
            "speedup": round(served / (work / seq_wall / 1e6), 3),
            "mix_equals_alone": same, "failed_requests": failed,
            "requests": len(reqs), "step_scale": step_scale, "site_steps": work,
            "stream": f"Poisson 200/s, sides U{{128..2048}}, steps U{{1000..50000}}/{step_scale}, "
                      "droplet/band 50/50",
            "sequential": "one plain handle per request, first come first served, same arrivals",
            "gpu_launches": int(stats["launches"]), "clocks": clk.summary(),
            "_target": opts.target_resident_sites}


def run_served(args):
    """The served workload alone, as its own JSON line."""
    import torch

    from paper_2003_07968_gb300 import build, capi as P

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    P.load()
    storage = {"f32": P.LBM_STORE_F32, "f32dev": P.LBM_STORE_F32_DEV,
               "f16dev": P.LBM_STORE_F16_DEV}[args.storage]
    sv = measure_served(P, storage, args.requests, args.step_scale, args.chunk, args.chunk_ms,
                        args.target_sites)
    target = sv.pop("_target")
    out = {"metric": METRIC, "value": sv["MLUPS"], "unit": "MLUPS",
           "n_gpus": world, "steps": sv["requests"], "warmup": 0,
           "ms_per_step": round(sv["wall_s"] / sv["requests"] * 1e3, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"served: {sv['requests']} requests, " + sv["stream"],
                      "storage": args.storage, "chunk_steps": args.chunk,
                      "chunk_ms": args.chunk_ms, "site_steps": sv["site_steps"],
                      "target_resident_sites": target},
           "served": sv, "gpu_launches": sv["gpu_launches"], "clocks": sv["clocks"]}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "served":
        run_served(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
