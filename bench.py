#!/usr/bin/env python
"""Throughput of the explicit RK3 Navier-Stokes time step (Taylor-Green vortex,
OpenSBLI paper Section 3.3) on GB300, in grid-point-stage updates per second.

Workload (default): 256^3 periodic box, 4th-order central differences, FP64,
Re 1600, M 0.1, gamma 1.4, Pr 0.71, dt = 3.385e-3 / 4 (the paper's 64^3 step
halved per doubling), Taylor-Green initial state with seeded Gaussian noise of
amplitude 1e-4 on each velocity component.  One bench step = one full RK3 step
(3 stages) over the whole grid.  Variants (8th order, FP32 path) are timed on
the same workload and reported under "variants".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank advances its own replica (independent problems, no
data-path collective): weak scaling, value = all ranks' point-stages / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-pt-stage updates/s and %HBM roofline vs plain FP64 at matched KE-decay error"
UNIT = "grid-point-stage updates/s"
BASE_DT_64 = 3.385e-3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=256, help="points per axis")
    ap.add_argument("--order", type=int, default=4)
    ap.add_argument("--precision", choices=("fp64", "fp32"), default="fp64")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--ensemble-steps", type=int, default=500)
    ap.add_argument("--no-closure", action="store_true")
    return ap.parse_args()


def workload(args):
    n = args.n
    return dict(workload=f"tgv_{n}^3_order{args.order}_{args.precision}", n=n, order=args.order,
                precision=args.precision, Re=1600.0, Mach=0.1, gamma=1.4, Pr=0.71,
                dt=BASE_DT_64 * 64.0 / n, noise_seed=1234, noise_amp=1e-4)


# ---------------------------------------------------------------------------
# Algorithmic work per point-stage: the operations of the stage as the
# equations define it (FMA = 2).  The kernels fold some constant factors into
# precomputed stencil weights and so issue fewer; the roofline divides this
# fixed count by their time.
# ---------------------------------------------------------------------------
def resid_flops_per_point(r: int) -> int:
    d1 = 3 * r          # r subtractions + r FMAs
    d2 = 3 * r + 1      # r additions + r FMAs + 1 multiply
    flops = 15 * d1                # D_j Q_m
    flops += 5 * (6 + 2) + 3 * 2   # advective/dilatation combination, mass flux
    flops += 12 * d1 + 12          # D_j Phi_ij, D_j F_j and their sums
    flops += 12 * d2 + 3 * 6 + 4   # Laplacians and their combination
    flops += 5 * 4                 # RK update (2 FMAs per field)
    return flops


def stage_flops_per_point(r: int) -> dict:
    prim = 1 + 3 + 5 + 2 + 2 + 9   # 1/rho, u_i, ke, p, T, momentum fluxes
    grad = 9 * 3 * r + 2 + 15 + 3 * 7 + 3 * 3 + 2
    return dict(prim=prim, grad=grad, resid=resid_flops_per_point(r))


ALG_BYTES = {"fp64": 400.0 / 3.0, "fp32": 320.0 / 3.0}  # fused minimum per point-stage
# Bytes the FP32 stage kernels move by design: the fused stage (orders 2, 4)
# keeps the FP64 accumulator out of stages 1-2 (300 B per step); the two z-march
# kernels (orders 6, 8) move 195 B per point-stage.
DESIGN_BYTES_FP32 = {"fused": 100.0, "zmarch": 195.0}


def fp32_kernel(order: int) -> str:
    return "k_fused" if order <= 4 else "k_zrhs"

# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu
# launch list of the same workload (profiles/launches_tgv256_o4_*.md).
# An entry is removed whenever its kernel changes; the key is the workload
# name bench.py reports.
TRAFFIC_PER_LAUNCH = {
    ("tgv_256^3_order4_fp64", "k_resid"): 4.6204e9,  # profiles/launches_tgv256_o4_fp64.md
    # average over the three stage launches, scaled from 192^3 by the points
    # (profiles/k_fused_tgv192_o4_fp32.md)
    ("tgv_256^3_order4_fp32", "k_fused"): 1.638e9,
}

# FP64 peak from unit counts and clocks: 2 DFMA thread-instructions per SM per
# cycle (ncu peak_sustained of sm__sass_thread_inst_executed_op_dfma_pred_on),
# 2 flops each, 152 SMs, 2070 MHz maximum SM clock.
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.070e9 / 1e12


def peaks():
    p = dict(hbm_gbs=None, fp64_tflops=FP64_PEAK_TFLOPS, fp32_tflops=None, src="fallback")
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            m = json.load(f)
        p["hbm_gbs"] = m.get("hbm_gbs")
        p["src"] = "measured"
        p["sm_max_mhz"] = m.get("sm_max_mhz")
        p["bf16_tflops"] = m.get("bf16_tflops")
    if p.get("bf16_tflops") is None:
        p["bf16_tflops"] = 1900.0  # fallback burst figure
    if p["hbm_gbs"] is None:
        p["hbm_gbs"] = 6800.0
        p["src"] = "fallback"
    return p


# ---------------------------------------------------------------------------
# nvidia-smi clock sampling during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ---------------------------------------------------------------------------
# Oracle timing (the CPU baseline and the reference arm)
# ---------------------------------------------------------------------------
def time_oracle(w, target_s=12.0, max_n=None, single_core=False):
    """Times the CPU oracle on a bounded sample of the workload: one RK3 step on
    the largest cubic grid (<= the workload's) whose step fits ~target_s."""
    from oracle import oracle as orc
    from paper_1609_01277_gb300 import inputs
    orc.build()
    n_cal = 48
    case = orc.Case(n_cal, n_cal, n_cal, order=w["order"], Re=w["Re"], Mach=w["Mach"], dt=w["dt"])
    Q = orc.tgv_init(case, inputs.gaussian_noise(n_cal, n_cal, n_cal, w["noise_seed"]), w["noise_amp"])
    t0 = time.perf_counter()
    orc.rk3_step(case, Q, 1)
    per_pt = (time.perf_counter() - t0) / n_cal ** 3
    n = int((target_s / per_pt) ** (1 / 3))
    n = max(16, min(max_n or w["n"], n))
    case = orc.Case(n, n, n, order=w["order"], Re=w["Re"], Mach=w["Mach"], dt=w["dt"])
    Q = orc.tgv_init(case, inputs.gaussian_noise(n, n, n, w["noise_seed"]), w["noise_amp"])
    t0 = time.perf_counter()
    orc.rk3_step(case, Q, 1)
    dt = time.perf_counter() - t0
    out = dict(value=3 * n ** 3 / dt, unit=UNIT, cores=orc.get_threads(), kind="oracle",
               sample=f"1 RK3 step (3 stages) of the same Taylor-Green case on a {n}^3 grid, "
                      f"order {w['order']}, FP64, {dt:.2f} s on {orc.get_threads()} OpenMP threads")
    if single_core:
        # the same on one core, on a smaller sample (about a second)
        threads = orc.get_threads()
        orc.set_threads(1)
        try:
            n1 = max(16, min(n, int((1.0 / (per_pt * threads)) ** (1 / 3))))
            case1 = orc.Case(n1, n1, n1, order=w["order"], Re=w["Re"], Mach=w["Mach"], dt=w["dt"])
            Q1 = orc.tgv_init(case1, inputs.gaussian_noise(n1, n1, n1, w["noise_seed"]), w["noise_amp"])
            t0 = time.perf_counter()
            orc.rk3_step(case1, Q1, 1)
            dt1 = time.perf_counter() - t0
        finally:
            orc.set_threads(threads)
        out["single_core"] = dict(value=3 * n1 ** 3 / dt1, unit=UNIT, cores=1,
                                  sample=f"1 RK3 step on a {n1}^3 grid, {dt1:.2f} s on 1 thread")
    return out


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, timed on bounded samples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as orc
    from paper_1609_01277_gb300 import inputs
    w = workload(args)
    orc.build()
    # size each step's sample so the whole run stays within a few minutes
    cal = time_oracle(w, target_s=2.0)
    n = int(round((cal["value"] * 2.0 / 3.0) ** (1 / 3)))
    n = max(16, min(w["n"], n))
    case = orc.Case(n, n, n, order=w["order"], Re=w["Re"], Mach=w["Mach"], dt=w["dt"])
    Q = orc.tgv_init(case, inputs.gaussian_noise(n, n, n, w["noise_seed"]), w["noise_amp"])
    for _ in range(args.warmup):
        Q = orc.rk3_step(case, Q, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        Q = orc.rk3_step(case, Q, 1)
    el = time.perf_counter() - t0
    value = args.steps * 3 * n ** 3 / el
    sample = f"each step: 1 RK3 step of the same Taylor-Green case on a {n}^3 grid (oracle, FP64)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["workload"], "sample_grid": n, "order": w["order"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.get_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Our CUDA path
# ---------------------------------------------------------------------------
def make_grid(osb, w, order, precision, noise):
    cfg = osb.Config(w["n"], w["n"], w["n"], order=order,
                     precision={"fp64": osb.OSB_FP64, "fp32": osb.OSB_FP32, "df64": osb.OSB_DF64}[precision],
                     Re=w["Re"], Mach=w["Mach"], gamma=w["gamma"], Pr=w["Pr"], dt=w["dt"])
    g = osb.Grid(cfg)
    g.init_taylor_green(noise, w["noise_amp"])
    return g


def time_steps(torch, g, steps, warmup, profile=False):
    g.step(warmup)
    torch.cuda.synchronize()
    if profile:
        g.profile_start(3 * steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(g.stream)
    g.step(steps)
    e1.record(g.stream)
    torch.cuda.synchronize()
    prof = g.profile_stop() if profile else None
    return e0.elapsed_time(e1), prof


def ke_series(torch, g, steps):
    """E_k after each step from the FP64 accumulator (the separate reduction:
    the FP32 path's fused series would add its own FP32 evaluation error)."""
    out = [g.diagnostics()["ke"]]
    for _ in range(steps):
        g.step(1)
        out.append(g.diagnostics()["ke"])
    return out


def ensemble_specs(count=64, seed=7):
    """The uneven Taylor-Green ensemble: N from {32,48,64,96,128}, Re in
    [100, 3200], M in [0.05, 0.3]; dt = 3.385e-3 (64/N) 11/(1 + 1/M) keeps the
    paper's acoustic Courant number of the 64^3, M = 0.1 case."""
    from paper_1609_01277_gb300 import inputs
    return inputs.ensemble_with_dt(count, seed, BASE_DT_64)


def run_ensemble(torch, osb, inputs, steps, precision):
    specs = ensemble_specs()
    prec = {"fp64": osb.OSB_FP64, "fp32": osb.OSB_FP32, "df64": osb.OSB_DF64}[precision]
    grids = []
    for i, e in enumerate(specs):
        n = e["n"]
        g = osb.Grid(osb.Config(n, n, n, order=4, precision=prec, Re=e["Re"], Mach=e["Mach"], dt=e["dt"]))
        g.init_taylor_green(torch.from_numpy(inputs.gaussian_noise(n, n, n, 1000 + i)).cuda(), 1e-4)
        grids.append(g)
    tuned = {}
    if ensemble_launches(precision, len(specs))["mode"] == "persistent":
        # tile depths of the persistent kernel, tuned on the whole ensemble
        tuned = {k[0]: v for k, v in osb.autotune_batch(grids, trial_steps=2).items()}
    pts = sum(g.cfg.n for g in grids)
    osb.batch_step(grids, 2)              # warm-up (kernels, step graphs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    osb.batch_step(grids, steps)          # synchronises internally
    t_batch = time.perf_counter() - t0
    for g in grids:                       # the same work as per-grid launches
        g.step(1)
    seq_steps = min(steps, 20)            # per-grid launches: a rate, over fewer steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(seq_steps):
        for g in grids:
            g.step(1)
    torch.cuda.synchronize()
    t_seq = (time.perf_counter() - t0) * steps / seq_steps
    ke = [g.diagnostics()["ke"] for g in grids[:4]]
    del grids
    torch.cuda.empty_cache()
    return {"instances": len(specs), "points": pts, "steps": steps, "tile_depth": tuned,
            "value": steps * 3 * pts / t_batch, "ms_per_step": 1e3 * t_batch / steps,
            "per_grid_launch_value": steps * 3 * pts / t_seq, "speedup_vs_per_grid_launches": t_seq / t_batch,
            "per_grid_launch_steps_timed": seq_steps,
            "ke_first4": ke, **ensemble_launches(precision, len(specs))}


def ensemble_launches(precision, count):
    """How the library runs an ensemble step (OSB_BATCH_MODE overrides the
    default): FP64 and FP32 in one persistent launch for all steps;
    double-float as each grid's own step graph (9 kernels; 3 for FP32 on
    request) replayed on 8 concurrent library streams, the grids spread over
    them by points."""
    mode = os.environ.get("OSB_BATCH_MODE") or ("streams" if precision == "df64" else "persistent")
    per_grid = (3 if precision == "fp32" else 9) * count
    if mode == "streams":
        return {"mode": "streams", "launches_per_step": f"{count} step graphs ({per_grid} kernels) on 8 streams",
                "per_grid_launches_per_step": per_grid, "items": "per-grid step graphs"}
    return {"mode": "persistent", "launches_per_step": "1 persistent launch for all steps",
            "per_grid_launches_per_step": (6 if precision == "fp32" else 9) * count,
            "items": "z-march column items" if precision == "fp32" else "three-kernel point items"}


def run_scalar(torch, osb, n, order, steps, warmup, peak):
    """Scalar advection-diffusion (the paper's Sections 3.1-3.2 equation) on a
    3D periodic grid: point-stages/s and the FP64 roofline of its one kernel
    (per point-stage 2 FMAs per tap on 3 axes, the centre multiply, the source
    and the two RK FMAs: 12 r + 6 flops)."""
    r = order // 2
    g = torch.Generator(device="cpu").manual_seed(11)
    phi = torch.randn((n, n, n), generator=g, dtype=torch.float64).cuda()
    src = torch.randn((n, n, n), generator=g, dtype=torch.float64).cuda()
    work = torch.empty(2 * n ** 3, dtype=torch.float64, device="cuda")
    adv, k, dt = (1.0, -0.5, 0.25), 0.75, 1e-4
    osb.scalar_rk3(phi, work, order, adv, k, dt, warmup, src)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    osb.scalar_rk3(phi, work, order, adv, k, dt, steps, src)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    flops = (12 * r + 6) * 3 * n ** 3 * steps
    del phi, src, work
    torch.cuda.empty_cache()
    return {"value": 3 * n ** 3 * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "fp64_tflops": flops / (ms * 1e-3) / 1e12, "fp64_frac": flops / (ms * 1e-3) / 1e12 / peak,
            "hbm_gbs_min_traffic": 40 * 3 * n ** 3 * steps / (ms * 1e-3) / 1e9,
            "flops_per_point_stage": 12 * r + 6, "steps": steps}


def run_ours(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1609_01277_gb300 import build, inputs
    build.build()
    from paper_1609_01277_gb300 import osb
    osb.load()
    w = workload(args)
    n = w["n"]
    npts = n ** 3
    r = w["order"] // 2
    noise = inputs.gaussian_noise(n, n, n, w["noise_seed"] + rank)
    noise_dev = torch.from_numpy(noise).cuda()
    g = make_grid(osb, w, w["order"], w["precision"], noise_dev)

    clocks = Clocks(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    g.step(args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks.start()
    ms, prof = time_steps(torch, g, args.steps, 0, profile=True)
    clk = clocks.stop()
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    units = world * args.steps * 3 * npts
    value = units / (ms_max * 1e-3)

    # roofline of the dominant kernel (the residual + update kernel)
    pk = peaks()
    fl = stage_flops_per_point(r)
    res = prof["resid"]
    avg_ms = res["total_ms"] / max(res["launches"], 1)
    if w["precision"] == "fp64":
        achieved = fl["resid"] * npts / (avg_ms * 1e-3) / 1e12
        roof = {"kernel": "k_resid", "bound": "alu", "achieved": achieved, "peak": pk["fp64_tflops"],
                "unit": "TFLOP/s", "frac": achieved / pk["fp64_tflops"],
                "traffic": TRAFFIC_PER_LAUNCH.get((w["workload"], "k_resid")),
                "peak_src": "FP64 FMA rate from unit counts and clock: 2 DFMA/SM/cycle x 2 flops x 152 SMs x 2070 MHz",
                "flops_per_point": fl["resid"]}
    else:
        kname = fp32_kernel(w["order"])
        achieved = ALG_BYTES["fp32"] * npts / (avg_ms * 1e-3) / 1e9
        design = DESIGN_BYTES_FP32["fused" if kname == "k_fused" else "zmarch"]
        roof = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                "traffic": TRAFFIC_PER_LAUNCH.get((w["workload"], kname)),
                "peak_src": pk["src"],
                "design_bytes_per_point_stage": design,
                "design_bytes_gbs": design * npts / (avg_ms * 1e-3) / 1e9}
    if w["precision"] == "fp64":
        # the same kernel against the FP64 rate measured by the probe kernel
        meas = osb.fp64_rate()
        roof["peak_measured"] = meas["tflops"]
        roof["frac_vs_measured"] = achieved / meas["tflops"]
        roof["peak_measured_src"] = ("osb_fp64_rate_probe: 8 independent FMA chains per thread, "
                                     f"{meas['blocks']} blocks of 256, CUDA events, best of 5")
    kernel_ms = {k: v["total_ms"] / max(v["launches"], 1) for k, v in prof.items()}
    stage_ms = sum(kernel_ms.values())
    roof["kernel_avg_ms"] = kernel_ms
    roof["stage_hbm_frac"] = ALG_BYTES[w["precision"]] * npts / (stage_ms * 1e-3) / 1e9 / pk["hbm_gbs"]

    # end to end through the C ABI with pinned host buffers, copies every step
    e2e = None
    if not args.no_e2e:
        import numpy as np
        host = torch.empty((5, n, n, n), dtype=torch.float64).pin_memory()
        hq = host.numpy()
        g.get_state(hq)
        torch.cuda.synchronize()
        ke = max(2, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(ke):
            g.set_state(hq)
            g.step(1)
            g.get_state(hq)
        el = time.perf_counter() - t0
        if world > 1:
            tt = torch.tensor([el], dtype=torch.float64, device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            el = float(tt.item())
        nbytes = 5 * npts * 8
        e2e = {"value": world * ke * 3 * npts / el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": ke}
        del host

    variants = {}
    if not args.no_variants and world == 1:
        ref_ke = {}
        combos = [(o, p) for o in (4, 8) for p in ("fp64", "fp32")]
        for order, prec in combos:
            if order == w["order"] and prec == w["precision"]:
                vms, vprof = ms, prof
            else:
                gv = make_grid(osb, w, order, prec, noise_dev)
                vms, vprof = time_steps(torch, gv, args.steps, args.warmup, profile=True)
                del gv
            vr = vprof["resid"]
            vavg = vr["total_ms"] / max(vr["launches"], 1)
            vstage = sum(v["total_ms"] / max(v["launches"], 1) for v in vprof.values())
            ent = {"value": args.steps * 3 * npts / (vms * 1e-3), "ms_per_step": vms / args.steps,
                   "stage_ms": vstage, "resid_ms": vavg,
                   "stage_hbm_frac": ALG_BYTES[prec] * npts / (vstage * 1e-3) / 1e9 / pk["hbm_gbs"]}
            if prec == "fp64":
                ent["resid_fp64_tflops"] = stage_flops_per_point(order // 2)["resid"] * npts / (vavg * 1e-3) / 1e12
            # KE-decay error against the FP64 run of the same order over a few steps
            nke = min(args.steps, 10)
            gk = make_grid(osb, w, order, prec, noise_dev)
            series = ke_series(torch, gk, nke)
            del gk
            ref_ke.setdefault(order, {})[prec] = series
            variants[f"order{order}_{prec}"] = ent
        for order in (4, 8):
            a, b = ref_ke[order]["fp32"], ref_ke[order]["fp64"]
            err = max(abs(x - y) for x, y in zip(a, b)) / b[0]
            variants[f"order{order}_fp32"]["ke_err_vs_fp64"] = err
            variants[f"order{order}_fp32"]["speedup_vs_fp64"] = (
                variants[f"order{order}_fp32"]["value"] / variants[f"order{order}_fp64"]["value"])
        # double-float arithmetic (FP64-class accuracy on the FP32 pipes)
        for order in (4, 8):
            gd = make_grid(osb, w, order, "df64", noise_dev)
            dms, dprof = time_steps(torch, gd, args.steps, args.warmup, profile=True)
            del gd
            gk = make_grid(osb, w, order, "df64", noise_dev)
            series = ke_series(torch, gk, min(args.steps, 10))
            del gk
            b = ref_ke[order]["fp64"]
            variants[f"order{order}_df64"] = {
                "value": args.steps * 3 * npts / (dms * 1e-3), "ms_per_step": dms / args.steps,
                "kernel_avg_ms": {k: v["total_ms"] / max(v["launches"], 1) for k, v in dprof.items()},
                "ke_err_vs_fp64": max(abs(x - y) for x, y in zip(series, b)) / b[0],
                "speedup_vs_fp64": args.steps * 3 * npts / (dms * 1e-3) / variants[f"order{order}_fp64"]["value"]}
            torch.cuda.empty_cache()

    if not args.no_ensemble and world == 1:
        for prec in ("fp64", "fp32", "df64"):
            variants[f"ensemble64_order4_{prec}"] = run_ensemble(torch, osb, inputs, args.ensemble_steps, prec)
        e64, e32 = variants["ensemble64_order4_fp64"], variants["ensemble64_order4_fp32"]
        e32["speedup_vs_fp64_ensemble"] = e32["value"] / e64["value"]
        e32["ke_err_vs_fp64_first4"] = max(abs(a - b) / b for a, b in zip(e32["ke_first4"], e64["ke_first4"]))
        edd = variants["ensemble64_order4_df64"]
        edd["speedup_vs_fp64_ensemble"] = edd["value"] / e64["value"]
        edd["ke_err_vs_fp64_first4"] = max(abs(a - b) / b for a, b in zip(edd["ke_first4"], e64["ke_first4"]))
        # FP32 grids' own step graphs (fused stage) on concurrent streams, beside
        # the persistent launch of the stated configuration
        prev = os.environ.get("OSB_BATCH_MODE")
        os.environ["OSB_BATCH_MODE"] = "streams"
        try:
            es = run_ensemble(torch, osb, inputs, args.ensemble_steps, "fp32")
        finally:
            if prev is None:
                os.environ.pop("OSB_BATCH_MODE", None)
            else:
                os.environ["OSB_BATCH_MODE"] = prev
        es["speedup_vs_fp64_ensemble"] = es["value"] / e64["value"]
        es["speedup_vs_persistent_fp32"] = es["value"] / e32["value"]
        es["ke_err_vs_fp64_first4"] = max(abs(a - b) / b for a, b in zip(es["ke_first4"], e64["ke_first4"]))
        variants["ensemble64_order4_fp32_streams"] = es

    if not args.no_variants and world == 1:
        # viscous-work form B (product rule) and forward Euler, FP64 order 4
        gB = osb.Grid(osb.Config(n, n, n, order=4, precision=osb.OSB_FP64, visc_form=osb.OSB_VISC_B, Re=w["Re"],
                                 Mach=w["Mach"], gamma=w["gamma"], Pr=w["Pr"], dt=w["dt"]))
        gB.init_taylor_green(noise_dev, w["noise_amp"])
        msB, _ = time_steps(torch, gB, args.steps, args.warmup)
        del gB
        variants["order4_fp64_viscB"] = {"value": args.steps * 3 * npts / (msB * 1e-3), "ms_per_step": msB / args.steps}
        gE = make_grid(osb, w, 4, "fp64", noise_dev)
        gE.euler_step(args.warmup)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(gE.stream)
        gE.euler_step(args.steps)
        e1.record(gE.stream)
        torch.cuda.synchronize()
        msE = e0.elapsed_time(e1)
        del gE
        variants["euler_order4_fp64"] = {"value": args.steps * npts / (msE * 1e-3), "ms_per_step": msE / args.steps,
                                         "stages_per_step": 1}
        # the 32^3 parity case (20 steps of dt 3.385e-3, no noise): it fits in
        # L2, so it is a latency figure, not a roofline one
        g32 = osb.Grid(osb.Config(32, 32, 32, order=4, precision=osb.OSB_FP64, Re=w["Re"], Mach=w["Mach"],
                                  gamma=w["gamma"], Pr=w["Pr"], dt=3.385e-3))
        g32.init_taylor_green()
        ms32, _ = time_steps(torch, g32, 20, args.warmup)
        del g32
        variants["tgv_32^3_order4_fp64_20steps"] = {
            "value": 20 * 3 * 32 ** 3 / (ms32 * 1e-3), "ms_per_step": ms32 / 20,
            "note": "3 stages x 3 kernels per step, replayed as one CUDA graph per step"}
        # kinetic energy and enstrophy of every step, fused into the first stage
        for prec in ("fp64", "fp32"):
            gD = make_grid(osb, w, 4, prec, noise_dev)
            gD.set_diag_series(args.steps + args.warmup)
            msD, _ = time_steps(torch, gD, args.steps, args.warmup)
            del gD
            base = variants.get(f"order4_{prec}", {}).get("ms_per_step")
            variants[f"order4_{prec}_with_diag_series"] = {
                "value": args.steps * 3 * npts / (msD * 1e-3), "ms_per_step": msD / args.steps,
                "overhead_vs_plain": (msD / args.steps) / base - 1.0 if base else None}
        # the Taylor-Green vortex of the full 2 pi box computed on one octant
        # between its symmetry planes: (n/2)^3 points, mirrored stencil loads
        h = n // 2
        gS = osb.Grid(osb.Config(h, h, h, order=4, precision=osb.OSB_FP64, Re=w["Re"], Mach=w["Mach"],
                                 gamma=w["gamma"], Pr=w["Pr"], dt=w["dt"],
                                 bc=(osb.OSB_BC_SYMMETRIC,) * 3))
        gS.init_taylor_green()
        msS, _ = time_steps(torch, gS, args.steps, args.warmup)
        del gS
        vS = args.steps * 3 * h ** 3 / (msS * 1e-3)
        variants[f"tgv_octant_{h}^3_symmetric_order4_fp64"] = {
            "value": vS, "ms_per_step": msS / args.steps,
            "full_box_point_stages_per_s": 8 * vS,
            "time_vs_full_box_periodic": msS / variants["order4_fp64"]["ms_per_step"] / args.steps
            if "order4_fp64" in variants else None}
        torch.cuda.empty_cache()
        variants["scalar_advdiff_256^3_order8_fp64"] = run_scalar(torch, osb, n=256, order=8, steps=args.steps,
                                                                  warmup=args.warmup, peak=pk["fp64_tflops"])

    if not args.no_closure and world == 1:
        from paper_1609_01277_gb300 import closure as clo
        r = clo.run_experiment(n_fine=128, factor=4, t_end=4.0, snap_every=48, epochs=20)
        keep = {k: v for k, v in r.items() if k != "curves"}
        best = r["closure"]["momentum_half"]
        keep["summary"] = {
            "case": "reduced: 128^3 fine run filtered to 32^3, t <= 4 (the stated 512^3 -> 64^3, t <= 10 case "
                    "needs a ~10 min fine run and is not timed here: python -m paper_1609_01277_gb300.closure "
                    "--fine 512 --factor 8 --t-end 10)",
            "closure_beats_plain_ke": bool(best["ke_err_vs_filtered_fine"] < r["plain"]["ke_err_vs_filtered_fine"]),
            "closure_beats_plain_dissipation": bool(best["dissipation_err"] < r["plain"]["dissipation_err"]),
            "reference": "KE of the box-filtered 128^3 run on the 32^3 grid",
            "ke_err_plain_32": r["plain"]["ke_err_vs_filtered_fine"],
            "ke_err_closure_32": best["ke_err_vs_filtered_fine"],
            "dissipation_err_plain_32": r["plain"]["dissipation_err"],
            "dissipation_err_closure_32": best["dissipation_err"],
            "closure_cost_vs_plain_32": best["seconds"] / r["plain"]["seconds"],
            "speedup_vs_filtered_fine_run": r["seconds"]["fine_data"] / best["seconds"],
            "fallback_t": best["fallback_t"],
            # the stated case is not rerun here (its 512^3 fine run takes ~10 min)
            "stated_case_512to64_t10": {
                "source": "separate run of python -m paper_1609_01277_gb300.closure --fine 512 --factor 8 --t-end 10",
                "closure_beats_plain": False, "correction": "momentum, half gain (as in the reduced case)",
                "a_priori_err": 0.135,
                "ke_err_plain_64": 0.0180, "ke_err_closure_64": 0.0380,
                "dissipation_err_plain_64": 0.165, "dissipation_err_closure_64": 0.924,
                "fallback_t": 2.15, "fine_run_s": 460.0, "train_s": 4.3}}
        # the network's kernels on their own: forward and loss + gradient at 128^3
        from paper_1609_01277_gb300 import experiments as ex
        kt = ex.closure_timing(128, reps=10)
        keep["summary"].update({
            "forward_ms_128": kt["forward_ms"], "loss_grad_ms_128": kt["loss_grad_ms"],
            "forward_tflops_128": kt["forward_tflops"],
            "forward_bf16_frac": kt["forward_tflops"] / pk["bf16_tflops"],
            "forward_flops": "2 x 27 x (5*32 + 32*32 + 32*5) per point (the network's, unpadded)"})
        variants["closure_tgv128to32"] = keep

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = time_oracle(w, single_core=True)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if w["precision"] == "fp64" else "f32",
                "data": "synthetic",
                "config": {"workload": w["workload"], "grid": [n, n, n], "order": w["order"],
                           "precision": w["precision"], "Re": w["Re"], "Mach": w["Mach"], "gamma": w["gamma"],
                           "Pr": w["Pr"], "dt": w["dt"], "noise": "seeded N(0,1) x 1e-4 on u_i",
                           "l2": f"inputs larger than L2 ({osb_bytes(w)/1e9:.1f} GB resident)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": 9 * args.steps, "variants_summary": summarize_variants(variants),
                "variants": variants}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def summarize_variants(variants):
    """A compact copy of the headline figures of every variant (rate, step
    time, fraction of the HBM roofline on the fused-minimum bytes, KE-decay
    error against FP64), ahead of the full variant records."""
    out = {}
    keys = ("value", "ms_per_step", "stage_hbm_frac", "ke_err_vs_fp64", "speedup_vs_fp64", "resid_fp64_tflops")
    for name, v in variants.items():
        if name.startswith("order") or name.startswith("euler") or name.startswith("tgv_"):
            out[name] = {k: v[k] for k in keys if k in v and v[k] is not None}
        elif name.startswith("ensemble"):
            out[name] = {k: v[k] for k in ("value", "ms_per_step", "steps", "mode", "speedup_vs_per_grid_launches",
                                           "speedup_vs_fp64_ensemble", "speedup_vs_persistent_fp32",
                                           "ke_err_vs_fp64_first4") if k in v}
        elif name.startswith("scalar"):
            out[name] = {k: v[k] for k in ("value", "fp64_frac") if k in v}
        elif name.startswith("closure") and "summary" in v:
            out[name] = v["summary"]
    return out


def osb_bytes(w):
    n = w["n"] ** 3
    es = 8 if w["precision"] == "fp64" else 4
    return 10 * n * 8 + 10 * n * es + 15 * n * es


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
