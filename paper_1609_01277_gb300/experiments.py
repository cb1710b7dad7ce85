"""Long Taylor-Green runs on the GPU (Section 3.3): the kinetic energy E_k(t),
the enstrophy and the dissipation rate eps = -dE_k/dt of the FP64 and FP32
paths, the KE-decay error of FP32 against FP64, and the per-field state error
of FP32 against FP64 after a fixed number of steps.

Every step runs in the library's kernels; this module only drives grids and
reads their FP64 diagnostics.  CLI:

    python -m paper_1609_01277_gb300.experiments curves --n 256 --order 4 --t-end 20
    python -m paper_1609_01277_gb300.experiments fp32-error --n 512 --order 8 --steps 200
    python -m paper_1609_01277_gb300.experiments scalar --n 256 --order 8 --steps 20
    python -m paper_1609_01277_gb300.experiments steps --n 256 --order 4 --precision df64
    python -m paper_1609_01277_gb300.experiments closure --n 64
"""
from __future__ import annotations

import argparse
import os
import json
import time

import numpy as np

DT_64 = 3.385e-3  # time step of the 64^3 case (Section 3.3); halved per doubling of N


def default_dt(n: int) -> float:
    return DT_64 * 64.0 / n


def _grid(osb, torch, n, order, precision, dt, seed, amp, Re=1600.0, Mach=0.1):
    from . import inputs
    cfg = osb.Config(n, n, n, order=order, precision=precision, Re=Re, Mach=Mach, dt=dt)
    g = osb.Grid(cfg)
    noise = torch.from_numpy(inputs.gaussian_noise(n, n, n, seed)).cuda() if amp > 0 else None
    g.init_taylor_green(noise, amp)
    return g


def tgv_curves(n: int, order: int, precision: str, t_end: float, every: int = 50, dt: float | None = None,
               seed: int = 1234, amp: float = 1e-4) -> dict:
    """E_k, enstrophy and max CFL every `every` steps up to t_end, and E_k and
    enstrophy of every step (the series fused into the first RK stage)."""
    import torch
    from . import osb
    osb.load()
    dt = dt or default_dt(n)
    prec = osb.OSB_FP64 if precision == "fp64" else osb.OSB_FP32
    g = _grid(osb, torch, n, order, prec, dt, seed, amp)
    nsteps = int(round(t_end / dt))
    t, ke, ens, cfl = [], [], [], []
    step_series = []
    d = g.diagnostics()
    t.append(d["t"]), ke.append(d["ke"]), ens.append(d["enstrophy"]), cfl.append(d["max_cfl"])
    g.set_diag_series(every)
    done = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while done < nsteps:
        k = min(every, nsteps - done)
        g.step(k)
        done += k
        step_series.append(g.diag_series()[-k:])
        d = g.diagnostics()
        t.append(d["t"]), ke.append(d["ke"]), ens.append(d["enstrophy"]), cfl.append(d["max_cfl"])
    seconds = time.perf_counter() - t0
    del g
    torch.cuda.empty_cache()
    # per step: the state at the start of steps 0 .. nsteps-1, plus the final state
    ser = np.concatenate(step_series)
    ke_step = ser[:, 0].tolist() + [ke[-1]]
    ens_step = ser[:, 1].tolist() + [ens[-1]]
    return dict(n=n, order=order, precision=precision, dt=dt, steps=nsteps, every=every, t=t, ke=ke,
                enstrophy=ens, max_cfl=cfl, seconds=seconds, point_stages_per_s=3.0 * n ** 3 * nsteps / seconds,
                t_step=[i * dt for i in range(nsteps + 1)], ke_step=ke_step, enstrophy_step=ens_step)


def dissipation(t, ke):
    """eps = -dE_k/dt by second-order central differences (one-sided at the ends)."""
    t, ke = np.asarray(t), np.asarray(ke)
    return -np.gradient(ke, t)


def write_series_csv(path: str, ke, enstrophy, dt: float, Re: float, step0: int = 0) -> None:
    """The per-step diagnostics series as CSV, one row per step: step, t,
    E_k, enstrophy, the dissipation rate eps = -dE_k/dt (second-order central
    differences, one-sided at the ends; empty for a single row) and its
    viscous estimate (2/Re) * enstrophy (Section 3.3 quantities)."""
    ke = np.asarray(ke, dtype=float)
    ens = np.asarray(enstrophy, dtype=float)
    if ke.shape != ens.shape or ke.ndim != 1:
        raise ValueError("ke and enstrophy must be 1-D series of the same length")
    t = (step0 + np.arange(ke.size)) * dt
    eps = dissipation(t, ke) if ke.size >= 2 else np.full(ke.size, np.nan)
    with open(path, "w") as f:
        f.write("step,t,ke,enstrophy,dissipation,visc_dissipation\n")
        for i in range(ke.size):
            e = "" if np.isnan(eps[i]) else f"{eps[i]:.17g}"
            f.write(f"{step0 + i},{t[i]:.17g},{ke[i]:.17g},{ens[i]:.17g},{e},{2.0 * ens[i] / Re:.17g}\n")


def summarize(c: dict) -> dict:
    # every step where the series is FP64-exact (the FP32 path evaluates it
    # from its FP32 stencil source: ~1e-7 relative noise, which a per-step
    # difference quotient would amplify); else the FP64 reductions every
    # `every` steps
    if "ke_step" in c and c["precision"] != "fp32":
        t, ke, ens = np.asarray(c["t_step"]), np.asarray(c["ke_step"]), np.asarray(c["enstrophy_step"])
    else:
        t, ke, ens = np.asarray(c["t"]), np.asarray(c["ke"]), np.asarray(c["enstrophy"])
    eps = dissipation(t, ke)
    i_eps, i_ens = int(np.argmax(eps)), int(np.argmax(ens))
    at = {}
    for tt in (0.0, 3.0, 5.0, 9.0, 10.0, 15.0, 20.0):
        if tt <= t[-1] + 1e-9:
            j = int(np.argmin(np.abs(t - tt)))
            at[f"{tt:g}"] = dict(ke=float(ke[j]), eps=float(eps[j]), enstrophy=float(ens[j]),
                                 two_over_re_enstrophy=float(2.0 / 1600.0 * ens[j]))
    return dict(n=c["n"], order=c["order"], precision=c["precision"], steps=c["steps"], dt=c["dt"],
                seconds=c["seconds"], point_stages_per_s=c["point_stages_per_s"],
                ke_drop_by_t3=float(1.0 - ke[int(np.argmin(np.abs(t - 3.0)))] / ke[0]) if t[-1] >= 3 else None,
                t_max_dissipation=float(t[i_eps]), max_dissipation=float(eps[i_eps]),
                t_max_enstrophy=float(t[i_ens]), max_enstrophy=float(ens[i_ens]),
                max_cfl=float(np.max(c["max_cfl"])), at=at)


def compare_curves(a: dict, ref: dict) -> dict:
    """KE-decay error of run a against the reference run: max_t |E_k - E_k^ref| / E_k^ref(0),
    and the same for the dissipation rate relative to its peak."""
    ka, kr = np.asarray(a["ke"]), np.asarray(ref["ke"])
    ea, er = dissipation(a["t"], ka), dissipation(ref["t"], kr)
    out = dict(ke_err=float(np.max(np.abs(ka - kr)) / kr[0]),
               eps_err=float(np.max(np.abs(ea - er)) / np.max(np.abs(er))),
               speedup=ref["seconds"] / a["seconds"])
    if "ke_step" in a and "ke_step" in ref:
        # the same maximum over every step (fused series)
        sa, sr = np.asarray(a["ke_step"]), np.asarray(ref["ke_step"])
        out["ke_err_every_step"] = float(np.max(np.abs(sa - sr)) / sr[0])
    return out


def fp32_error(n: int, order: int, steps: int, dt: float | None = None, seed: int = 1234, amp: float = 1e-4) -> dict:
    """Relative L2 error of every conserved field of the FP32 path against the
    FP64 path after `steps` steps from the same state (momentum fields relative
    to the norm of the whole momentum, which starts with rho w = 0)."""
    import torch
    from . import osb
    osb.load()
    dt = dt or default_dt(n)
    out = {}
    states = {}
    for name, prec in (("fp64", osb.OSB_FP64), ("fp32", osb.OSB_FP32)):
        g = _grid(osb, torch, n, order, prec, dt, seed, amp)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(steps)
        torch.cuda.synchronize()
        out[f"{name}_seconds"] = time.perf_counter() - t0
        states[name] = g.get_state_device()
        del g
    a, b = states["fp32"], states["fp64"]
    mnorm = float(torch.linalg.vector_norm(b[1:4]))
    names = ("rho", "rho_u", "rho_v", "rho_w", "rho_E")
    for m in range(5):
        scale = mnorm if 1 <= m <= 3 else float(torch.linalg.vector_norm(b[m]))
        out[f"rel_l2_{names[m]}"] = float(torch.linalg.vector_norm(a[m] - b[m])) / scale
    out.update(n=n, order=order, steps=steps, dt=dt)
    return out


def scalar_timing(n: int, order: int, steps: int, warmup: int = 3) -> dict:
    """Scalar advection-diffusion (Sections 3.1-3.2 equation) on an n^3 grid:
    CUDA-event time of `steps` RK3 steps after `warmup` steps."""
    import torch
    from . import osb
    osb.load()
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
    r = order // 2
    return dict(n=n, order=order, steps=steps, ms_per_step=ms / steps,
                point_stages_per_s=3 * n ** 3 * steps / (ms * 1e-3),
                fp64_tflops=(12 * r + 6) * 3 * n ** 3 * steps / (ms * 1e-3) / 1e12)


def step_timing(n: int, order: int, precision: str, steps: int, warmup: int = 3) -> dict:
    """Taylor-Green steps on an n^3 grid in the given precision (fp64, fp32,
    df64): CUDA-event time per step and per kernel kind."""
    import torch
    from . import inputs, osb
    osb.load()
    prec = {"fp64": osb.OSB_FP64, "fp32": osb.OSB_FP32, "df64": osb.OSB_DF64}[precision]
    g = osb.Grid(osb.Config(n, n, n, order=order, precision=prec, dt=default_dt(n)))
    g.init_taylor_green(torch.from_numpy(inputs.gaussian_noise(n, n, n, 1234)).cuda(), 1e-4)
    g.step(warmup)
    torch.cuda.synchronize()
    g.profile_start(3 * steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(g.stream)
    g.step(steps)
    e1.record(g.stream)
    torch.cuda.synchronize()
    prof = g.profile_stop()
    ms = e0.elapsed_time(e1)
    return dict(n=n, order=order, precision=precision, steps=steps, ms_per_step=ms / steps,
                point_stages_per_s=3 * n ** 3 * steps / (ms * 1e-3),
                kernel_ms={k: v["total_ms"] / max(v["launches"], 1) for k, v in prof.items()})


def ensemble_run(steps: int, precisions=("fp64", "fp32"), every: int = 50, count: int = 64, seed: int = 7,
                 autotune: bool = True) -> dict:
    """The uneven Taylor-Green ensemble (64 grids of 32^3..128^3, Re in
    [100, 3200], M in [0.05, 0.3], order 4) advanced `steps` RK3 steps by
    osb_batch_step in chunks of `every` (one call per chunk: FP64 one
    persistent launch, FP32 and double-float the grids' step graphs on
    concurrent streams), with every grid's E_k after each chunk.  Per precision: time, point-stages
    per second; FP32 against FP64: the KE-decay error max over grids and
    chunks of |E_k - E_k^FP64| / E_k^FP64(0), and the speed-up."""
    import torch
    from . import inputs, osb
    osb.load()
    specs = inputs.ensemble_with_dt(count, seed)
    out = {}
    for precision in precisions:
        prec = {"fp64": osb.OSB_FP64, "fp32": osb.OSB_FP32, "df64": osb.OSB_DF64}[precision]
        grids = []
        for i, e in enumerate(specs):
            n = e["n"]
            g = osb.Grid(osb.Config(n, n, n, order=4, precision=prec, Re=e["Re"], Mach=e["Mach"], dt=e["dt"]))
            g.init_taylor_green(torch.from_numpy(inputs.gaussian_noise(n, n, n, 1000 + i)).cuda(), 1e-4)
            grids.append(g)
        tuned = {}
        mode = os.environ.get("OSB_BATCH_MODE") or ("streams" if precision == "df64" else "persistent")
        if autotune and mode == "persistent":  # tile depths of the persistent kernel, tuned on the ensemble
            tuned = {k[0]: v for k, v in osb.autotune_batch(grids, trial_steps=2).items()}
        ke = [[g.diagnostics()["ke"] for g in grids]]
        seconds, done = 0.0, 0
        while done < steps:
            k = min(every, steps - done)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            osb.batch_step(grids, k)
            seconds += time.perf_counter() - t0
            done += k
            ke.append([g.diagnostics()["ke"] for g in grids])
        pts = sum(g.cfg.n for g in grids)
        out[precision] = dict(steps=steps, points=pts, seconds=seconds, tile_depth=tuned,
                              point_stages_per_s=3.0 * pts * steps / seconds, ke=ke)
        del grids
        torch.cuda.empty_cache()
    if "fp64" in out:
        ref = np.asarray(out["fp64"]["ke"])
        for p in out:
            if p == "fp64":
                continue
            k = np.asarray(out[p]["ke"])
            out[p]["ke_err_vs_fp64"] = float(np.max(np.abs(k - ref) / ref[0][None, :]))
            out[p]["speedup_vs_fp64"] = out["fp64"]["seconds"] / out[p]["seconds"]
    for p in out:
        out[p].pop("ke")
    return out


def closure_timing(n: int, reps: int, warmup: int = 2) -> dict:
    """Learned-closure network on an n^3 grid: CUDA-event time of one forward
    pass and of one loss + gradient evaluation (BF16 tensor-core convolutions),
    with the forward pass's dense flop count (2 x 27 taps x channel products
    per point: 5->32, 32->32, 32->5)."""
    import torch
    from . import closure as clo, inputs, osb
    osb.load()
    c = clo.Closure(n, n, n, seed=0)
    g = osb.Grid(osb.Config(n, n, n, order=4))
    g.init_taylor_green(torch.from_numpy(inputs.gaussian_noise(n, n, n, 3)).cuda(), 1e-3)
    Q = g.get_state_device()
    c.set_normalization(Q.mean(dim=(1, 2, 3)).cpu().numpy(), Q.std(dim=(1, 2, 3)).cpu().numpy() + 1e-6,
                        np.ones(5))
    Cstar = torch.zeros_like(Q)
    for _ in range(warmup):
        c.forward(Q)
        c.loss_grad(Q, Cstar)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    for _ in range(reps):
        c.forward(Q)
    e[1].record()
    for _ in range(reps):
        c.loss_grad(Q, Cstar)
    e[2].record()
    torch.cuda.synchronize()
    fwd_ms, bwd_ms = e[0].elapsed_time(e[1]) / reps, e[1].elapsed_time(e[2]) / reps
    flops = 2 * 27 * (5 * 32 + 32 * 32 + 32 * 5) * n ** 3
    return dict(n=n, forward_ms=fwd_ms, loss_grad_ms=bwd_ms, forward_gflop=flops / 1e9,
                forward_tflops=flops / (fwd_ms * 1e-3) / 1e12)


def fp64_peak(blocks: int, iters: int, repeats: int) -> dict:
    """The FP64 FMA rate measured by the library's probe kernel, with the SM
    clock sampled by nvidia-smi while it runs, next to the rate the unit
    counts give at the sampled clock (2 FP64 FMAs per SM per cycle)."""
    import subprocess
    import tempfile

    import torch
    from . import build, osb
    build.build()
    osb.load()
    torch.cuda.set_device(0)
    fd, path = tempfile.mkstemp(suffix=".csv")
    os.close(fd)
    proc = subprocess.Popen(["nvidia-smi", "--id=0", "--query-gpu=clocks.sm,clocks.max.sm",
                             "--format=csv,noheader,nounits", "-lms", "50"], stdout=open(path, "w"),
                            stderr=subprocess.DEVNULL)
    try:
        osb.fp64_rate(blocks, max(1, iters // 10), 1)  # warm-up, clocks ramp
        r = osb.fp64_rate(blocks, iters, repeats)
    finally:
        proc.terminate()
        proc.wait(timeout=5)
    sm = []
    with open(path) as f:
        for line in f:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 2 and parts[0].replace(".", "").isdigit():
                sm.append((float(parts[0]), float(parts[1])))
    os.unlink(path)
    busy = [a for a, _ in sm]
    med = sorted(busy)[len(busy) // 2] if busy else None
    props = torch.cuda.get_device_properties(0)
    r["sm_mhz_median"] = med
    r["sm_max_mhz"] = max((b for _, b in sm), default=None)
    r["sms"] = props.multi_processor_count
    if med:
        r["unit_count_tflops_at_sampled_clock"] = 2 * 2 * props.multi_processor_count * med * 1e6 / 1e12
    return r


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    c = sub.add_parser("curves")
    c.add_argument("--n", type=int, default=256)
    c.add_argument("--order", type=int, default=4)
    c.add_argument("--t-end", type=float, default=20.0)
    c.add_argument("--every", type=int, default=50)
    c.add_argument("--precisions", default="fp64,fp32")
    c.add_argument("--curves-out", default=None, help="write the full curves as JSON here")
    c.add_argument("--csv", default=None, help="write the per-step series of each precision as CSV "
                                               "(PATH with {precision} replaced)")
    sc = sub.add_parser("scalar")
    sc.add_argument("--n", type=int, default=256)
    sc.add_argument("--order", type=int, default=8)
    sc.add_argument("--steps", type=int, default=20)
    sc.add_argument("--warmup", type=int, default=3)
    st = sub.add_parser("steps")
    st.add_argument("--n", type=int, default=256)
    st.add_argument("--order", type=int, default=4)
    st.add_argument("--precision", default="df64", choices=("fp64", "fp32", "df64"))
    st.add_argument("--steps", type=int, default=10)
    st.add_argument("--warmup", type=int, default=3)
    cl = sub.add_parser("closure")
    cl.add_argument("--n", type=int, default=64)
    cl.add_argument("--reps", type=int, default=10)
    en = sub.add_parser("ensemble")
    en.add_argument("--steps", type=int, default=500)
    en.add_argument("--every", type=int, default=50)
    en.add_argument("--precisions", default="fp64,fp32")
    en.add_argument("--count", type=int, default=64)
    en.add_argument("--no-autotune", action="store_true")
    pk = sub.add_parser("fp64-peak")
    pk.add_argument("--blocks", type=int, default=152 * 8)
    pk.add_argument("--iters", type=int, default=2000)
    pk.add_argument("--repeats", type=int, default=5)
    e = sub.add_parser("fp32-error")
    e.add_argument("--n", type=int, default=512)
    e.add_argument("--order", type=int, default=8)
    e.add_argument("--steps", type=int, default=200)
    args = ap.parse_args(argv)
    if args.cmd == "curves":
        runs = {p: tgv_curves(args.n, args.order, p, args.t_end, args.every) for p in args.precisions.split(",")}
        res = {p: summarize(r) for p, r in runs.items()}
        if "fp64" in runs and "fp32" in runs:
            res["fp32_vs_fp64"] = compare_curves(runs["fp32"], runs["fp64"])
        if args.curves_out:
            with open(args.curves_out, "w") as f:
                json.dump(runs, f)
        if args.csv:
            for p, r in runs.items():
                write_series_csv(args.csv.replace("{precision}", p), r["ke_step"], r["enstrophy_step"], r["dt"],
                                 1600.0)
        print(json.dumps(res))
    elif args.cmd == "steps":
        print(json.dumps(step_timing(args.n, args.order, args.precision, args.steps, args.warmup)))
    elif args.cmd == "ensemble":
        print(json.dumps(ensemble_run(args.steps, tuple(args.precisions.split(",")), args.every, args.count,
                                      autotune=not args.no_autotune)))
    elif args.cmd == "closure":
        print(json.dumps(closure_timing(args.n, args.reps)))
    elif args.cmd == "fp64-peak":
        print(json.dumps(fp64_peak(args.blocks, args.iters, args.repeats)))
    elif args.cmd == "scalar":
        print(json.dumps(scalar_timing(args.n, args.order, args.steps, args.warmup)))
    else:
        print(json.dumps(fp32_error(args.n, args.order, args.steps)))


if __name__ == "__main__":
    main()
