"""Benchmark of the compressed patch-relaxation hot path on GB300.

One step = the whole path on one synthetic workload: setup (patch extraction,
multiplicity weights, Alg. 1 with the certified criterion, FP64 inverses of
the database entries, conversion to the storage precision, sweep layout) and
the outer solve (right-preconditioned FGMRES(30) or PCG, sweeps + SpMV +
orthogonalisation) from x0 = 0, inputs already resident in HBM.

Default workload: 2D Stokes, Taylor-Hood Q2-Q1 on 128 x 128 quads graded in y
(ratio 1.05), 22-DOF Vanka cell patches, FGMRES(30) in FP64, criterion tol
1e-2, representative inverses stored in FP32.  The one-level Vanka
preconditioner does not reach 1e-8 on this mesh within a practical budget, so
a step runs a fixed iteration budget (--maxit, default 300) and reports the
relative residual reached; the full-storage FP64 form is measured beside it.

value = n x (preconditioner applications in the step) / step time, i.e. the
Schwarz sweep DOF/s of the whole step with setup included (unit DOF/s).

Prints ONE JSON line (rank 0).  --impl reference times the CPU FP64 oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

METRIC = "Schwarz sweep DOF/s + setup s, clustered vs full, iters to 1e-8 rel. residual"

CONFIGS = {
    "stokes2d": dict(builder="stokes2d_q2q1", kw=dict(N=128, ratio=1.05), tol=1e-2, prec="fp32",
                     weighting="left", krylov="fgmres",
                     desc="2D Stokes Taylor-Hood Q2-Q1, 128x128 quads graded 1.05 in y, 22-DOF Vanka patches"),
    "poisson2d": dict(builder="poisson2d_q2", kw=dict(N=16), tol=1e-12, prec="fp64", weighting="sym",
                      krylov="cg", desc="2D Q2 diffusion 16x16, 9-DOF patches"),
    "nedelec3d": dict(builder="nedelec3d", kw=dict(N=64), tol=1e-1, prec="fp32", weighting="sym",
                      krylov="cg", desc="3D Nedelec curl-curl 64^3, 12-DOF patches"),
    "diffusion3d": dict(builder="diffusion3d_q2", kw=dict(N=32), tol=1e-1, prec="fp32", weighting="sym",
                        krylov="cg", desc="3D Q2 lognormal diffusion 32^3, 27-DOF patches"),
    "stokes3d": dict(builder="stokes3d_q2q1", kw=dict(N=24), tol=0.0, prec="fp32", weighting="left",
                     krylov="fgmres",
                     desc="3D Stokes Q2-Q1 24^3 hexes, vertex jitter 0.2h, Dirichlet-trimmed Vanka patches "
                          "{89, 62, 44, 32} in one grouped persistent sweep, full storage"),
}

# FP64 peak of one GB300 from its unit counts and clock: 152 SMs x 2 FP64
# fused multiply-adds per clock x 2 flops x 2.07 GHz (no measured FP64 peak
# is on record; a probe kernel of independent FMA chains reached 84 % of it)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12

# kernel(s) behind each timing class of the library's per-kernel timing
KT_KERNEL_NAMES = {"sweep": "patch sweep (k_sweep_staged / k_sweep_*)", "spmv": "k_spmv_sell (SELL SpMV, FP64)",
                   "mdot": "k_arnoldi (fused FGMRES Gram-Schmidt step on FP32 pairs) / k_mdot", "maxpy": "k_maxpy (FGMRES w -= V h)",
                   "vec": "vector kernels (k_fg_scale / CG updates)"}

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, ncu,
# averaged over the captured launches) for (config, class), valid only for
# the kernel source they were taken on; None until captured.
TRAFFIC = {
    # ncu --set full of the fused Gram-Schmidt step on pairs at j = 20
    # (26.30 MB: one DRAM read of the 21 pair rows and of w, later passes
    # from L2) scaled to the mean basis size of a step, (j+2) averaged over
    # j = 0..29
    ("stokes2d", "mdot"): 26.30e6 * 16.5 / 22.0,
    # ncu --set full, one launch inside the FGMRES cycle (k_spmv_sell):
    # 89.11 MB read + 2.47 MB written
    ("stokes2d", "spmv"): 91.6e6,
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="stokes2d", choices=sorted(CONFIGS))
    ap.add_argument("--maxit", type=int, default=300)
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--prec", default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--apply-reps", type=int, default=200)
    ap.add_argument("--mlp", action="store_true", help="learned-assignment gain on the 3D lognormal workload")
    ap.add_argument("--exp1", action="store_true",
                    help="Experiment 1: iterations of FGMRES(20) + M_combo for Q2..Q5 (Table 1 of the paper)")
    ap.add_argument("--tol-sweep", action="store_true",
                    help="compressibility curve: m_p, setup and residual per criterion tolerance and precision")
    ap.add_argument("--mlp-n", type=int, default=32)
    ap.add_argument("--mlp-epochs", type=int, default=300)
    ap.add_argument("--mlp-lr", type=float, default=1e-3)
    return ap.parse_args()


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def build_problem(cfg):
    import problems
    return getattr(problems, cfg["builder"])(**cfg["kw"])


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.p = None
        self.idx = gpu_index
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ replicas
def aggregate_replicas(seconds: float, units: float, device=None):
    """Whole-job throughput of independent replicas (one per rank, no
    collective on the data path): the units every rank processed, divided
    by the slowest rank's time.  Returns (value, max_seconds, total_units)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return units / seconds, seconds, units
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return u.item() / t.item(), t.item(), u.item()


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, cfg, ws, rank, local):
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2306_10025_gb300 as L

    torch.cuda.set_device(local)
    devc = torch.device("cuda", local)
    pr = build_problem(cfg)
    tol = cfg["tol"] if args.tol is None else args.tol
    prec = cfg["prec"] if args.prec is None else args.prec
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=devc)
    rp, ci, va = t(pr.rowptr, torch.int32), t(pr.colidx, torch.int32), t(pr.vals, torch.float64)
    dofs = t(pr.patch_dofs, torch.int32)
    offs = None if pr.uniform_size else t(pr.patch_offsets, torch.int32)
    b = t(pr.rhs(0), torch.float64)
    x = torch.zeros_like(b)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=devc)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def mk_opts(tol_, prec_):
        return L.make_opts(tol=tol_, store_prec=prec_, weighting=cfg["weighting"], krylov=cfg["krylov"],
                           restart=30, rtol=1e-8, maxit=args.maxit)

    def one_step(tol_, prec_):
        ctx = L.psr_setup(rp, ci, va, dofs, offsets=offs, uniform_size=pr.uniform_size, opts=mk_opts(tol_, prec_))
        info = ctx.solve(b, x)
        return ctx, info

    # warm-up
    for _ in range(args.warmup):
        ctx, info = one_step(tol, prec)
        ctx.destroy()
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    clk = ClockSampler(local)
    clk.start()
    launches0 = L.psr_kernel_launches()
    times, infos, stats = [], [], []
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    for _ in range(args.steps):
        flush.zero_()                               # L2 flush between steps (outside the timing)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx, info = one_step(tol, prec)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
        infos.append(info)
        stats.append(ctx.stats())
        if len(times) < args.steps:
            ctx.destroy()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches = L.psr_kernel_launches() - launches0
    clocks = clk.stop()
    step_s = sum(times) / len(times)
    iters = infos[-1]["iterations"]
    units_local = pr.n * sum(i["iterations"] for i in infos)
    value, total_s, _ = aggregate_replicas(sum(times), units_local, devc)

    # kernel-level: sweep (apply) timing with CUDA events over many launches
    last = ctx
    r = torch.randn(pr.n, dtype=torch.float64, device=devc)
    z = torch.empty_like(r)
    for _ in range(20):
        last.apply(r, z)
    big_r = [torch.randn(pr.n, dtype=torch.float64, device=devc) for _ in range(2)]
    torch.cuda.synchronize()
    ev = []
    for i in range(args.apply_reps):
        flush.zero_() if i % 8 == 0 else None
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        last.apply(big_r[i % 2], z)
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    apply_ms = sorted(a.elapsed_time(b_) for a, b_ in ev)
    apply_med = apply_ms[len(apply_ms) // 2] * 1e-3
    st = stats[-1]
    n, npch = pr.n, pr.n_patches
    psum = int(pr.patch_offsets[-1])
    eb = {"fp64": 8, "fp32": 4, "bf16": 2}[prec]
    ntile_bytes = 12 * (st["m_p"] + npch // 32 + 1)
    alg_bytes = 3 * 8 * n + 4 * psum + st["factor_bytes"] + ntile_bytes
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
    hbm = peaks.get("hbm_gbs", 6800.0)
    peak_source = "measured" if "hbm_gbs" in peaks else "fallback"
    sweep_alone = {"alg_bytes_per_launch": alg_bytes, "launch_us": apply_med * 1e6,
                   "achieved_gbs": alg_bytes / apply_med / 1e9, "frac": alg_bytes / apply_med / 1e9 / hbm}

    # per-kernel device time inside one more solve of the same step, from
    # CUDA events the library records around every per-iteration launch on
    # its stream (inside the cycle graph); the dominant class is the roofline
    last.set_kernel_timing(True)
    flush.zero_()
    last.solve(b, x)
    torch.cuda.synchronize()
    kt = last.kernel_timing()
    last.set_kernel_timing(False)
    kernels = {}
    for name, (ms, cnt, by, fl) in kt.items():
        if cnt:
            kernels[name] = {"launches": cnt, "ms": ms, "us_per_launch": 1e3 * ms / cnt,
                             "alg_bytes_per_launch": by / cnt, "achieved_gbs": by / (ms * 1e-3) / 1e9,
                             "frac": by / (ms * 1e-3) / 1e9 / hbm,
                             "fp64_flops_per_launch": fl / cnt, "achieved_fp64_tflops": fl / (ms * 1e-3) / 1e12,
                             "frac_fp64": fl / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS}
    tot_ms = sum(v["ms"] for v in kernels.values())
    for v in kernels.values():
        v["share"] = v["ms"] / tot_ms
    top = max(kernels, key=lambda k: kernels[k]["ms"])
    kd = kernels[top]
    # the binding resource of the dominant class: HBM bytes or FP64 flops,
    # whichever it uses the larger fraction of
    if kd["frac_fp64"] > kd["frac"]:
        bound = {"bound": "alu", "achieved": kd["achieved_fp64_tflops"], "peak": FP64_PEAK_TFLOPS,
                 "unit": "TFLOP/s (FP64)", "frac": kd["frac_fp64"],
                 "peak_source": "derived: 152 SMs x 2 FP64 FMA/clock x 2 flops x 2070 MHz"}
    else:
        bound = {"bound": "hbm", "achieved": kd["achieved_gbs"], "peak": hbm, "unit": "GB/s", "frac": kd["frac"],
                 "peak_source": peak_source}
    roofline = dict(kernel=KT_KERNEL_NAMES[top], **bound, traffic=TRAFFIC.get((args.config, top)),
                    alg_bytes_per_launch=kd["alg_bytes_per_launch"], hbm_frac=kd["frac"],
                    fp64_flops_per_launch=kd["fp64_flops_per_launch"], fp64_frac=kd["frac_fp64"],
                    launch_us=kd["us_per_launch"], share_of_iteration_kernels=kd["share"],
                    timing="CUDA events on the solve stream around each launch, one extra solve after the timed steps",
                    kernels=kernels, sweep_alone=sweep_alone)
    last.destroy()

    # full-storage FP64 comparison (outside the timed steps)
    ctx_f, info_f = one_step(0.0, "fp64")
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx_f2, info_f2 = one_step(0.0, "fp64")
    e1.record(stream)
    e1.synchronize()
    full_step_s = e0.elapsed_time(e1) * 1e-3
    st_f = ctx_f2.stats()
    ctx_f.destroy()
    ctx_f2.destroy()

    # end to end: host (pinned) inputs -> device -> setup + solve -> x to host
    e2e = None
    if not args.no_e2e:
        hp = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).pin_memory()
        h_rp, h_ci, h_va = hp(pr.rowptr, torch.int32), hp(pr.colidx, torch.int32), hp(pr.vals, torch.float64)
        h_d, h_b = hp(pr.patch_dofs, torch.int32), hp(pr.rhs(0), torch.float64)
        h_o = None if pr.uniform_size else hp(pr.patch_offsets, torch.int32)
        h_x = torch.empty(n, dtype=torch.float64).pin_memory()
        h2d = sum(a.numel() * a.element_size() for a in (h_rp, h_ci, h_va, h_d, h_b) ) + (0 if h_o is None else h_o.numel() * 4)
        ets = []
        for i in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d_rp, d_ci, d_va = h_rp.to(devc, non_blocking=True), h_ci.to(devc, non_blocking=True), h_va.to(devc, non_blocking=True)
            d_d, d_b = h_d.to(devc, non_blocking=True), h_b.to(devc, non_blocking=True)
            d_o = None if h_o is None else h_o.to(devc, non_blocking=True)
            d_x = torch.zeros(n, dtype=torch.float64, device=devc)
            c2 = L.psr_setup(d_rp, d_ci, d_va, d_d, offsets=d_o, uniform_size=pr.uniform_size, opts=mk_opts(tol, prec))
            inf2 = c2.solve(d_b, d_x)
            h_x.copy_(d_x, non_blocking=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            c2.destroy()
            if i >= args.warmup:
                ets.append(dt)
        e2e = {"value": n * inf2["iterations"] / (sum(ets) / len(ets)), "unit": "DOF/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(n * 8),
               "ms_per_step": 1e3 * sum(ets) / len(ets)}

    out = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * step_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+" + prec, "data": "synthetic",
        "config": {"workload": cfg["desc"], "n": n, "n_patches": npch, "tol": tol, "store_prec": prec,
                   "krylov": cfg["krylov"] + ("(30)" if cfg["krylov"] == "fgmres" else ""),
                   "weighting": cfg["weighting"], "maxit": args.maxit, "rhs": "uniform(-1,1) seed 0",
                   "l2": "flushed (256 MB write) before every timed step",
                   "allocations": "library caching allocator, filled by the warm-up steps",
                   "value_def": "n x preconditioner applications / step time (setup + solve)",
                   "parallelism": f"replicas x{ws}"},
        "setup_s": {"clustered": st["t_extract"] + st["t_rounds"] + st["t_convert"],
                    "full": st_f["t_extract"] + st_f["t_rounds"] + st_f["t_convert"],
                    "clustered_phases": {k: st[k] for k in ("t_extract", "t_rounds", "t_convert")}},
        "iters": {"clustered": iters, "full": info_f2["iterations"], "relres_clustered": infos[-1]["relres"],
                  "relres_full": info_f2["relres"], "converged_clustered": infos[-1]["converged"],
                  "converged_full": info_f2["converged"], "rtol": 1e-8},
        "step_s": {"clustered": step_s, "full_fp64": full_step_s},
        "sweep_dof_per_s": n / apply_med,
        "m_p": st["m_p"], "retained_fraction": st["m_p"] / npch,
        "factor_bytes": {"clustered": st["factor_bytes"], "full": st_f["factor_bytes"]},
        "criterion_evals": st["criterion_evals"], "criterion_exact": st["criterion_exact"], "criterion_screened": st["criterion_screened"],
        "roofline": roofline, "clocks": clocks, "e2e": e2e, "gpu_launches": launches,
    }
    return out, pr, infos[-1], st


# ------------------------------------------------------------------ CPU oracle
SAMPLE_KW = {"stokes2d": dict(N=16, ratio=1.05), "poisson2d": dict(N=16), "nedelec3d": dict(N=8),
             "diffusion3d": dict(N=6), "stokes3d": dict(N=4)}


def cpu_oracle_sample(args, cfg, name):
    """The numpy FP64 oracle, as it stands, on a bounded sample of the same
    workload: the same family, solver and options on a smaller mesh, the
    whole step (setup with Alg. 1 + outer solve with the same iteration
    budget).  Returns the line's cpu_baseline object (same unit)."""
    import problems
    from oracle import psr_oracle as O
    kw = SAMPLE_KW[name]
    pr = getattr(problems, cfg["builder"])(**kw)
    tol = cfg["tol"] if args.tol is None else args.tol
    t0 = time.perf_counter()
    if pr.uniform_size:
        st = O.setup(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.dofs2d(), tol)
        t1 = time.perf_counter()
        x, hist, it, conv = O.solve(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.rhs(0), st, cfg["krylov"],
                                    cfg["weighting"], restart=30, rtol=1e-8, maxit=args.maxit)
    else:
        # patches of several sizes, full storage (the criterion path takes one size)
        Ak = O.extract_patches_ragged(pr.rowptr, pr.colidx, pr.vals, pr.n, pr.patch_offsets, pr.patch_dofs)
        Binv = [O.lu_inverse(a[None])[0][0] for a in Ak]
        W = O.weights(O.multiplicity(pr.n, pr.patch_dofs))
        phi = np.arange(len(Ak))
        t1 = time.perf_counter()
        mv = lambda v: O.csr_matvec(pr.rowptr, pr.colidx, pr.vals, v)
        pc = lambda v: O.apply_ragged(v, pr.patch_offsets, pr.patch_dofs, Binv, phi, W, cfg["weighting"])
        x, hist, it, conv = O.fgmres(mv, pc, pr.rhs(0), restart=30, rtol=1e-8, maxit=args.maxit)
    t2 = time.perf_counter()
    return {"value": pr.n * it / (t2 - t0), "unit": "DOF/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"numpy FP64 oracle, whole step (setup with Alg. 1 at tol {tol:g}: {t1 - t0:.2f} s; "
                       f"{it} outer iterations: {t2 - t1:.2f} s) on the same workload family at "
                       f"{kw} (n = {pr.n}, {pr.n_patches} patches); BLAS default threading"),
            "step_s": t2 - t0}


def run_reference(args, cfg, ws, rank):
    if rank != 0:
        return None
    vals, walls = [], []
    for i in range(args.warmup + args.steps):
        cb = cpu_oracle_sample(args, cfg, args.config)
        if i >= args.warmup:
            vals.append(cb["value"])
            walls.append(cb["step_s"])
    v = statistics.median(vals)
    cb["value"] = v
    return {"metric": METRIC, "value": v, "unit": "DOF/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(walls), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": cfg["desc"] + " (bounded CPU sample, see cpu_baseline)",
                       "maxit": args.maxit},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ learned assignment
def run_mlp_gain(args):
    """What the learned assignment gains on the 3D lognormal Q2 workload:
    Alg. 1 on the first half of the patches (in patch order) gives the
    database and the training labels; an MLP (731 -> 256 -> 256 -> m, trained
    on the GPU) predicts the entry of every patch; Alg. 1 then runs on all
    patches from that database without and with the verified predictions."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2306_10025_gb300 as L
    import problems
    dev = torch.device("cuda", 0)
    N = args.mlp_n
    pr = problems.diffusion3d_q2(N=N, seed=0)
    tol = 0.1 if args.tol is None else args.tol
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    rp, ci, va = t(pr.rowptr, torch.int32), t(pr.colidx, torch.int32), t(pr.vals, torch.float64)
    dofs = t(pr.patch_dofs, torch.int32)
    opts = L.make_opts(tol=tol, weighting="sym", krylov="cg")
    p = pr.uniform_size
    A = torch.empty(pr.n_patches, p, p, dtype=torch.float64, device=dev)
    L.psr_extract(rp, ci, va, dofs, uniform_size=p, A_out=A)
    full = L.psr_setup(rp, ci, va, dofs, uniform_size=p, opts=opts)
    phi, reps, m = full.assignment()
    st_full = full.stats()
    half = pr.n_patches // 2
    reps_h = reps[reps < half]
    m0 = int(reps_h.numel())
    seed_A = A[reps_h.long()].contiguous()
    d = p * p + 2
    X = torch.empty(pr.n_patches, d, dtype=torch.float32, device=dev)
    L.psr_features(A, t(pr.cell_coef, torch.float64), X)
    net = L.MLP(d, 256, m0)
    g = np.random.Generator(np.random.PCG64(1))
    params = [g.standard_normal((256, d)) / np.sqrt(d), np.zeros(256), g.standard_normal((256, 256)) / 16.0,
              np.zeros(256), g.standard_normal((m0, 256)) / 16.0, np.zeros(m0)]
    net.set_params(t(np.concatenate([q.reshape(-1) for q in params]).astype(np.float32), torch.float32))
    Xtr = X[:half].contiguous()
    ytr = phi[:half].contiguous()
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ep in range(args.mlp_epochs):
        net.train_step(Xtr, ytr, args.mlp_lr, loss)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    t0 = time.perf_counter()
    hints = net.predict(X)
    torch.cuda.synchronize()
    t_pred = time.perf_counter() - t0
    acc_train = (hints[:half] == ytr).float().mean().item()
    # GEMM work of one training step (forward 3 GEMMs, backward 5), as
    # FP32-equivalent flops; the tensor-core kernels do each product as three
    # TF32 MMAs (hi*hi + hi*lo + lo*hi)
    Bn, h = half, 256
    step_flops = 2.0 * Bn * (2 * d * h + 3 * h * h + 3 * h * m0)
    gemm_tflops = step_flops * args.mlp_epochs / t_train / 1e12
    res = {}
    for name, h in (("without", None), ("with", hints)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c = L.psr_setup_seeded(rp, ci, va, dofs, p, seed_A, h, opts=opts)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        s = c.stats()
        res[name] = {"setup_s": dt, "t_rounds": s["t_rounds"], "criterion_evals": s["criterion_evals"],
                     "hits": s["mlp_hits"], "m_p": s["m_p"]}
        c.destroy()
    out = {"metric": "learned assignment gain (criterion evaluations, setup s)", "workload":
           f"3D Q2 lognormal diffusion {N}^3 (sigma 1, correlation 8 cells), tol {tol}",
           "n_patches": pr.n_patches, "m_p_full_alg1": m, "m_seed_first_half": m0,
           "mlp": {"shape": f"{d}->256->256->{m0}", "epochs": args.mlp_epochs, "lr": args.mlp_lr,
                   "train_s": t_train, "predict_s": t_pred, "final_loss": loss.item(),
                   "train_accuracy": acc_train,
                   "gemm": {"flops_per_step": step_flops, "tflops_whole_step": gemm_tflops,
                            "note": "GEMM flops over the whole training-step time (softmax, masks, Adam included): "
                                    "a lower bound of the GEMM rate; 3xTF32 on tcgen05"}},
           "alg1_full_evals": st_full["criterion_evals"], "seeded": res,
           "evals_saved_fraction": 1.0 - res["with"]["criterion_evals"] / max(res["without"]["criterion_evals"], 1)}
    print(json.dumps(out))


def run_tol_sweep(args, cfg, name):
    """Compressibility of the workload (the tolerance sweep of the 2D Stokes
    configuration, 1e-3 .. 1e-1, FP64 and FP32 inverses): for every setting
    the number of database entries, the retained fraction, the setup time
    and the outer solve (fixed iteration budget) with its residual."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2306_10025_gb300 as L
    dev = torch.device("cuda", 0)
    pr = build_problem(cfg)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    rp, ci, va = t(pr.rowptr, torch.int32), t(pr.colidx, torch.int32), t(pr.vals, torch.float64)
    dofs = t(pr.patch_dofs, torch.int32)
    offs = None if pr.uniform_size else t(pr.patch_offsets, torch.int32)
    b = t(pr.rhs(0), torch.float64)
    rows = []
    for prec in ("fp64", "fp32"):
        for tol in (0.0, 1e-3, 3e-3, 1e-2, 3e-2, 1e-1):
            opts = L.make_opts(tol=tol, store_prec=prec, weighting=cfg["weighting"], krylov=cfg["krylov"],
                               restart=30, rtol=1e-8, maxit=args.maxit)
            for rep in range(2):                      # the second is timed (the first warms up)
                x = torch.zeros_like(b)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ctx = L.psr_setup(rp, ci, va, dofs, offsets=offs, uniform_size=pr.uniform_size, opts=opts)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                info = ctx.solve(b, x)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                st = ctx.stats()
                ctx.destroy()
            rows.append({"store_prec": prec, "tol": tol, "m_p": st["m_p"], "retained_fraction": st["m_p"] / pr.n_patches,
                         "factor_bytes": st["factor_bytes"], "setup_s": t1 - t0, "solve_s": t2 - t1,
                         "iterations": info["iterations"], "relres": info["relres"],
                         "criterion_evals": st["criterion_evals"], "criterion_screened": st["criterion_screened"]})
    print(json.dumps({"metric": "compressibility (database entries, setup s, residual) per criterion tolerance",
                      "workload": cfg["desc"], "n": pr.n, "n_patches": pr.n_patches, "maxit": args.maxit,
                      "rows": rows}))


def run_exp1(args):
    """Experiment 1 of the paper (section 4): 60 x 60 mesh, Q_p for p = 2..5,
    rho = sin^2(pi x) sin^2(pi y) + 0.1, FGMRES(20) with the two-level
    M_combo (Eq. 2, direct coarse solve), x0 = 0, 1e-8.  For every p the full
    storage and Alg. 1 at a few tolerances: database entries, iterations,
    setup (with the coarse operator) and solve times.  The paper's Table 1
    (Matlab GMRES(20)): 11, 12, 14, 15 iterations with full storage for
    p = 2..5; 12, 12, 14, 16 with its best algorithms at 34-35 entries."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2306_10025_gb300 as L
    dev = torch.device("cuda", 0)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    rows = []
    for pdeg in (2, 3, 4, 5):
        pr = build_problem({"builder": "smooth2d_qp", "kw": {"N": 60, "p": pdeg}})
        rp, ci, va = t(pr.rowptr, torch.int32), t(pr.colidx, torch.int32), t(pr.vals, torch.float64)
        dofs = t(pr.patch_dofs, torch.int32)
        prow, pcol, pval, n0 = pr.meta["P0"]
        P0 = (t(prow, torch.int32), t(pcol, torch.int32), t(pval, torch.float64), n0)
        b = t(pr.meta["b"], torch.float64)
        tols = (0.0,) if pr.uniform_size > 32 else (0.0, 0.02, 0.05, 0.1, 0.2)
        for tol in tols:
            opts = L.make_opts(tol=tol, store_prec="fp64", weighting="left", krylov="fgmres", restart=20,
                               rtol=1e-8, maxit=1000)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx = L.psr_setup(rp, ci, va, dofs, uniform_size=pr.uniform_size, opts=opts)
            ctx.set_coarse(*P0)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            x = torch.zeros_like(b)
            info = ctx.solve(b, x)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            st = ctx.stats()
            err = float((x.cpu() - torch.as_tensor(pr.meta["u_nodes"])).abs().max())
            rows.append({"p": pdeg, "tol": tol, "m_p": st["m_p"], "iterations": info["iterations"],
                         "converged": info["converged"], "setup_s": t1 - t0, "solve_s": t2 - t1,
                         "max_error_vs_exact_solution": err})
            ctx.destroy()
    print(json.dumps({"metric": "Experiment 1: FGMRES(20) + M_combo iterations to 1e-8 (60 x 60 mesh, Q_p)",
                      "workload": "smooth2d_qp N=60, p=2..5, rho = sin^2 sin^2 + 0.1, u = sin sin",
                      "paper_table1": {"full": {"2": 11, "3": 12, "4": 14, "5": 15},
                                       "best_compressed_34_35_entries": {"2": 12, "3": 12, "4": 14, "5": 16}},
                      "rows": rows}))


def main():
    args = parse()
    if args.exp1:
        run_exp1(args)
        return
    if args.tol_sweep:
        run_tol_sweep(args, CONFIGS[args.config], args.config)
        return
    if args.mlp:
        run_mlp_gain(args)
        return
    cfg = CONFIGS[args.config]
    ws, rank, local = dist_info()
    if args.impl == "reference":
        out = run_reference(args, cfg, ws, rank)
        if out is not None:
            print(json.dumps(out))
        return
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    out, pr, info, st = run_gpu(args, cfg, ws, rank, local)
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_oracle_sample(args, cfg, args.config)
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
