"""Benchmark of the compressed patch-relaxation hot path on GB300.

One step = the whole path on one synthetic workload, inputs resident in HBM:
setup (patch extraction, multiplicity weights, the database -- Alg. 1, or
every patch its own entry at tol 0 (Eq. 1) -- FP64 inverses, conversion to
the storage layout, autotuned sweep layout) and the outer solve
(right-preconditioned FGMRES(30) or PCG from x0 = 0, sweeps + SpMV +
orthogonalisation) to 1e-8 or a fixed iteration budget.

Default workload: 3D Stokes, Taylor-Hood Q2-Q1 on 48^3 hexahedra with vertex
jitter 0.2h, Dirichlet-trimmed Vanka cell patches of 89 / 62 / 44 / 32 DOFs
(2,689,774 DOFs, 110,592 patches), full storage of FP64 inverses, all size
groups in one streamed sweep launch, FGMRES(30) in FP64.  On this jittered
mesh no two interior patches are within any useful tolerance of each other
(d = 13.7 .. 28.8 between interior patches of the 6^3 instance), so Alg. 1
would keep every patch; the one-level Vanka preconditioner does not reach
1e-8 on it either, so a step runs a fixed FGMRES budget (--maxit).  The
clustered-vs-full comparison to 1e-8 is the `per_config` sub-line on the 3D
lognormal Q2 workload (32^3, PCG), where the one-level method converges.

value = the Schwarz sweep rate of the timed steps: n x (sweeps in the steps)
/ (device time of those sweeps), the sweeps timed by CUDA events the library
records on the solve stream around each launch.  ms_per_step is the whole
step (setup + solve).

Prints ONE JSON line (rank 0).  --impl reference times the CPU FP64 oracle on
a bounded sample of the same instance instead.
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

import numpy as np

METRIC = "Schwarz sweep DOF/s + setup s, clustered vs full, iters to 1e-8 rel. residual"

CONFIGS = {
    "stokes3d": dict(builder="stokes3d_q2q1", kw=dict(N=48), tol=0.0, prec="fp64", weighting="left",
                     krylov="fgmres", maxit=60,
                     desc="3D Stokes Q2-Q1 48^3 hexes, vertex jitter 0.2h, Dirichlet-trimmed Vanka patches "
                          "{89, 62, 44, 32} in one streamed sweep launch, FP64 full storage, FGMRES(30)"),
    "diffusion3d": dict(builder="diffusion3d_q2", kw=dict(N=32), tol=1e-1, prec="fp64", weighting="sym",
                        krylov="cg", maxit=3000, desc="3D Q2 lognormal diffusion 32^3, 27-DOF patches, PCG"),
    "stokes2d": dict(builder="stokes2d_q2q1", kw=dict(N=128, ratio=1.05), tol=1e-2, prec="fp64",
                     weighting="left", krylov="fgmres", maxit=300,
                     desc="2D Stokes Taylor-Hood Q2-Q1, 128x128 quads graded 1.05 in y, 22-DOF Vanka patches"),
    "poisson2d": dict(builder="poisson2d_q2", kw=dict(N=16), tol=1e-12, prec="fp64", weighting="sym",
                      krylov="cg", maxit=1000, desc="2D Q2 diffusion 16x16, 9-DOF patches"),
    "nedelec3d": dict(builder="nedelec3d", kw=dict(N=64), tol=0.0, prec="fp64", weighting="sym",
                      krylov="cg", maxit=300, desc="3D Nedelec curl-curl 64^3, 12-DOF patches"),
}

# FP64 peak of one GB300 from its unit counts and clock: 152 SMs x 2 FP64
# fused multiply-adds per clock x 2 flops x 2.07 GHz; a kernel of independent
# FMA chains (8 warps per SM or more) measured 628 G FMA/s, this figure
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12

# kernel(s) behind each timing class of the library's per-kernel timing
KT_KERNEL_NAMES = {"sweep": "patch sweep (k_sweep_stream for full-storage groups / k_sweep_* tiles)",
                   "spmv": "k_spmv_sell (SELL SpMV, FP64)",
                   "mdot": "k_arnoldi (fused FGMRES Gram-Schmidt step on FP32 pairs) / k_mdot",
                   "maxpy": "k_maxpy (FGMRES w -= V h)", "vec": "vector kernels (k_fg_scale / CG updates)",
                   "inverse": "k_batched_inverse_block / k_batched_inverse (setup: Gauss-Jordan, FP64)"}

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum, one
# ncu capture) over the algorithmic bytes of that launch, for (config,
# class).  Taken on the 24^3 instance of the 3D Stokes workload (one launch
# each, --set full; the 48^3 run holds ~20 GB on the device, above the size
# an ncu replay capture may take) and applied to the algorithmic bytes of the
# run: traffic grows with the bytes (both are the stored inverses / matrix
# entries plus vectors).  Valid only for the kernel sources they were taken on.
TRAFFIC = {
    ("stokes3d", "sweep"): {"ratio": (785.054976e6 + 6.025984e6) / 780664560.0,
                            "capture": "k_sweep_stream, 3D Stokes 24^3: 791.08 MB DRAM for 780.66 MB algorithmic"},
    ("stokes3d", "spmv"): {"ratio": (808.000256e6 + 6.935552e6) / 788402076.0,
                           "capture": "k_spmv_sell (length-sorted slices), 3D Stokes 24^3: 814.94 MB DRAM for "
                                      "788.40 MB algorithmic"},
    ("stokes3d", "inverse"): {"ratio": (679.40224e6 + 619.680768e6) / (10648 * 89 * 89 * 16.0),
                              "capture": "k_batched_inverse_block (the 10,648 patches of 89 DOFs), 3D Stokes 24^3: "
                                         "1299.08 MB DRAM for 1349.48 MB algorithmic"},
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="stokes3d", choices=sorted(CONFIGS))
    ap.add_argument("--maxit", type=int, default=None)
    ap.add_argument("--N", type=int, default=None, help="mesh size of the workload (a smaller instance, e.g. "
                    "for a profiler capture); the default is the configuration's")
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--prec", default=None)
    ap.add_argument("--prec-check", type=float, default=0.5,
                    help="psr_opts.prec_check of the main line (0 keeps every entry in the storage precision)")
    ap.add_argument("--match", default="first", choices=["first", "closest"],
                    help="Alg. 1 assignment rule of the main line (section 3.1: first or closest match)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the precision variants and the sub-line")
    ap.add_argument("--apply-reps", type=int, default=200)
    ap.add_argument("--clock-dir", default=None, help="folder for the nvidia-smi clock samples (default: a temp dir)")
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


def build_problem(cfg, N=None):
    import problems
    kw = dict(cfg["kw"])
    if N is not None:
        kw["N"] = N
    return getattr(problems, cfg["builder"])(**kw)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, folder: str | None = None):
        self.p = None
        self.idx = gpu_index
        folder = folder or tempfile.mkdtemp(prefix="psr_clocks_")
        self.path = os.path.join(folder, f"clocks_rank{gpu_index}.csv")

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
def _setup_solve(L, dev_in, pr, opts, b, x, timing):
    """One step: setup + solve.  Returns (ctx, solve info)."""
    rp, ci, va, dofs, offs = dev_in
    ctx = L.psr_setup(rp, ci, va, dofs, offsets=offs, uniform_size=pr.uniform_size, opts=opts)
    if timing:
        ctx.set_kernel_timing(True)
    info = ctx.solve(b, x)
    return ctx, info


def _apply_median(ctx, n, reps, devc, flush=None, seed=1):
    """Median device time (s) of `reps` applies on random r (CUDA events on
    the current stream), after 10 untimed ones; flush (a tensor larger than
    L2) is zeroed before every timed apply when given."""
    import torch
    stream = torch.cuda.current_stream()
    g = torch.Generator(device=devc).manual_seed(seed)
    rs = [torch.randn(n, dtype=torch.float64, device=devc, generator=g) for _ in range(2)]
    z = torch.empty_like(rs[0])
    for _ in range(10):
        ctx.apply(rs[0], z)
    ev = []
    for i in range(reps):
        if flush is not None:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.apply(rs[i % 2], z)
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    ms = sorted(a.elapsed_time(b_) for a, b_ in ev)
    return ms[len(ms) // 2] * 1e-3


def _sweep_alg_bytes(pr, st):
    """Algorithmic bytes of one apply: r, W and z (24 n), the DOF map (4 per
    patch DOF), phi (4 per patch) and the stored inverses."""
    return 24 * pr.n + 4 * int(pr.patch_offsets[-1]) + 4 * pr.n_patches + st["factor_bytes"]


def _kernels_from_timing(kt, hbm):
    out = {}
    for name, (ms, cnt, by, fl) in kt.items():
        if cnt:
            out[name] = {"launches": cnt, "ms": ms, "us_per_launch": 1e3 * ms / cnt,
                         "alg_bytes_per_launch": by / cnt, "achieved_gbs": by / (ms * 1e-3) / 1e9,
                         "frac": by / (ms * 1e-3) / 1e9 / hbm,
                         "fp64_flops_per_launch": fl / cnt, "achieved_fp64_tflops": fl / (ms * 1e-3) / 1e12,
                         "frac_fp64": fl / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS}
    tot = sum(v["ms"] for v in out.values()) or 1.0
    for v in out.values():
        v["share"] = v["ms"] / tot
    return out


def _roofline_of(name, kd, hbm, peak_source, config):
    if kd["frac_fp64"] > kd["frac"]:
        bound = {"bound": "alu", "achieved": kd["achieved_fp64_tflops"], "peak": FP64_PEAK_TFLOPS,
                 "unit": "TFLOP/s (FP64)", "frac": kd["frac_fp64"],
                 "peak_source": "derived: 152 SMs x 2 FP64 FMA/clock x 2 flops x 2070 MHz (a kernel of "
                                "independent FMA chains measured 628 G FMA/s, the same)"}
    else:
        bound = {"bound": "hbm", "achieved": kd["achieved_gbs"], "peak": hbm, "unit": "GB/s", "frac": kd["frac"],
                 "peak_source": peak_source}
    tr = TRAFFIC.get((config, name))
    return dict(kernel=KT_KERNEL_NAMES[name], **bound,
                traffic=None if tr is None else tr["ratio"] * kd["alg_bytes_per_launch"],
                traffic_source=None if tr is None else tr["capture"] + " (ratio applied to this launch)",
                alg_bytes_per_launch=kd["alg_bytes_per_launch"], launch_us=kd["us_per_launch"],
                share_of_timed_kernels=kd["share"])


def _variant(L, dev_in, pr, cfg, b, devc, reps, tol, prec, arith, maxit, r_ref=None, z_ref=None, solve=True):
    """One setup in another precision / arithmetic: its apply rate, its error
    against the reference apply, and (optionally) its solve with the same
    budget."""
    import torch
    opts = L.make_opts(tol=tol, store_prec=prec, weighting=cfg["weighting"], krylov=cfg["krylov"], restart=30,
                       rtol=1e-8, maxit=maxit, fp64_arith=arith)
    x = torch.zeros_like(b)
    ctx, info = _setup_solve(L, dev_in, pr, opts, b, x, True) if solve else (None, None)
    if ctx is None:
        rp, ci, va, dofs, offs = dev_in
        ctx = L.psr_setup(rp, ci, va, dofs, offsets=offs, uniform_size=pr.uniform_size, opts=opts)
    st = ctx.stats()
    out = {"store_prec": prec, "fp64_arith": arith if prec == "fp64" else None, "m_p": st["m_p"],
           "factor_bytes": st["factor_bytes"]}
    ams = _apply_median(ctx, pr.n, reps, devc)
    out["apply_ms"] = ams * 1e3
    out["sweep_dof_per_s"] = pr.n / ams
    out["sweep_gbs"] = _sweep_alg_bytes(pr, st) / ams / 1e9
    if r_ref is not None:
        z = torch.empty_like(r_ref)
        ctx.apply(r_ref, z)
        out["apply_err_vs_fp64"] = float((z - z_ref).abs().max() / z_ref.abs().max())
    if info is not None:
        out.update(iterations=info["iterations"], relres=info["relres"], converged=info["converged"])
        kt = ctx.kernel_timing()
        out["us_per_launch"] = {k: 1e3 * v[0] / v[1] for k, v in kt.items() if v[1]}
    ctx.destroy()
    return out


def forms_subline(L, key, forms, devc, reps=4, learned=False):
    """Storage forms of one workload (CONFIGS[key]) side by side: per form the
    setup and solve seconds (CUDA events, median after one warm-up, L2
    flushed before each), iterations, relative residual reached, database
    size, apply rate, and the speedup of setup + solve over the first form
    (FP64 full storage).  A form's optional fourth item holds further
    options (the norm-window search)."""
    import torch
    cfg = CONFIGS[key]
    pr = build_problem(cfg)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=devc)
    dev_in = (t(pr.rowptr, torch.int32), t(pr.colidx, torch.int32), t(pr.vals, torch.float64),
              t(pr.patch_dofs, torch.int32), None if pr.uniform_size else t(pr.patch_offsets, torch.int32))
    b = t(pr.rhs(0), torch.float64)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=devc)
    stream = torch.cuda.current_stream()
    rows = {}
    for form in forms:
        name, tol, prec = form[:3]
        extra = form[3] if len(form) > 3 else {}
        opts = L.make_opts(tol=tol, store_prec=prec, weighting=cfg["weighting"], krylov=cfg["krylov"], restart=30,
                           rtol=1e-8, maxit=cfg["maxit"], **extra)
        rp, ci, va, dofs, offs = dev_in
        setups, solves = [], []
        for rep in range(reps):
            flush.zero_()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            x = torch.zeros_like(b)
            e0.record(stream)
            ctx = L.psr_setup(rp, ci, va, dofs, offsets=offs, uniform_size=pr.uniform_size, opts=opts)
            e1.record(stream)
            info = ctx.solve(b, x)
            e2.record(stream)
            e2.synchronize()
            if rep > 0:
                setups.append(e0.elapsed_time(e1) * 1e-3)
                solves.append(e1.elapsed_time(e2) * 1e-3)
            st = ctx.stats()
            if rep < reps - 1:
                ctx.destroy()
        ams = _apply_median(ctx, pr.n, 100, devc, flush=flush)
        ctx.destroy()
        rows[name] = {"tol": tol, "store_prec": prec, **extra, "m_p": st["m_p"], "retained_fraction": st["m_p"] / pr.n_patches,
                      "factor_bytes": st["factor_bytes"], "setup_s": statistics.median(setups),
                      "solve_s": statistics.median(solves), "iterations": info["iterations"],
                      "converged": info["converged"], "relres": info["relres"],
                      "criterion_evals": st["criterion_evals"], "criterion_screened": st["criterion_screened"],
                      "criterion_exact": st["criterion_exact"], "alg1_rounds": st["rounds"],
                      "sweep_dof_per_s": pr.n / ams, "apply_ms": ams * 1e3}
    full = rows[forms[0][0]]
    for name, r in rows.items():
        r["speedup_setup_plus_solve_vs_full_fp64"] = (full["setup_s"] + full["solve_s"]) / (r["setup_s"] + r["solve_s"])
        r["within_plus_one_iteration"] = bool(r["converged"] and r["iterations"] <= full["iterations"] + 1)
    out = {"workload": cfg["desc"] + f", {cfg['krylov']}, {cfg['weighting']} weighting, rtol 1e-8, "
                                     f"at most {cfg['maxit']} iterations",
           "n": pr.n, "n_patches": pr.n_patches, "patch_sizes": sorted(set(pr.patch_sizes.tolist())),
           "rhs": "uniform(-1,1) seed 0", "forms": rows}
    if learned:
        out["learned"] = learned_subline(L, cfg, pr, dev_in, b, devc)
    return out


def config_sublines(L, devc):
    """The other workloads of the benchmark, full storage against the
    clustered forms: 2D Q2 Poisson 16^2 (tol 1e-12), graded 2D Stokes 128^2
    (tol 1e-3 .. 1e-1, FP64 and FP32 entries, the norm-window search), 3D
    Nedelec 64^3 (FP32 / BF16 entries, tol 0.1, the norm-window search), 3D
    lognormal Q2 32^3 (tol 0.1, FP64 / FP32 / BF16, the norm-window search,
    and the learned assignment on a matrix sequence)."""
    return {
        "poisson2d_16": forms_subline(L, "poisson2d", [("full_fp64", 0.0, "fp64"), ("clustered_fp64", 1e-12, "fp64")],
                                      devc),
        "stokes2d_128": forms_subline(L, "stokes2d", [("full_fp64", 0.0, "fp64"),
                                                      ("clustered_fp64_tol_1e-3", 1e-3, "fp64"),
                                                      ("clustered_fp64", 1e-2, "fp64"),
                                                      ("clustered_fp64_norm_window", 1e-2, "fp64",
                                                       {"search": "norm_window"}),
                                                      ("clustered_fp32", 1e-2, "fp32"),
                                                      ("clustered_fp64_tol_1e-1", 1e-1, "fp64")], devc),
        "nedelec3d_64": forms_subline(L, "nedelec3d", [("full_fp64", 0.0, "fp64"), ("full_fp32", 0.0, "fp32"),
                                                       ("full_bf16", 0.0, "bf16"), ("clustered_fp32", 0.1, "fp32"),
                                                       ("clustered_fp32_norm_window", 0.1, "fp32",
                                                        {"search": "norm_window"}),
                                                       ("clustered_bf16", 0.1, "bf16")], devc, reps=2),
        "diffusion3d_32": forms_subline(L, "diffusion3d", [("full_fp64", 0.0, "fp64"),
                                                           ("clustered_fp64", 0.1, "fp64"),
                                                           ("clustered_fp64_norm_window", 0.1, "fp64",
                                                            {"search": "norm_window"}),
                                                           ("clustered_fp32", 0.1, "fp32"),
                                                           ("clustered_bf16", 0.1, "bf16")], devc, learned=True),
    }


def learned_subline(L, cfg, pr, dev_in, b, devc):
    """The learned assignment on a matrix sequence (section 3.2: a database
    carried from one linear problem to the next): a setup of the 3D lognormal
    workload with closest-match labels trains its network on the GPU (half of
    its patches, 300 full-batch Adam steps); the next matrix of the sequence
    (the coefficient field's amplitude 1.0 -> 1.02) is set up (a) by plain
    Alg. 1, (b) seeded with the first setup's database, (c) seeded and hinted
    by the network (psr_setup_learned, use_mlp), in FP32 storage: criterion
    evaluations, setup seconds (prediction included; training reported
    apart) and PCG iterations to 1e-8 against FP64 full storage of the same
    matrix."""
    import torch
    tol = cfg["tol"]
    rp, ci, va, dofs, _ = dev_in
    p = pr.uniform_size
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    train, t_setup1 = timed(lambda: L.psr_setup(rp, ci, va, dofs, uniform_size=p, opts=L.make_opts(
        tol=tol, weighting=cfg["weighting"], krylov=cfg["krylov"], match="closest")))
    info, t_train = timed(lambda: train.mlp_train(hidden=256, epochs=300, lr=1e-3, train_fraction=0.5, seed=1))
    import problems
    pr2 = problems.diffusion3d_q2(N=cfg["kw"]["N"], sigma=1.02, seed=0)
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=devc)
    rp2, ci2, va2 = t(pr2.rowptr, torch.int32), t(pr2.colidx, torch.int32), t(pr2.vals, torch.float64)
    d2 = t(pr2.patch_dofs, torch.int32)
    b2 = t(pr2.rhs(0), torch.float64)
    out = {"matrix_2": "3D Q2 lognormal 32^3, amplitude 1.02 (same noise)", "train": {
        "setup_s": t_setup1, "m_p": train.stats()["m_p"], "train_s": t_train, **info}}
    forms = {
        "full_fp64": lambda: L.psr_setup(rp2, ci2, va2, d2, uniform_size=p, opts=L.make_opts(
            tol=0.0, weighting=cfg["weighting"], krylov=cfg["krylov"], maxit=cfg["maxit"])),
        "alg1_fp32": lambda: L.psr_setup(rp2, ci2, va2, d2, uniform_size=p, opts=L.make_opts(
            tol=tol, store_prec="fp32", weighting=cfg["weighting"], krylov=cfg["krylov"], maxit=cfg["maxit"])),
        "seeded_fp32": lambda: L.psr_setup_learned(rp2, ci2, va2, d2, p, train, opts=L.make_opts(
            tol=tol, store_prec="fp32", weighting=cfg["weighting"], krylov=cfg["krylov"], maxit=cfg["maxit"],
            use_mlp=False)),
        "learned_fp32": lambda: L.psr_setup_learned(rp2, ci2, va2, d2, p, train, opts=L.make_opts(
            tol=tol, store_prec="fp32", weighting=cfg["weighting"], krylov=cfg["krylov"], maxit=cfg["maxit"],
            use_mlp=True)),
    }
    for name, mk in forms.items():
        best = None
        for rep in range(2):
            ctx, ts = timed(mk)
            x = torch.zeros_like(b2)
            inf, tsol = timed(lambda: ctx.solve(b2, x))
            st = ctx.stats()
            ctx.destroy()
            if best is None or ts < best[0]:
                best = (ts, tsol, inf, st)
        ts, tsol, inf, st = best
        out[name] = {"setup_s": ts, "solve_s": tsol, "m_p": st["m_p"], "criterion_evals": st["criterion_evals"],
                     "mlp_hits": st["mlp_hits"], "iterations": inf["iterations"], "converged": inf["converged"]}
    full = out["full_fp64"]["iterations"]
    for name in ("alg1_fp32", "seeded_fp32", "learned_fp32"):
        out[name]["within_plus_one_iteration"] = bool(out[name]["converged"] and out[name]["iterations"] <= full + 1)
    out["evals_saved_vs_seeded"] = 1.0 - out["learned_fp32"]["criterion_evals"] / max(out["seeded_fp32"]["criterion_evals"], 1)
    out["evals_saved_vs_alg1"] = 1.0 - out["learned_fp32"]["criterion_evals"] / max(out["alg1_fp32"]["criterion_evals"], 1)
    train.destroy()
    return out


def run_gpu(args, cfg, ws, rank, local):
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2306_10025_gb300 as L

    torch.cuda.set_device(local)
    devc = torch.device("cuda", local)
    t_gen = time.perf_counter()
    pr = build_problem(cfg, args.N)
    t_gen = time.perf_counter() - t_gen
    tol = cfg["tol"] if args.tol is None else args.tol
    prec = cfg["prec"] if args.prec is None else args.prec
    maxit = cfg["maxit"] if args.maxit is None else args.maxit
    t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=devc)
    dev_in = (t(pr.rowptr, torch.int32), t(pr.colidx, torch.int32), t(pr.vals, torch.float64),
              t(pr.patch_dofs, torch.int32), None if pr.uniform_size else t(pr.patch_offsets, torch.int32))
    b = t(pr.rhs(0), torch.float64)
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()
    opts = L.make_opts(tol=tol, store_prec=prec, weighting=cfg["weighting"], krylov=cfg["krylov"], restart=30,
                       rtol=1e-8, maxit=maxit, fp64_arith="pairs", prec_check=args.prec_check, match=args.match)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    peak_source = "measured" if "hbm_gbs" in peaks else "fallback"
    # the stored inverses alone exceed L2 (129 MB) on the large workloads;
    # smaller ones get an L2 flush (256 MB write) before every timed step
    nnz_bytes = 12 * pr.nnz
    big = nnz_bytes > 4 * 129e6
    flush = None if big else torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=devc)

    for _ in range(args.warmup):
        ctx, info = _setup_solve(L, dev_in, pr, opts, b, x, True)
        ctx.destroy()
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    clk = ClockSampler(local, args.clock_dir)
    clk.start()
    launches0 = L.psr_kernel_launches()
    times, infos, stats, kts = [], [], [], []
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    for k in range(args.steps):
        if flush is not None:
            flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx, info = _setup_solve(L, dev_in, pr, opts, b, x, True)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) * 1e-3)
        infos.append(info)
        stats.append(ctx.stats())
        kts.append(ctx.kernel_timing())
        if k < args.steps - 1:
            ctx.destroy()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    launches = L.psr_kernel_launches() - launches0
    clocks = clk.stop()
    last = ctx
    step_s = sum(times) / len(times)
    sweep_ms = sum(kt["sweep"][0] for kt in kts)
    sweeps = sum(kt["sweep"][1] for kt in kts)
    units_local = pr.n * sweeps
    value, total_sweep_s, _ = aggregate_replicas(sweep_ms * 1e-3, units_local, devc)
    st = stats[-1]
    # per-kernel picture of the timed steps (summed over them)
    kt_sum = {}
    for kt in kts:
        for name, (ms, cnt, by, fl) in kt.items():
            a = kt_sum.setdefault(name, [0.0, 0, 0.0, 0.0])
            a[0] += ms
            a[1] += cnt
            a[2] += by
            a[3] += fl
    # the setup's batched inverses: GPU time from the CUDA events the library
    # records around their launches (stats t_invert); 2 p^3 flops and 16 p^2
    # bytes (the patch in, the inverse out) per patch, one launch per size group
    inv_ms = 1e3 * sum(s_["t_invert"] for s_ in stats)
    if inv_ms > 0:
        ps = pr.patch_sizes.astype(np.float64)
        kt_sum["inverse"] = [inv_ms, st["n_groups"] * len(stats), 16.0 * float((ps ** 2).sum()) * len(stats),
                             2.0 * float((ps ** 3).sum()) * len(stats)]
    kernels = _kernels_from_timing({k: tuple(v) for k, v in kt_sum.items()}, hbm)
    top = max(kernels, key=lambda k: kernels[k]["ms"])
    roofline = _roofline_of(top, kernels[top], hbm, peak_source, args.config)
    roofline["timing"] = ("CUDA events the library records around the batched-inverse launches of each setup, "
                          "timed steps" if top == "inverse" else
                          "CUDA events the library records on the solve stream around each launch, timed steps")
    roofline["kernels"] = kernels
    solve_names = [k for k in kernels if k != "inverse"]
    solve_top = max(solve_names, key=lambda k: kernels[k]["ms"])
    solve_roof = _roofline_of(solve_top, kernels[solve_top], hbm, peak_source, args.config)
    solve_roof["timing"] = "CUDA events the library records on the solve stream around each launch, timed steps"
    sweep_roof = _roofline_of("sweep", kernels["sweep"], hbm, peak_source, args.config)
    # the sweep alone: median of back-to-back applies (larger-than-L2 inputs)
    r_ref = torch.randn(pr.n, dtype=torch.float64, device=devc, generator=torch.Generator(device=devc).manual_seed(7))
    z_ref = torch.empty_like(r_ref)
    last.apply(r_ref, z_ref)
    ams = _apply_median(last, pr.n, args.apply_reps, devc, flush=flush)
    sweep_roof["alone"] = {"apply_ms": ams * 1e3, "alg_bytes": _sweep_alg_bytes(pr, st),
                           "achieved_gbs": _sweep_alg_bytes(pr, st) / ams / 1e9,
                           "frac": _sweep_alg_bytes(pr, st) / ams / 1e9 / hbm, "reps": args.apply_reps}
    last.destroy()

    out = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * step_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg["desc"] + ("" if args.N is None else f" (mesh size overridden: N = {args.N})"),
                   "n": pr.n, "nnz": pr.nnz, "n_patches": pr.n_patches,
                   "patch_sizes": sorted(set(pr.patch_sizes.tolist())), "tol": tol, "store_prec": prec,
                   "fp64_arith": "pairs (FP64 inverses as (hi, lo) FP32 pairs, compensated products, ~47 bits)",
                   "krylov": cfg["krylov"] + ("(30)" if cfg["krylov"] == "fgmres" else ""),
                   "weighting": cfg["weighting"], "maxit": maxit, "match": args.match, "rhs": "uniform(-1,1) seed 0",
                   "l2": ("inputs larger than L2 (the stored inverses alone)" if big
                          else "flushed (256 MB write) before every timed step"),
                   "allocations": "library caching allocator, filled by the warm-up steps",
                   "value_def": "n x sweeps in the timed steps / device time of those sweeps (CUDA events)",
                   "generation_s": t_gen, "parallelism": f"replicas x{ws}"},
        "setup_s": {"total": st["t_extract"] + st["t_rounds"] + st["t_convert"] + st["t_autotune"],
                    "phases": {k: st[k] for k in ("t_extract", "t_rounds", "t_convert", "t_autotune")}},
        "iters": {"iterations": infos[-1]["iterations"], "relres": infos[-1]["relres"],
                  "converged": infos[-1]["converged"], "rtol": 1e-8},
        "m_p": st["m_p"], "retained_fraction": st["m_p"] / pr.n_patches, "factor_bytes": st["factor_bytes"],
        "criterion_evals": st["criterion_evals"],
        "step_dof_per_s": pr.n * sweeps / sum(times),
        "roofline": roofline, "solve_roofline": solve_roof, "sweep_roofline": sweep_roof, "clocks": clocks,
        "gpu_launches": launches,
    }
    if not args.no_extras:
        # the same setup with other storage / arithmetic: rate, error against
        # the FP64 (pairs) apply and the solve with the same budget
        variants = {}
        for name, pv, ar in (("fp64_native", "fp64", "native"), ("fp32", "fp32", "pairs"), ("bf16", "bf16", "pairs")):
            variants[name] = _variant(L, dev_in, pr, cfg, b, devc, 50, tol, pv, ar, maxit, r_ref, z_ref)
        out["precisions"] = variants
        out["per_config"] = config_sublines(L, devc)

    # end to end: host (pinned) inputs -> device -> setup + solve -> x to host
    if not args.no_e2e:
        hp = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt).pin_memory()
        h_in = [hp(pr.rowptr, torch.int32), hp(pr.colidx, torch.int32), hp(pr.vals, torch.float64),
                hp(pr.patch_dofs, torch.int32), hp(pr.rhs(0), torch.float64)]
        h_o = None if pr.uniform_size else hp(pr.patch_offsets, torch.int32)
        h_x = torch.empty(pr.n, dtype=torch.float64).pin_memory()
        h2d = sum(a.numel() * a.element_size() for a in h_in) + (0 if h_o is None else h_o.numel() * 4)
        del dev_in
        torch.cuda.empty_cache()
        ets, its = [], []
        for i in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d = [a.to(devc, non_blocking=True) for a in h_in]
            d_o = None if h_o is None else h_o.to(devc, non_blocking=True)
            d_x = torch.zeros(pr.n, dtype=torch.float64, device=devc)
            c2 = L.psr_setup(d[0], d[1], d[2], d[3], offsets=d_o, uniform_size=pr.uniform_size, opts=opts)
            inf2 = c2.solve(d[4], d_x)
            h_x.copy_(d_x, non_blocking=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            c2.destroy()
            del d, d_o, d_x
            if i >= args.warmup:
                ets.append(dt)
                its.append(inf2["iterations"])
        out["e2e"] = {"value": pr.n * sum(its) / sum(ets), "unit": "DOF/s", "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(pr.n * 8), "ms_per_step": 1e3 * sum(ets) / len(ets),
                      "def": "n x sweeps per host wall second of the whole call (copies, setup, solve, read-back)"}
    return out, pr


# ------------------------------------------------------------------ CPU oracle
_SHM = {}


def _shm_attach(spec):
    """Worker initialiser: attach the shared arrays of the oracle sample."""
    from multiprocessing import shared_memory
    for key, (name, shape, dt) in spec.items():
        h = shared_memory.SharedMemory(name=name)
        _SHM[key] = (h, np.ndarray(shape, dtype=dt, buffer=h.buf))


def _oracle_apply_chunk(rng):
    """The oracle's apply (Eq. 3, ragged sizes) over sampled patches
    k0..k1-1, on the DOFs they touch (renumbered locally); returns the
    seconds of the apply_ragged call."""
    from oracle import psr_oracle as O
    k0, k1 = rng
    arr = lambda k: _SHM[k][1]
    offs, flat, boff, bflat, r, W = (arr(k) for k in ("offs", "flat", "boff", "bflat", "r", "W"))
    fl = flat[offs[k0]:offs[k1]]
    uniq, loc = np.unique(fl, return_inverse=True)
    o = offs[k0:k1 + 1] - offs[k0]
    sizes = np.diff(o)
    Binv = [bflat[boff[k]:boff[k + 1]].reshape(int(s), int(s)) for k, s in zip(range(k0, k1), sizes)]
    t0 = time.perf_counter()
    O.apply_ragged(r[uniq], o, loc, Binv, np.arange(k1 - k0), W[uniq], "left")
    return time.perf_counter() - t0


def cpu_oracle_sample(pr, cfg, n_apply=6000, n_inv=400, cores=None):
    """The numpy FP64 oracle, as it stands, on a bounded sample of the same
    instance: O.lu_inverse on `n_inv` of its patches (setup part) and
    O.apply_ragged on `n_apply` sampled patches (sweep part), single-threaded
    and cut into one chunk per host core (spawned workers, data in shared
    memory); scaled to the full instance by sum(p^2) (apply) and sum(p^3)
    (inverses), the work of each being proportional to it.
    value = n / (scaled all-core oracle time of one apply)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    from oracle import psr_oracle as O
    cores = cores or os.cpu_count() or 1
    offs_all = pr.patch_offsets.astype(np.int64)
    sizes = np.diff(offs_all)
    g = np.random.Generator(np.random.PCG64(11))
    pick = np.sort(g.choice(pr.n_patches, size=min(n_apply, pr.n_patches), replace=False))
    flat_s = np.concatenate([pr.patch_dofs[offs_all[k]:offs_all[k + 1]] for k in pick]).astype(np.int64)
    offs_s = np.concatenate([[0], np.cumsum(sizes[pick])]).astype(np.int64)
    # the sampled patch matrices (not timed): one O.csr_lookup over a copy of
    # the CSR that keeps only the rows the sample uses
    rows = np.unique(flat_s)
    rp64 = pr.rowptr.astype(np.int64)
    keep = np.zeros(pr.n, dtype=bool)
    keep[rows] = True
    lens = np.where(keep, np.diff(rp64), 0)
    sub_ptr = np.concatenate([[0], np.cumsum(lens)])
    take = np.concatenate([np.arange(rp64[i], rp64[i + 1]) for i in rows])
    rr = np.concatenate([np.repeat(flat_s[offs_s[k]:offs_s[k + 1]], sizes[pick[k]]) for k in range(len(pick))])
    cc = np.concatenate([np.tile(flat_s[offs_s[k]:offs_s[k + 1]], sizes[pick[k]]) for k in range(len(pick))])
    vals = O.csr_lookup(sub_ptr, pr.colidx[take], pr.vals[take], pr.n, rr, cc)
    sq = np.concatenate([[0], np.cumsum(sizes[pick] ** 2)])
    A_s = [vals[sq[k]:sq[k + 1]].reshape(sizes[pick[k]], sizes[pick[k]]) for k in range(len(pick))]
    del rr, cc, vals
    # setup part: inverses of the first n_inv sampled patches, per size
    sub = A_s[:n_inv]
    t0 = time.perf_counter()
    by_size = {}
    for p in sorted(set(a.shape[0] for a in sub)):
        by_size[p] = O.lu_inverse(np.stack([a for a in sub if a.shape[0] == p]))[0]
    t_inv = time.perf_counter() - t0
    # every sampled patch needs an inverse for the apply: the computed ones
    # are reused cyclically within each size (the apply's work is the same)
    cnt = {}
    blocks = []
    for a in A_s:
        p = a.shape[0]
        if p not in by_size:
            by_size[p] = O.lu_inverse(a[None])[0]
        j = cnt.get(p, 0)
        blocks.append(by_size[p][j % by_size[p].shape[0]].reshape(-1))
        cnt[p] = j + 1
    bflat = np.concatenate(blocks)
    boff = np.concatenate([[0], np.cumsum([blk.size for blk in blocks])]).astype(np.int64)
    W = O.weights(O.multiplicity(pr.n, pr.patch_dofs))
    r = np.random.Generator(np.random.PCG64(5)).uniform(-1, 1, pr.n)
    shms, spec = [], {}
    try:
        for key, a in (("offs", offs_s), ("flat", flat_s), ("boff", boff), ("bflat", bflat), ("r", r), ("W", W)):
            h = shared_memory.SharedMemory(create=True, size=max(a.nbytes, 1))
            np.ndarray(a.shape, dtype=a.dtype, buffer=h.buf)[...] = a
            shms.append(h)
            spec[key] = (h.name, a.shape, a.dtype)
        _shm_attach(spec)
        ns = len(pick)
        t_one = _oracle_apply_chunk((0, ns))
        cuts = np.linspace(0, ns, cores + 1).astype(int)
        ranges = [(int(cuts[i]), int(cuts[i + 1])) for i in range(cores) if cuts[i + 1] > cuts[i]]
        ctx = mp.get_context("spawn")
        with ctx.Pool(len(ranges), initializer=_shm_attach, initargs=(spec,)) as pool:
            pool.map(_oracle_apply_chunk, ranges)          # warm: imports, first touch
            t0 = time.perf_counter()
            pool.map(_oracle_apply_chunk, ranges)
            t_all = time.perf_counter() - t0
    finally:
        for key in list(_SHM):
            _SHM.pop(key)[0].close()
        for h in shms:
            h.close()
            h.unlink()
    s2_full = float(np.sum(sizes.astype(np.float64) ** 2))
    s2_app = float(np.sum(sizes[pick].astype(np.float64) ** 2))
    s3_full = float(np.sum(sizes.astype(np.float64) ** 3))
    s3_inv = float(sum(a.shape[0] ** 3 for a in sub))
    apply_one = t_one * s2_full / s2_app
    apply_all = t_all * s2_full / s2_app
    return {"value": pr.n / apply_all, "unit": "DOF/s", "cores": len(ranges), "kind": "oracle",
            "nproc": os.cpu_count(),
            "single_thread": {"value": pr.n / apply_one, "apply_s_full": apply_one},
            "apply_s_full": apply_all,
            "setup_inverses_s_full_single_thread": t_inv * s3_full / s3_inv,
            "sample": (f"numpy FP64 oracle on the same instance ({pr.n} DOFs): apply_ragged over {ns} sampled "
                       f"patches ({t_one:.3f} s single-threaded, {t_all:.3f} s in {len(ranges)} spawned workers, "
                       f"one chunk each) and lu_inverse of {len(sub)} of them ({t_inv:.2f} s); scaled to all "
                       f"{pr.n_patches} patches by sum(p^2) (apply) and sum(p^3) (inverses)")}


def run_reference(args, cfg, ws, rank):
    if rank != 0:
        return None
    pr = build_problem(cfg, args.N)
    vals, walls, cb = [], [], None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        cb = cpu_oracle_sample(pr, cfg, n_apply=3000, n_inv=200)
        if i >= args.warmup:
            vals.append(cb["value"])
            walls.append(time.perf_counter() - t0)
    v = statistics.median(vals)
    cb["value"] = v
    return {"metric": METRIC, "value": v, "unit": "DOF/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(walls), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": cfg["desc"] + " (bounded CPU sample of the same instance, see cpu_baseline)",
                       "n": pr.n, "n_patches": pr.n_patches},
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
        tols = (0.0, 0.02, 0.05, 0.1, 0.2)
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
    out, pr = run_gpu(args, cfg, ws, rank, local)
    if rank == 0:
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_oracle_sample(pr, cfg)
        print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
