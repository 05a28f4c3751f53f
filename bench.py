"""Benchmark of the AFC hot path on GB300.

Workload (one "step"): one Crank-Nicolson time step of nonlinear Zalesak FCT on
trilinear Q1 hexahedra, 65^3-node uniform grid of the unit cube (274,625 dofs),
rotating velocity b = (0.5 - y, x - 0.5, 0), eps = 1e-6, c = 0, cosine hump of
radius 0.15 at (0.5, 0.75, 0.5), homogeneous Dirichlet data on the boundary,
dt from CFL 1; the fixed point runs to ||res|| < sqrt(N) 1e-10 with a
Jacobi-BiCGStab inner solve to atol 1e-12, all in FP64.  Metric: dof-iters/s =
dofs x fixed-point corrections / time.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
With N > 1 (torchrun) every rank runs its own instance (weak scaling).
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

# the CPU oracle is timed single-threaded (set before numpy loads its BLAS)
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 65
ELEM = "q1"
CFL = 1.0
FP_TOL = 1e-10
KSP_ATOL = 1e-12
METRIC = "dof-iters/s for AFC fixed-point"
WORKLOAD = "CN nonlinear Zalesak FCT, Q1 65^3 (274625 dofs), rotating b, eps=1e-6, CFL 1, fp tol 1e-10, " \
           "Jacobi-BiCGStab atol 1e-12"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 FMA pipe of GB300: 152 SMs x 2 DFMA/clk x 2 flop x 2.070 GHz (recipe unit counts and max clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def whole_job(units, ms, ws, device="cpu"):
    """Whole-job throughput of N replicas: the units all ranks processed divided by the
    slowest rank's time (MAX over ranks), in units per second; (value, max_ms).  With one
    rank no process group is needed."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(units), float(ms)], dtype=torch.float64, device=device)
        u = t[:1].clone()
        m = t[1:].clone()
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        dist.all_reduce(m, op=dist.ReduceOp.MAX)
        units, ms = float(u.item()), float(m.item())
    return units / (ms / 1e3), ms


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _make_problem(afc, W, precision):
    wl = W.rotating_transient(ELEM, N_SIDE)
    P = afc.Problem.structured(wl.elem, wl.n)
    P.set_coefficients(wl.eps, wl.b, wl.c, wl.f)
    P.set_dirichlet(wl.dir_mask, wl.u_dir)
    P.assemble(afc.AFC_FAMILY_FCT, precision)
    P.set_solution(wl.u0)
    return P, wl


def _opts(afc, dt, mixed=False):
    if mixed:
        return afc.default_opts(scheme=afc.AFC_CN_NONLINEAR, dt=dt, fp_tol=FP_TOL, fp_maxit=100, ksp_atol=0.0,
                                ksp_rtol=1e-6, precision=afc.AFC_MIXED)
    return afc.default_opts(scheme=afc.AFC_CN_NONLINEAR, dt=dt, fp_tol=FP_TOL, fp_maxit=100, ksp_atol=KSP_ATOL)


# Algorithmic FP64 work per launch of the kernels that can dominate a CN step (the design
# notes state the counts): SpMV 2 flops per pattern entry, a fused dot 2 per row; the CN
# flux of Eq. flux_002 with node sums precomputed 5 per pair + 1 for the prelimiter
# argument; P+/- 1 per directed pair; alpha r_ij accumulated 2 per directed pair.
def _kernel_work(name, N, nnz, E, its_per_launch=0.0):
    if name == "k_bicg_fused":
        # one persistent launch per BiCGStab solve: per iteration 2 SpMV (4 nnz) and the
        # vector updates and dots (26 N)
        return ("alu", its_per_launch * (4.0 * nnz + 26.0 * N), "TFLOP/s")
    if name == "k_bicg_spmv1":
        return ("alu", 2.0 * nnz + 2.0 * N, "TFLOP/s")
    if name == "k_bicg_spmv2":
        return ("alu", 2.0 * nnz + 4.0 * N, "TFLOP/s")
    if name == "k_cn_residual":
        return ("alu", 2.0 * (2 * E) + 2.0 * nnz, "TFLOP/s")
    if name == "k_cn_factors":
        return ("alu", 1.0 * (2 * E), "TFLOP/s")
    if name == "k_cn_edges":
        return ("alu", 6.0 * E, "TFLOP/s")
    return (None, None, None)


def _timed_steps(P, opts, steps, flush, stream, torch):
    """Time `steps` steps one by one with CUDA events on the problem's stream, L2 flushed
    (not timed) before each.  Returns (ms, fixed-point its, Krylov its, statuses)."""
    ms_total, its_total, inner_total, statuses = 0.0, 0, 0, []
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = P.step(opts)
        e1.record(stream)
        e1.synchronize()
        ms_total += e0.elapsed_time(e1)
        its_total += st["outer_its"]
        inner_total += st["inner_its"]
        statuses.append(st["status"])
    return ms_total, its_total, inner_total, statuses


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture
# (profiles/k_bicg_fused_q1_65.md), valid while the kernel's sources hash as they did then.
_NCU_TRAFFIC = {
    "k_bicg_fused": {"bytes": 76.80e6, "sha1": "11b039bea6594c49",
                     "sources": ("krylov.cu", "kernels_common.cuh", "afc_internal.h", "grid_sync.cuh")},
}


def _traffic(name):
    import hashlib
    t = _NCU_TRAFFIC.get(name)
    if t is None:
        return None
    h = hashlib.sha1()
    for f in t["sources"]:
        with open(os.path.join(ROOT, "paper_2110_15676_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return t["bytes"] if h.hexdigest()[:16] == t["sha1"] else None


def _roofline(name, kms, kcount, work_flops, share):
    achieved = work_flops / (kms / kcount / 1e3) / 1e12
    return {"bound": "alu", "kernel": name, "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": _traffic(name),
            "traffic_unit": "bytes per launch (ncu, cold cache)",
            "peak_source": "FP64 pipe: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz (recipe unit counts, max clock)",
            "avg_launch_us": kms / kcount * 1e3, "share": share}


# Inner tolerance of the stationary MC solves (config 3 and the serving requests): the
# relative GMRES reduction per fixed-point correction.  Measured on the config-3 solve
# (bench.py --only-mc-sweep --mc-inner-rtols): every inner tolerance from 1e-6 to 1e-1
# takes the same ~360 corrections and ends 1.27e-3 to 1.28e-3 from a reference
# converged to 1e-13, so the outer stop decides the accuracy; 1e-2 needs 19 GMRES
# iterations per correction instead of 182 at 1e-6.
MC_INNER_RTOL = 1e-2


def _mc_solve(afc, P, wl, torch, stream, rtol=MC_INNER_RTOL, ref=None, sweep_ms=None):
    # the whole stationary MC solve of this workload (damped fixed point, omega = 0.5,
    # tol 1e-10, mixed-precision Jacobi-GMRES(20) inner solves to a relative rtol);
    # with ref, also the largest difference from that solution relative to its maximum
    sopts = afc.default_opts(limiter=afc.AFC_LIM_MC, omega=0.5, ksp=afc.AFC_KSP_GMRES, ksp_atol=0.0, ksp_rtol=rtol,
                             fp_tol=1e-10, fp_maxit=1000, precision=afc.AFC_MIXED)
    P.set_solution(wl.u0)
    P.solve_stationary(afc.default_opts(limiter=afc.AFC_LIM_MC, omega=0.5, ksp=afc.AFC_KSP_GMRES, ksp_atol=0.0,
                                        ksp_rtol=rtol, fp_fixed_its=1, precision=afc.AFC_MIXED))   # build / warm
    P.set_solution(wl.u0)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sst = P.solve_stationary(sopts)
    e1.record(stream)
    e1.synchronize()
    solve_ms = e0.elapsed_time(e1)
    u_sol = P.get_solution()
    N = P.info()["n_nodes"]
    out = {"ms": solve_ms, "fixed_point_its": sst["outer_its"], "gmres_its": sst["inner_its"],
           "status": sst["status"], "res_final": sst["res_final"],
           "dof_iters_per_s": N * sst["outer_its"] / (solve_ms / 1e3),
           "umin": float(u_sol.min()), "umax": float(u_sol.max()), "dmp_violation": sst["dmp_violation"],
           "options": f"omega 0.5, tol 1e-10, mixed: FP32 Jacobi-GMRES(20) rtol {rtol:g}, float-pair MC residual, "
                      f"FP64 outer"}
    if ref is not None:
        out["rel_diff_vs_main_solve"] = float(np.abs(u_sol - ref).max() / np.abs(ref).max())
    if sweep_ms is not None and sst["inner_its"] > 0:
        # the inner solves' share: the solve's time without its residual sweeps (one per
        # fixed-point iteration and a final one), per GMRES iteration, against the
        # algorithmic bytes of one Arnoldi step with single-precision vectors: the product
        # (CSR count, 8 nnz + 12 N) and classical Gram-Schmidt without the
        # re-orthogonalisation pass over the average k + 1 = 10.5 basis vectors of
        # GMRES(20) (4 N (2 k + 5)) plus the normalisation (16 N): 8 nnz + 132 N
        info = P.info()
        nnz = info["nnz"]
        g_ms = solve_ms - (sst["outer_its"] + 1) * sweep_ms
        per = g_ms / sst["inner_its"]
        b = 8.0 * nnz + 132.0 * N
        peaks, src = _peaks()
        out["gmres"] = {"ms_per_iteration": per, "algorithmic_bytes_per_iteration": b,
                        "achieved_gbs": b / (per / 1e3) / 1e9, "peak_gbs": peaks["hbm_gbs"],
                        "frac": b / (per / 1e3) / 1e9 / peaks["hbm_gbs"], "peak_source": src}
    return out, u_sol


def mc_sweep(afc, W, torch, flush, stream, reps, solve=True, inner_rtols=()):
    """The stationary MC limiter + residual sweep on Kuhn P1 129^3 (2,146,689 dofs):
    bounds, limited fluxes of all 14.8 M pairs, residual SpMV and norm, timed on the
    iterate after 6 damped fixed-point corrections from u0."""
    wl = W.stationary_inflow("p1", 129)
    P = afc.Problem.structured(wl.elem, wl.n)
    P.set_coefficients(wl.eps, wl.b, wl.c, wl.f)
    P.set_dirichlet(wl.dir_mask, wl.u_dir)
    P.assemble(afc.AFC_FAMILY_MC, afc.AFC_MIXED)
    # a realistic state of the fixed point: the iterate after a few damped corrections
    # from u0 (mixed-precision inner GMRES), not a random field
    P.set_solution(wl.u0)
    # (host-driven loop: the same arithmetic as the graph, and its kernels stay visible to profilers)
    P.solve_stationary(afc.default_opts(limiter=afc.AFC_LIM_MC, omega=0.5, ksp=afc.AFC_KSP_GMRES, ksp_atol=0.0,
                                        ksp_rtol=MC_INNER_RTOL, fp_fixed_its=6, precision=afc.AFC_MIXED, graph=0))
    info = P.info()
    N, nnz, E = info["n_nodes"], info["nnz"], info["n_edges"]
    for _ in range(3):
        P.mc_residual_sweep(afc.AFC_LIM_MC)
    torch.cuda.synchronize()
    ms = 0.0
    for _ in range(reps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P.mc_residual_sweep(afc.AFC_LIM_MC)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    P.profile(True)
    for _ in range(reps):
        flush.fill_(1.0)
        P.mc_residual_sweep(afc.AFC_LIM_MC)
    prof, _ = P.profile_read()
    P.profile(False)
    sweep_ms = ms / reps
    solve_out = None
    inner = None
    if solve:
        solve_out, u_ref = _mc_solve(afc, P, wl, torch, stream, sweep_ms=ms / reps)
        if inner_rtols:
            # a reference converged far below the stopping tolerance (FP64 throughout, inner
            # GMRES to 1e-10 relative, fixed point to 1e-13): how far each solve to 1e-10 lies
            # from the fixed point itself, for every inner tolerance
            P.set_solution(wl.u0)
            rst = P.solve_stationary(afc.default_opts(limiter=afc.AFC_LIM_MC, omega=0.5, ksp=afc.AFC_KSP_GMRES,
                                                      ksp_atol=0.0, ksp_rtol=1e-10, ksp_maxit=5000, fp_tol=1e-13,
                                                      fp_maxit=3000, precision=afc.AFC_FP64))
            u_star = P.get_solution()
            scale = np.abs(u_star).max()
            inner = {"reference": {"fixed_point_its": rst["outer_its"], "gmres_its": rst["inner_its"],
                                   "status": rst["status"], "res_final": rst["res_final"],
                                   "options": "FP64, inner GMRES(20) rtol 1e-10, fixed point tol 1e-13"},
                     f"{MC_INNER_RTOL:g}": {"rel_err_vs_reference": float(np.abs(u_ref - u_star).max() / scale)}}
            for r in inner_rtols:
                o_r, u_r = _mc_solve(afc, P, wl, torch, stream, rtol=r, ref=u_ref, sweep_ms=ms / reps)
                o_r["rel_err_vs_reference"] = float(np.abs(u_r - u_star).max() / scale)
                inner[f"{r:g}"] = o_r
    # algorithmic work of one sweep (design notes): FP64 flops 14 per pair + 2 per entry;
    # bytes of the CSR count 4(N+1) + 12 nnz + 24 E + 24 N
    flops = 14.0 * E + 2.0 * nnz
    alg_bytes = 4.0 * (N + 1) + 12.0 * nnz + 24.0 * E + 24.0 * N
    peaks, src = _peaks()
    out = {"workload": "stationary MC, Kuhn P1 129^3 (2146689 dofs, 14827904 pairs), eps=1e-8, c=1, b=(1,-0.5,0.25)",
           "ms_per_sweep": sweep_ms, "dof_sweeps_per_s": N / (sweep_ms / 1e3),
           "hbm": {"bound": "hbm", "achieved": alg_bytes / (sweep_ms / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                   "unit": "GB/s", "frac": alg_bytes / (sweep_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                   "algorithmic_bytes": alg_bytes, "peak_source": src},
           "alu": {"bound": "alu", "achieved": flops / (sweep_ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                   "unit": "TFLOP/s", "frac": flops / (sweep_ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS,
                   "algorithmic_flops": flops},
           "kernels": {k: {"ms": v[0] / reps, "launches": v[1] // reps} for k, v in prof.items()},
           "solve": solve_out, "inner_rtol_sweep": inner}
    del P
    return out


def batched(afc, W, torch, stream, steps=50, count=256, seed=4, shape=None, solo=True):
    """256 independent transient Q1 problems (nodes per side uniform in [17, 49], eps
    log-uniform in [1e-8, 1e-4], random constant unit b, random hump centre), 50
    SSP3 Zalesak steps each at CFL 0.5: batched mixed precision, batched FP64 and the
    plain one-at-a-time FP64 path (afc_step per instance and step)."""
    rng = np.random.default_rng(seed)
    wls = [W.random_transient(rng, "q1", (17, 49)) for _ in range(count)]
    gs = []
    N = nnz = E = 0
    for wl in wls:
        g = afc.Problem.structured(wl.elem, wl.n)
        g.set_coefficients(wl.eps, wl.b, wl.c, wl.f)
        g.set_dirichlet(wl.dir_mask, wl.u_dir)
        g.assemble(afc.AFC_FAMILY_FCT, afc.AFC_FP64)
        g.set_solution(wl.u0)
        inf = g.info()
        N += inf["n_nodes"]
        nnz += inf["nnz"]
        E += inf["n_edges"]
        gs.append(g)
    dts = [g.cfl_timestep(0.5) for g in gs]

    def reset():
        for g, wl in zip(gs, wls):
            g.set_solution(wl.u0)

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    b = afc.Batch(gs)
    res = {}
    sols = {}
    for name, prec in (("mixed", afc.AFC_MIXED), ("fp64", afc.AFC_FP64)):
        opts = afc.default_opts(scheme=afc.AFC_SSP3, precision=prec)
        if shape is None:
            tuning = b.tune(opts, dt=dts)
        else:
            b.set_tuning(*shape)
            tuning = b.get_tuning()
        reset()
        b.step(opts, dt=dts, nsteps=2)   # warm
        reset()
        _, l0 = b.info()
        ms = timed(lambda: b.step(opts, dt=dts, nsteps=steps))
        _, l1 = b.info()
        sols[name] = [g.get_solution() for g in gs]
        umin = min(float(u.min()) for u in sols[name])
        umax = max(float(u.max()) for u in sols[name])
        # algorithmic FP64 work per stage: SpMV 2 nnz, raw fluxes 5 per pair (FP64 only),
        # P+/- 1 per directed pair, alpha r 2 per directed pair, 16 per node
        flops = 3 * steps * (2.0 * nnz + (5.0 * E if prec == afc.AFC_FP64 else 0.0) + 6.0 * E + 16.0 * N)
        res[name] = {"ms": ms, "solves_per_s": count / (ms / 1e3), "dof_stages_per_s": N * 3 * steps / (ms / 1e3),
                     "tuning": tuning, "gpu_launches": l1 - l0 - 1, "umin": umin, "umax": umax,
                     "alu": {"bound": "alu", "achieved": flops / (ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                             "unit": "TFLOP/s", "frac": flops / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS}}
    b.close()
    # the plain path: one problem at a time, afc_step (FP64, one CUDA graph per step)
    reset()
    ms_solo = 0.0
    for q, g in enumerate(gs if solo else []):
        o = afc.default_opts(scheme=afc.AFC_SSP3, dt=dts[q])
        g.step(o)   # graph build
        g.set_solution(wls[q].u0)

        def run(g=g, o=o):
            for _ in range(steps):
                g.step(o)
        ms_solo += timed(run)
    solo_u = [g.get_solution() for g in gs]
    same = all(np.array_equal(a, c) for a, c in zip(solo_u, sols["fp64"])) if solo else None
    err = max(float(np.abs(m - f).max()) for m, f in zip(sols["mixed"], sols["fp64"]))
    scale = max(float(np.abs(f).max()) for f in sols["fp64"])
    for g in gs:
        g.close()
    return {"workload": f"{count} independent transient Q1 problems, nodes per side uniform in [17, 49] "
                        f"(numpy default_rng({seed})), eps log-uniform [1e-8, 1e-4], random unit constant b, hump "
                        f"radius 0.15 at a random centre; SSP3 Zalesak FCT, CFL 0.5, {steps} steps",
            "instances": count, "total_dofs": N, "nnz": nnz, "edges": E, "steps": steps,
            "batched_mixed": res["mixed"], "batched_fp64": res["fp64"],
            "one_at_a_time_fp64": {"ms": ms_solo, "solves_per_s": count / (ms_solo / 1e3),
                                   "dof_stages_per_s": N * 3 * steps / (ms_solo / 1e3)} if solo else None,
            "speedup_mixed_vs_one_at_a_time_fp64": ms_solo / res["mixed"]["ms"] if solo else None,
            "mixed_max_abs_diff_vs_fp64": err, "mixed_rel_diff_vs_fp64": err / scale,
            "batched_fp64_bitwise_equal_to_one_at_a_time": same}


def serving(afc, W, rates=(10.0, 20.0, 50.0, 100.0, 200.0, 500.0), count=48, seed=5, stat_maxit=1000,
            serial_rates=(10.0, 500.0), workers=8, builders=4):
    """Poisson streams of stationary and transient CDR requests (P1 or Q1, nodes per
    side uniform in [17, 97], eps log-uniform [1e-8, 1e-4], c uniform [0, 1]):
    the batched server with mixed precision against the serial server with FP64
    (one request at a time), latency p50 / p99 and solves/s per arrival rate.  Only
    converged results count: a stationary request that ends AFC_NOT_CONVERGED (the
    fixed point did not reach its tolerance within stat_maxit iterations) is
    reported as not converged and left out of solves/s and the latencies.  The
    serial arm runs at `serial_rates` only: one request at a time, it is saturated
    at every rate of the sweep."""
    mix = W.serving_mix(np.random.default_rng(seed), count)

    def opts(kind, prec):
        if kind == "transient":
            return afc.default_opts(scheme=afc.AFC_SSP3, precision=prec)
        return afc.default_opts(limiter=afc.AFC_LIM_MC, omega=0.5, ksp=afc.AFC_KSP_GMRES, ksp_atol=0.0,
                                ksp_rtol=MC_INNER_RTOL, fp_tol=1e-8, fp_maxit=stat_maxit, precision=prec)

    def reqs(prec):
        out = []
        for kind, wl in mix:
            k = afc.AFC_REQ_TRANSIENT if kind == "transient" else afc.AFC_REQ_STATIONARY
            out.append(afc.Request(k, wl.elem, wl.n, wl.eps, wl.c, wl.b, wl.u0, wl.dir_mask, wl.u_dir, f=wl.f,
                                   opts=opts(kind, prec), steps=50, cfl=0.5))
        return out

    arms = {"batched_mixed": (afc.AFC_SERVE_BATCHED, reqs(afc.AFC_MIXED)),
            "serial_fp64": (afc.AFC_SERVE_SERIAL, reqs(afc.AFC_FP64))}
    rows = []
    sols = {}
    for rate in rates:
        arr = np.cumsum(np.random.default_rng(int(seed * 1000 + rate)).exponential(1.0 / rate, size=count))
        row = {"rate_per_s": rate}
        for name, (mode, rq) in arms.items():
            if name == "serial_fp64" and rate not in serial_rates:
                continue
            with afc.Server(mode=mode, stationary_workers=workers, max_chunk=10, builders=builders) as srv:
                t0 = time.perf_counter()
                ids = []
                for t_arr, r in zip(arr, rq):
                    dt = t0 + t_arr - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                    ids.append(srv.submit(r))
                lat, done, first, conv, failed, fp_its = [], [], None, [], [], []
                for q, rid in enumerate(ids):
                    res, u = srv.wait(rid, timeout=-1.0, want_u=(rate == rates[-1]))
                    ok = res["state"] == afc.AFC_REQ_DONE and res["status"] == afc.AFC_OK
                    conv.append(ok)
                    if not ok:
                        kind, wl = mix[q]
                        failed.append({"request": q, "kind": kind, "name": wl.name, "state": res["state"],
                                       "status": res["status"], "message": res["message"]})
                    if mix[q][0] == "stationary":
                        fp_its.append(res["stats"]["outer_its"])
                    lat.append(res["t_done"] - res["t_submit"])
                    done.append(res["t_done"])
                    first = res["t_submit"] if first is None else min(first, res["t_submit"])
                    if u is not None:
                        sols.setdefault(name, []).append(u)
                    srv.release(rid)
                info = srv.info()
            lat = np.asarray(lat) * 1e3
            conv = np.asarray(conv)
            span = max(done) - first
            lc = lat[conv] if conv.any() else np.asarray([np.nan])
            row[name] = {"p50_ms": float(np.percentile(lc, 50)), "p99_ms": float(np.percentile(lc, 99)),
                         "solves_per_s": int(conv.sum()) / span, "makespan_s": span,
                         "converged": int(conv.sum()), "not_converged": failed,
                         "stationary_fp_its_mean": float(np.mean(fp_its)) if fp_its else None,
                         "max_batch": info["max_batch"], "chunks": info["chunks"],
                         "mean_batch": info["instance_steps"] / info["batched_steps"] if info["batched_steps"] else None,
                         "p50_ms_by_kind": {k: float(np.percentile([l for l, c, (kk, _) in zip(lat, conv, mix)
                                                                    if kk == k and c] or [np.nan], 50))
                                            for k in ("stationary", "transient")}}
        if "serial_fp64" in row:
            row["speedup_solves_per_s"] = row["batched_mixed"]["solves_per_s"] / row["serial_fp64"]["solves_per_s"]
        rows.append(row)
    diff = max((float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
                for a, b in zip(sols.get("batched_mixed", []), sols.get("serial_fp64", [])) if np.abs(a).max() > 0),
               default=None)
    n_st = sum(k == "stationary" for k, _ in mix)
    return {"workload": f"{count} requests per rate (numpy default_rng({seed})): {n_st} stationary MC (inflow problem, "
                        f"omega 0.5, tol 1e-8, at most {stat_maxit} fixed-point iterations, Jacobi-GMRES(20) rtol "
                        f"{MC_INNER_RTOL:g}), {count - n_st} transient SSP3 Zalesak (50 steps, CFL 0.5); P1/Q1, "
                        f"n in [17, 97], "
                        f"eps log-uniform [1e-8, 1e-4], c in [0, 1]; Poisson arrivals",
            "rates": rows, "mixed_max_rel_diff_vs_fp64": diff,
            "arms": f"batched_mixed: {builders} builders, continuous batching of transient requests, {workers} "
                    "concurrent stationary solves, FP32 inner solves / fluxes, float-pair MC residual; serial_fp64: "
                    "one request at a time, "
                    f"FP64, at rates {list(serial_rates)}"}


def _summary(value, e2e, roof, mixed, sweep, bat, srv, cpu):
    """The headline numbers of every leg in a few hundred bytes (the full records follow)."""
    r3 = lambda x: None if x is None else float(f"{x:.4g}")   # noqa: E731
    out = {"cn_q1_65": {"dof_iters_per_s": r3(value), "e2e": r3(e2e["value"]),
                        "mixed": r3(mixed["value"]) if mixed else None,
                        "top_kernel": roof["kernel"] if roof else None, "top_frac_fp64": r3(roof["frac"]) if roof else None}}
    if sweep:
        out["mc_sweep_p1_129"] = {"ms": r3(sweep["ms_per_sweep"]), "hbm_frac": r3(sweep["hbm"]["frac"]),
                                  "hbm_gbs": r3(sweep["hbm"]["achieved"])}
        if sweep.get("solve"):
            sv = sweep["solve"]
            out["mc_solve_p1_129"] = {"s": r3(sv["ms"] / 1e3), "fp_its": sv["fixed_point_its"],
                                      "gmres_its": sv["gmres_its"], "umin": r3(sv["umin"])}
    if bat:
        out["batched_256"] = {"mixed_solves_per_s": r3(bat["batched_mixed"]["solves_per_s"]),
                              "fp64_solves_per_s": r3(bat["batched_fp64"]["solves_per_s"]),
                              "one_at_a_time_fp64_solves_per_s": r3((bat["one_at_a_time_fp64"] or {}).get("solves_per_s")),
                              "speedup": r3(bat["speedup_mixed_vs_one_at_a_time_fp64"]),
                              "mixed_rel_diff": r3(bat["mixed_rel_diff_vs_fp64"])}
    if srv:
        out["serving"] = [{"rate": r["rate_per_s"],
                           "batched": [r3(r["batched_mixed"]["solves_per_s"]), r3(r["batched_mixed"]["p50_ms"]),
                                       r3(r["batched_mixed"]["p99_ms"]), r["batched_mixed"]["max_batch"],
                                       r3(r["batched_mixed"]["mean_batch"]), r["batched_mixed"]["converged"]],
                           "serial": [r3(r["serial_fp64"]["solves_per_s"]), r3(r["serial_fp64"]["p50_ms"]),
                                      r3(r["serial_fp64"]["p99_ms"]), r["serial_fp64"]["converged"]]
                           if "serial_fp64" in r else None} for r in srv["rates"]]
        out["serving_fields"] = ("batched: solves/s, p50 ms, p99 ms, max batch, mean batch, converged; "
                                 "serial: solves/s, p50 ms, p99 ms, converged")
    if cpu:
        out["cpu"] = {"dof_iters_per_s": r3(cpu["value"]), "cores": cpu["cores"],
                      "single_thread": r3(cpu["single_thread"]["value"])}
    return out


def run_ours(args, ws, rank, local):
    import torch
    import torch.distributed as dist

    from paper_2110_15676_gb300 import afc
    from paper_2110_15676_gb300 import workloads as W

    torch.cuda.set_device(local)
    if args.only_serving:
        print(json.dumps({"serving": serving(afc, W, count=args.serving_count, workers=args.serving_workers,
                                             builders=args.serving_builders)}))
        return
    if args.only_batched:
        shape = None
        if args.batched_mode != "auto":
            mode = {"pass": afc.AFC_BATCH_PER_PASS, "stage": afc.AFC_BATCH_PER_STAGE,
                    "step": afc.AFC_BATCH_PER_STEP}[args.batched_mode]
            shape = (mode, args.batched_block)
        print(json.dumps({"batched": batched(afc, W, torch, torch.cuda.current_stream(), count=args.batched_count,
                                             shape=shape, solo=not args.no_solo)}))
        return
    if args.only_mc_sweep:
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        rt = tuple(float(x) for x in args.mc_inner_rtols.split(",")) if args.mc_inner_rtols else ()
        print(json.dumps({"mc_sweep": mc_sweep(afc, W, torch, flush, torch.cuda.current_stream(),
                                               max(args.steps, 1), solve=not args.no_mc_solve, inner_rtols=rt)}))
        return
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    P, wl = _make_problem(afc, W, afc.AFC_MIXED)
    info = P.info()
    N, nnz, E = info["n_nodes"], info["nnz"], info["n_edges"]
    dt = P.cfl_timestep(CFL)
    opts = _opts(afc, dt)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 512 MB > L2
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        P.step(opts)
    barrier()
    clocks = ClockSampler(local)
    time.sleep(0.3)
    launches0 = P.launches()
    barrier()
    ms_total, its_total, inner_total, statuses = _timed_steps(P, opts, args.steps, flush, stream, torch)
    barrier()
    clk = clocks.stop()
    gpu_launches = P.launches() - launches0
    value, ms_max = whole_job(float(N) * its_total, ms_total, ws, device="cuda")

    # per-kernel device time: the same steps again, issued launch by launch (a CUDA graph's
    # nodes cannot carry events), with every launch bracketed by events on the stream
    P.profile(True)
    popts = _opts(afc, dt)
    popts.graph = 0
    _, _, p_inner, _ = _timed_steps(P, popts, args.steps, flush, stream, torch)
    prof, _ = P.profile_read()
    P.profile(False)
    tot_ms = sum(v[0] for v in prof.values())
    name, (kms, kcount) = max(prof.items(), key=lambda kv: kv[1][0])
    bound, work, unit = _kernel_work(name, N, nnz, E, p_inner / max(kcount, 1))
    roof = _roofline(name, kms, kcount, work, kms / tot_ms) if bound == "alu" else None

    # mixed precision variant (FP32 inner BiCGStab), same workload
    mixed = None
    if args.steps > 0:
        Pm, _ = _make_problem(afc, W, afc.AFC_MIXED)
        om = _opts(afc, dt, mixed=True)
        for _ in range(max(1, args.warmup)):
            Pm.step(om)
        torch.cuda.synchronize()
        mms, mits, _, _ = _timed_steps(Pm, om, args.steps, flush, stream, torch)
        Pr, _ = _make_problem(afc, W, afc.AFC_FP64)
        for _ in range(max(1, args.warmup) + args.steps):
            Pr.step(opts)
        um, ur = Pm.get_solution(), Pr.get_solution()
        mixed = {"value": float(N) * mits / (mms / 1e3), "ms_per_step": mms / args.steps,
                 "fixed_point_its": mits, "rel_err_vs_fp64": float(np.abs(um - ur).max() / np.abs(ur).max())}
        del Pm, Pr

    # end to end through the public API with host buffers (H2D of u, step, D2H of u)
    import ctypes
    host_u = torch.empty(N, dtype=torch.float64).pin_memory()
    host_u.copy_(torch.from_numpy(P.get_solution()))
    out_u = torch.empty(N, dtype=torch.float64).pin_memory()
    e2e_ms, e2e_its = 0.0, 0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        afc._check(afc._lib.afc_set_solution(P.h, ctypes.c_void_p(host_u.data_ptr()), 0), "afc_set_solution")
        st = P.step(opts)
        afc._check(afc._lib.afc_get_solution(P.h, ctypes.c_void_p(out_u.data_ptr()), 0), "afc_get_solution")
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_its += st["outer_its"]
        host_u.copy_(out_u)
    e2e_value, _ = whole_job(float(N) * e2e_its, e2e_ms, ws, device="cuda")
    e2e = {"value": e2e_value, "unit": "dof-iters/s", "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N}

    sweep = None
    if not args.no_mc_sweep and args.steps > 0:
        del P
        sweep = mc_sweep(afc, W, torch, flush, stream, max(args.steps, 5))

    bat = None
    if not args.no_batched and args.steps > 0:
        bat = batched(afc, W, torch, stream)

    srv = None
    if not args.no_serving and args.steps > 0:
        srv = serving(afc, W, count=args.serving_count, workers=args.serving_workers, builders=args.serving_builders)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_rounds)

    # every profiled kernel with its algorithmic FP64 work: achieved rate and fraction of the pipe
    kernel_table = {}
    for k, (kms_k, kc_k) in sorted(prof.items(), key=lambda kv: -kv[1][0])[:10]:
        row = {"ms": kms_k, "launches": kc_k, "share": kms_k / tot_ms}
        b_k, w_k, _ = _kernel_work(k, N, nnz, E, p_inner / max(kc_k, 1))
        if b_k == "alu":
            ach = w_k / (kms_k / kc_k / 1e3) / 1e12
            row.update({"bound": "alu", "achieved_tflops": ach, "frac": ach / FP64_PEAK_TFLOPS})
        kernel_table[k] = row

    if rank == 0:
        summary = _summary(value, e2e, roof, mixed, sweep, bat, srv, cpu)
        line = {
            "metric": METRIC, "value": value, "unit": "dof-iters/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "dofs": N, "nnz": nnz, "edges": E, "dt": dt,
                       "fixed_point_its": its_total, "krylov_its": inner_total,
                       "l2": "flushed (512 MB write) before every timed step", "parallelism": f"replicas x{ws}"},
            "summary": summary,
            "clocks": clk, "e2e": e2e, "gpu_launches": gpu_launches, "roofline": roof,
            "kernels": kernel_table,
            "kernel_times": "second pass of the same steps, launches issued one by one with per-launch CUDA "
                            "events (the timed pass runs each step as one CUDA graph)",
            "mixed": mixed, "mc_sweep": sweep, "batched": bat, "serving": srv, "cpu_baseline": cpu,
            "summary_again": summary,
        }
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def _oracle_problem():
    from oracle import afc_oracle as O
    from paper_2110_15676_gb300 import workloads as W
    wl = W.rotating_transient(ELEM, N_SIDE)
    mesh = O.structured_mesh(wl.elem, wl.n)
    o = O.assemble(mesh, wl.eps, wl.b, wl.c, wl.f, wl.dir_mask.astype(bool), wl.u_dir)
    dt = O.cfl_timestep(o, CFL)
    return O, o, wl, dt


# The CPU unit of work, the same for the CPU baseline and the reference arm: one call of
# the oracle's CN step from u0 with a single fixed-point correction (its predictor, its
# system matrix, one limiter pass, one BiCGStab solve to atol 1e-12, the update).
_ORACLE = {}


def _oracle_worker_init():
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    _ORACLE["p"] = _oracle_problem()


def _oracle_unit(_=None):
    O, o, wl, dt = _ORACLE["p"]
    t0 = time.perf_counter()
    _, st = O.cn_step(o, wl.u0, dt, tol=FP_TOL, ksp_atol=KSP_ATOL, fixed_iterations=1)
    return st["outer_its"], time.perf_counter() - t0


def _host_cores():
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return n, model


class OraclePool:
    """The oracle on every host core: one spawned process per core (spawn, so that no
    child inherits a CUDA context), each with the problem assembled once and one BLAS
    thread; a round runs one unit per core and is timed on the parent's clock."""

    def __init__(self, procs):
        import multiprocessing as mp
        self.procs = procs
        self.pool = mp.get_context("spawn").Pool(procs, initializer=_oracle_worker_init)
        self.pool.map(_oracle_unit, range(procs))     # warm-up round (and assembly)

    def round(self):
        t0 = time.perf_counter()
        its = sum(i for i, _ in self.pool.map(_oracle_unit, range(self.procs)))
        return its, time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(rounds: int) -> dict:
    """The CPU oracle, as it stands, on a bounded sample of the same workload: the
    unit above (one CN step with one fixed-point correction), one thread, and all host
    cores (one process per core) for `rounds` rounds."""
    _oracle_worker_init()
    N = _ORACLE["p"][1].mesh.n_nodes
    _oracle_unit()
    its1, sec1 = 0, 0.0
    for _ in range(rounds):
        i, t = _oracle_unit()
        its1 += i
        sec1 += t
    cores, model = _host_cores()
    pool = OraclePool(cores)
    itsc, secc = 0, 0.0
    for _ in range(rounds):
        i, t = pool.round()
        itsc += i
        secc += t
    pool.close()
    unit = "one oracle CN step (Q1 65^3) with one fixed-point correction"
    return {"value": N * itsc / secc, "unit": "dof-iters/s", "cores": cores, "kind": "oracle", "cpu": model,
            "sample": f"{rounds} rounds of {cores} concurrent units ({unit}), one per core ({secc:.1f} s)",
            "single_thread": {"value": N * its1 / sec1, "cores": 1,
                              "sample": f"{rounds} units ({unit}) on one thread ({sec1:.1f} s)"}}


def run_reference(args, ws, rank):
    """Reference arm: the CPU oracle timed on the same workload and unit as the CPU
    baseline; each step is one round of one unit per host core."""
    if rank != 0:
        return
    cores, model = _host_cores()
    pool = OraclePool(cores)
    O, o, wl, dt = _oracle_problem()
    N = o.mesh.n_nodes
    for _ in range(args.warmup):
        pool.round()
    its, sec = 0, 0.0
    for _ in range(args.steps):
        i, t = pool.round()
        its += i
        sec += t
    pool.close()
    value = N * its / sec
    sample = (f"per step one round of {cores} concurrent units (one oracle CN step with one fixed-point "
              f"correction each), one per host core")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "dof-iters/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "dofs": N, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "dof-iters/s", "cores": cores, "kind": "oracle", "cpu": model,
                             "sample": sample},
            "e2e": {"value": value, "unit": "dof-iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mc-sweep", action="store_true")
    ap.add_argument("--only-mc-sweep", action="store_true", help="time only the P1 129^3 MC sweep")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--only-batched", action="store_true", help="time only the 256-instance batched SSP3 run")
    ap.add_argument("--batched-count", type=int, default=256, help="instances of the batched run (--only-batched)")
    ap.add_argument("--batched-mode", default="auto", choices=["auto", "pass", "stage", "step"],
                    help="launch shape of the batched run (--only-batched); auto = tuned")
    ap.add_argument("--batched-block", type=int, default=128)
    ap.add_argument("--no-solo", action="store_true", help="skip the one-at-a-time path (--only-batched)")
    ap.add_argument("--no-mc-solve", action="store_true", help="time the MC sweep but not the whole MC solve")
    ap.add_argument("--mc-inner-rtols", default="", help="--only-mc-sweep: also solve with these inner GMRES "
                                                          "tolerances (comma separated) and compare")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--only-serving", action="store_true", help="time only the request-server streams")
    ap.add_argument("--serving-count", type=int, default=48)
    ap.add_argument("--serving-workers", type=int, default=8, help="concurrent stationary solves of the server")
    ap.add_argument("--serving-builders", type=int, default=4, help="problem-building threads of the server")
    ap.add_argument("--cpu-rounds", type=int, default=2, help="timed rounds of the CPU baseline")
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
