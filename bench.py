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


# Algorithmic work per launch of the kernels that can dominate (stated in the design notes):
#   FP64 flops: SpMV 2 per pattern entry; BiCGStab fused dots 2 per row.
def _kernel_work(name, N, nnz, E):
    if name.startswith("k_bicg_spmv"):
        return ("alu", 2.0 * nnz + 2.0 * N, "TFLOP/s")
    if name == "k_cn_residual":
        # r_ij (8) + alpha r_ij (1) per directed pair, SpMV 2 per entry
        return ("alu", 9.0 * 2 * E + 2.0 * nnz, "TFLOP/s")
    if name == "k_cn_factors":
        return ("alu", 9.0 * 2 * E, "TFLOP/s")
    return (None, None, None)


def run_ours(args, ws, rank, local):
    import torch
    import torch.distributed as dist

    from paper_2110_15676_gb300 import afc
    from paper_2110_15676_gb300 import workloads as W

    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    P, wl = _make_problem(afc, W, afc.AFC_MIXED)
    info = P.info()
    N, nnz, E = info["n_nodes"], info["nnz"], info["n_edges"]
    dt = P.cfl_timestep(CFL)
    opts = _opts(afc, dt)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # 512 MB > L2

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
    P.profile(True)
    stream = torch.cuda.current_stream()
    ms_total, its_total, inner_total = 0.0, 0, 0
    statuses = []
    barrier()
    for _ in range(args.steps):
        flush.fill_(1.0)                       # evict L2 between timed steps (not timed)
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
    barrier()
    clk = clocks.stop()
    prof, launches1 = P.profile_read()
    P.profile(False)
    gpu_launches = launches1 - launches0
    t = torch.tensor([ms_total], device="cuda", dtype=torch.float64)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    units = float(N) * its_total * ws
    value = units / (ms_max / 1e3)

    # dominant kernel and its roofline
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    name, (kms, kcount) = dom
    bound, work, unit = _kernel_work(name, N, nnz, E)
    peaks, peak_src = _peaks()
    roof = None
    if bound == "alu":
        achieved = work / (kms / kcount / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": unit,
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "FP64 pipe 152 SM x 2 DFMA/clk x 2.07 GHz",
                "avg_launch_us": kms / kcount * 1e3, "share": kms / sum(v[0] for v in prof.values())}

    # mixed precision variant (FP32 inner BiCGStab), same workload, fewer steps
    mixed = None
    if args.steps > 0:
        Pm, _ = _make_problem(afc, W, afc.AFC_MIXED)
        om = _opts(afc, dt, mixed=True)
        for _ in range(max(1, args.warmup)):
            Pm.step(om)
        torch.cuda.synchronize()
        mms, mits = 0.0, 0
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = Pm.step(om)
            e1.record(stream)
            e1.synchronize()
            mms += e0.elapsed_time(e1)
            mits += st["outer_its"]
        # accuracy of the mixed result against the FP64 path after the same number of steps
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
    te = torch.tensor([e2e_ms], device="cuda", dtype=torch.float64)
    if ws > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e = {"value": float(N) * e2e_its * ws / (float(te.item()) / 1e3), "unit": "dof-iters/s",
           "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample_its)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "dof-iters/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "dofs": N, "nnz": nnz, "edges": E, "dt": dt,
                       "fixed_point_its": its_total, "krylov_its": inner_total,
                       "l2": "flushed (512 MB write) before every timed step", "parallelism": f"replicas x{ws}"},
            "clocks": clk, "e2e": e2e, "gpu_launches": gpu_launches, "roofline": roof,
            "kernels": {k: {"ms": v[0], "launches": v[1]} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])[:8]},
            "mixed": mixed, "cpu_baseline": cpu,
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


def cpu_baseline(sample_its: int) -> dict:
    """The CPU oracle, as it stands, on a bounded sample of the same workload: the
    first `sample_its` fixed-point corrections of one CN step (single thread)."""
    O, o, wl, dt = _oracle_problem()
    t0 = time.perf_counter()
    _, st = O.cn_step(o, wl.u0, dt, tol=FP_TOL, ksp_atol=KSP_ATOL, fixed_iterations=sample_its)
    sec = time.perf_counter() - t0
    N = o.mesh.n_nodes
    return {"value": N * st["outer_its"] / sec, "unit": "dof-iters/s", "cores": 1, "kind": "oracle",
            "sample": f"{st['outer_its']} fixed-point corrections of one CN step on the same 65^3 Q1 problem "
                      f"({sec:.1f} s)"}


def run_reference(args, ws, rank):
    """Reference arm: the CPU oracle timed on the same workload; each step is a
    bounded sample (one fixed-point correction of a CN step)."""
    if rank != 0:
        return
    O, o, wl, dt = _oracle_problem()
    N = o.mesh.n_nodes
    u = wl.u0.copy()
    for _ in range(args.warmup):
        O.cn_step(o, u, dt, tol=FP_TOL, ksp_atol=KSP_ATOL, fixed_iterations=1)
    t0 = time.perf_counter()
    its = 0
    for _ in range(args.steps):
        _, st = O.cn_step(o, u, dt, tol=FP_TOL, ksp_atol=KSP_ATOL, fixed_iterations=1)
        its += st["outer_its"]
    sec = time.perf_counter() - t0
    value = N * its / sec
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "dof-iters/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "dofs": N, "sample": "one fixed-point correction of a CN step per step"},
            "cpu_baseline": {"value": value, "unit": "dof-iters/s", "cores": 1, "kind": "oracle",
                             "sample": "one fixed-point correction of a CN step per step"},
            "e2e": {"value": value, "unit": "dof-iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-its", type=int, default=6)
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
