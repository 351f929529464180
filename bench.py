#!/usr/bin/env python3
"""Benchmark: PCG time-to-1e-8 with the two-level GenEO preconditioner.

Workload: the 32^3 unit cube with a through-hole (central 8x8x32 column
removed), mu^-1 log-uniform in [1, 1e3] inside four random 2x2 channels,
eps = 1, gamma = 1e-4, f uniform in [-1, 1]^3 per edge (seeded), 4x4x4 = 64
subdomains, overlap 2, GenEO threshold lambda > 10 (tau = 0.1, reciprocal).

A step is one preconditioned CG solve to ||r|| / ||b|| <= 1e-8 on the GPU in
the balanced form (x0 = Z E^-1 Z^T b, one coarse solve per iteration), the
right-hand side resident in HBM (the local factors, 10-22 GB, exceed the
129 MB L2, so no flush is needed).  The literal form (x0 = 0, two coarse
solves per iteration), plain float64 local factors and the refined solves
(accurate residuals) are timed beside it, and every solution is compared
with the oracle's stored accurate solution.  Set-up (assembly, local
inverses, GenEO eigensolves, coarse factor) is timed separately.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch with torch.distributed.run; each rank solves its own
replica of the problem (replicas only: the method is not sharded here).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG time-to-1e-8 (s)"
TOL = 1e-8
WORKLOAD = "cube32_hole_channels"
BLOCK_WORKLOAD = "beam128_layered"
WARM_WORKLOAD = "cube24_blocks"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="mixed", choices=["fp64", "mixed"],
                   help="mixed: float32 split local factors (headline) and float64 beside it")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--many-gb", type=float, default=24.0,
                   help="many_problems: memory budget for the local factors (float64 + float32)")
    p.add_argument("--workload", default=WORKLOAD,
                   choices=[WORKLOAD, "cube16_hole_channels", BLOCK_WORKLOAD, "beam128_mild",
                            "beam64_layered", WARM_WORKLOAD, "paper_beam", "spmv_cube48",
                            "many_problems"],
                   help="cube16_hole_channels: the profiling-size companion (ncu captures); "
                        f"{BLOCK_WORKLOAD}: 16 right-hand sides as a block, bfloat16 local "
                        "factors on the tensor cores")
    return p.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# DRAM traffic of the float32 streaming SYMV per algorithmic byte, from one ncu
# capture on cube16_hole_channels of the configuration the autotuner chose there
# ({6 stages, 4 tiles per barrier, 8 warps, 2 CTAs per SM}; every configuration
# reads each stored tile once and writes one float column partial per tile):
# (204.64 MB read + 5.04 MB written) / 203.69 MB of stored tiles.  Traffic
# scales with the stored tiles, so the full launch's traffic is this ratio
# times its algorithmic bytes.  Set to None when the kernel changes until it is
# captured again.
SYMV_F32_TRAFFIC_RATIO = (204.6372 + 5.0365) / 203.6859  # (read + written) / stored tiles

# FP64 FMA rate of GB300: 152 SMs x 2 FP64 FMA / clock / SM x 2 flop x 2070 MHz
# (the recipe's 1.25 TFLOP/s nominal figure at the maximum SM clock)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070


def peaks_hbm():
    return load_peaks()[0]["hbm_gbs"]


def max_over_ranks(value, world, device):
    """Largest value over the ranks: a timed region ends when the slowest rank
    ends (each rank solves its own replica)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, seconds, world):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return units_per_rank * world / seconds


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = str(index)
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9 or f[0] != self.index:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle, bounded sample (baseline only)

def cpu_model():
    """Host CPU model name (lscpu, else /proc/cpuinfo, else the platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


class OracleSample:
    """One preconditioned CG iteration of the CPU oracle on the same
    workload: the local sparse-LU solves of all 64 subdomains, the coarse
    solves on the split near-kernel columns (the GenEO columns add under 1%
    to n0; the oracle's dense GenEO eigensolves take about an hour, so they
    are left out of this baseline's set-up), the global SpMVs and the vector
    updates.  Set-up happens once in the constructor."""

    def __init__(self, seed=0):
        import numpy as np
        import scipy.sparse as sp
        import scipy.sparse.linalg as spla
        import workloads as W
        from oracle.mesh import build_mesh
        from oracle.fem import assemble_A
        from oracle.dd import decompose
        from oracle.coarse import snk_columns, assemble_Z, coarse_matrix
        w = getattr(W, WORKLOAD)()
        m = build_mesh(w.nx, w.ny, w.nz, (w.hx, w.hy, w.hz), w.active)
        self.A = assemble_A(m, w)
        dec = decompose(m, w.parts, w.overlap)
        self.nsub = dec.nsub
        self.Z = assemble_Z(self.A.shape[0], snk_columns(m, dec))
        self.Elu = spla.splu(sp.csc_matrix(coarse_matrix(m, w, self.Z)))
        self.facs = [(dec.N[i], spla.splu(sp.csc_matrix(self.A[dec.N[i]][:, dec.N[i]])))
                     for i in range(dec.nsub)]
        rng = np.random.default_rng(seed)
        self.r = rng.standard_normal(self.A.shape[0])
        self.info = {"sample": f"one PCG iteration of the oracle on {WORKLOAD} "
                               f"(n={self.A.shape[0]}): local sparse-LU solves of all "
                               f"{dec.nsub} subdomains, coarse sparse-LU solves on the "
                               f"{self.Z.shape[1]} split near-kernel columns",
                     "cores": os.cpu_count(), "cpu": cpu_model()}

    def step(self):
        import numpy as np
        A, Z, Elu, r = self.A, self.Z, self.Elu, self.r
        t0 = time.perf_counter()
        y0 = Z @ Elu.solve(Z.T @ r)
        s = r - A @ y0
        wv = np.zeros_like(r)
        for Ni, f in self.facs:
            wv[Ni] += f.solve(s[Ni])
        z = y0 + wv - Z @ Elu.solve(Z.T @ (A @ wv))
        q = A @ z
        alpha = (r @ z) / (z @ q)
        rr = r - alpha * q
        _ = rr @ rr
        return time.perf_counter() - t0


def oracle_iterations(default):
    path = os.path.join(ROOT, "tests", "golden", "cube32_reference.json")
    if os.path.exists(path):
        with open(path) as f:
            return int(json.load(f)["pcg_iters"]), "oracle PCG iteration count (tests/golden)"
    return default, "iteration count of the GPU run (same method)"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    o = OracleSample()
    for _ in range(args.warmup):
        o.step()
    per_iter = statistics.median([o.step() for _ in range(max(1, args.steps))])
    info = o.info
    iters, src = oracle_iterations(40)
    value = per_iter * iters
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": value * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "tol": TOL, "iterations": iters,
                       "iterations_source": src},
            "cpu_baseline": {"value": value, "unit": "s", "cores": info["cores"],
                             "cpu": info["cpu"], "kind": "oracle",
                             "sample": info["sample"] + f"; per-iteration median x {iters} "
                                       f"iterations ({src})"},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------

def run_block(args):
    """Block of 16 right-hand sides (beam128_layered): time to 1e-8 for every
    column with bfloat16 split local factors on the tensor cores, the float32
    split and float64 local factors (all with the exact gradient shift), on
    the same GPU.  A variant whose preconditioner does not converge is
    reported with its status; the headline is the fastest variant that
    converged.  The tensor-core kernel's roofline is measured in any case."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import workloads as W
    import paper_2311_18783_gb300 as pkg
    w = getattr(W, args.workload)()
    t0 = time.perf_counter()
    # gamma = 1e-6 under a 1e6 jump of mu^-1 makes the local matrices
    # numerically singular: invert them with the exact gradient shift
    # balanced form: one coarse solve per iteration, as in the headline
    s = pkg.Solver.from_workload(w, precision=pkg.PREC_BF16, gradient_shift=1, balanced=1)
    setup_s = time.perf_counter() - t0
    n, k = s.n, w.f_slot.shape[0]
    B = torch.empty((k, n), dtype=torch.float64, device="cuda")
    for j in range(k):
        s.assemble_rhs(w.f_slot[j], B[j])
    X = torch.empty_like(B)
    stream = torch.cuda.current_stream()
    maxit = 400

    def timed(prec, steps, warmup, prof=False):
        s.use_precision(prec)
        for _ in range(warmup):
            s.solve_block(B, X, tol=TOL, maxit=maxit)
        torch.cuda.synchronize()
        if prof:
            s.profile(True)
            s.profile_read()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            st, infos = s.solve_block(B, X, tol=TOL, maxit=maxit)
        e1.record(stream)
        torch.cuda.synchronize()
        prof_out = None
        if prof:
            prof_out = s.profile_read()
            s.profile(False)
        return {"ms": e0.elapsed_time(e1) / steps, "status": st,
                "converged": st == 0, "pcg_iters": [i["iters"] for i in infos],
                "max_relres": max(i["relres"] for i in infos)}, prof_out

    variants = {}
    short = max(1, args.steps // 2)
    variants["fp64"], _ = timed(pkg.PREC_FP64, short, 1)
    X64 = X.clone()
    variants["fp32_split"], _ = timed(pkg.PREC_FP32, short, 1)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    variants["bf16_tensor_cores"], prof = timed(pkg.PREC_BF16, args.steps, args.warmup, True)
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    conv = {kk: v for kk, v in variants.items() if v["converged"]}
    head = min(conv, key=lambda kk: conv[kk]["ms"]) if conv else "bf16_tensor_cores"
    prec_of = {"fp64": pkg.PREC_FP64, "fp32_split": pkg.PREC_FP32,
               "bf16_tensor_cores": pkg.PREC_BF16}
    # headline variant, max over ranks
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(variants[head]["ms"], world, "cuda")
    s.use_precision(prec_of[head])
    s.solve_block(B, X, tol=TOL, maxit=maxit)
    diff = max((torch.linalg.norm(X[j] - X64[j]) / torch.linalg.norm(X64[j])).item()
               for j in range(k))
    # end to end with the headline variant: pinned host right-hand sides in,
    # solutions out, every step
    Bh = B.cpu().pin_memory()
    Xh = torch.empty_like(Bh).pin_memory()
    te = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        Bd = Bh.to("cuda", non_blocking=True)
        Xd = torch.empty_like(Bd)
        s.solve_block(Bd, Xd, tol=TOL, maxit=maxit)
        Xh.copy_(Xd, non_blocking=True)
        torch.cuda.synchronize()
        te.append(time.perf_counter() - t1)
    peaks, peak_src = load_peaks()
    t_launch = prof["local_symv_ms"] / max(1, prof["local_symv_launches"]) * 1e-3
    nbytes = prof["local_symv_bytes"]
    flops = prof["local_symv_flops"] * k
    roof = {"kernel": "k_tc_symm (bfloat16 C_j x 16 right-hand sides, tcgen05)", "bound": "hbm",
            "achieved": nbytes / t_launch / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": nbytes / t_launch / 1e9 / peaks["hbm_gbs"],
            "peak_source": f"hbm_gbs of {peak_src}", "traffic": None,
            "algorithmic_bytes_per_launch": nbytes, "launch_ms": t_launch * 1e3,
            "tensor_tflops": flops / t_launch / 1e12,
            "tensor_frac_of_bf16_peak": flops / t_launch / 1e12 / peaks["bf16_tflops"]}
    dtype = {"fp64": "f64", "fp32_split": "f32+f64", "bf16_tensor_cores": "bf16+f64"}[head]
    line = {"metric": METRIC + ", 16 right-hand sides", "value": ms / 1e3, "unit": "s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype, "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "nrhs": k, "nsub": s.sizes["nsub"],
                       "max_ni": s.sizes["max_ni"], "n0": s.sizes["n0"],
                       "n0_geneo": s.sizes["n0_geneo"], "tol": TOL, "maxit": maxit,
                       "headline_variant": head, "gradient_shift": True,
                       "l2": "inputs larger than L2 (bfloat16 factors "
                             f"{nbytes / 1e9:.2f} GB)", "setup_s": setup_s},
            "variants": {kk: {"value": v["ms"] / 1e3, "unit": "s", "status": v["status"],
                              "converged": v["converged"], "pcg_iters": v["pcg_iters"],
                              "max_relres": v["max_relres"]} for kk, v in variants.items()},
            "headline_vs_fp64_solution_max_rel_diff": diff,
            "roofline": roof, "clocks": clk, "gpu_launches": prof["launches"],
            "e2e": {"value": statistics.mean(te), "unit": "s", "h2d_bytes_per_step": k * n * 8,
                    "d2h_bytes_per_step": k * n * 8}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


def run_warm(args):
    """Learned warm start on cube24_blocks (64 subdomains of the 48^3 blocks
    workload's size, mu^-1 in [1, 1e6] on 3^3-cell blocks): the network is
    trained on the eigenvectors the exact set-up produces for 4 coefficient
    draws (4 x 64 local eigenproblems), then the held-out draw of the
    workload is set up cold and warm.  Reports
    GenEO set-up time, LOBPCG iterations (first block and all) and the GenEO
    counts of both starts (the method's result must not change)."""
    import torch
    import numpy as np
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import workloads as W
    import paper_2311_18783_gb300 as pkg
    net = pkg.Mlp(seed=7)
    t_train, losses = 0.0, []
    for seed in (100, 101, 102, 103):
        s = pkg.Solver.from_workload(W.cube24_blocks(seed), keep_eigvecs=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ls = net.train(s, 150, lr=2e-3)
        torch.cuda.synchronize()
        t_train += time.perf_counter() - t0
        losses.append([float(ls[0]), float(ls[-1])])
        s.close()
    w = W.cube24_blocks()
    out = {}
    for name, kw in (("cold", {}), ("warm", {"warm_start": net.handle})):
        t0 = time.perf_counter()
        s = pkg.Solver.from_workload(w, keep_eigvecs=1, **kw)
        setup = time.perf_counter() - t0
        loss, _ = net.loss_grad(s)
        b = torch.empty(s.n, dtype=torch.float64, device="cuda")
        s.assemble_rhs(w.f_slot[0], b)
        x = torch.zeros_like(b)
        info = s.solve(b, x, tol=TOL, maxit=1000)
        out[name] = {"setup_s": setup, "lobpcg_iters_first_block": int(s.export("lobpcg_iters_first").sum()),
                     "lobpcg_iters_all": int(s.export("lobpcg_iters").sum()),
                     "geneo_found": int(s.export("geneo_found").sum()),
                     "n0_geneo": s.sizes["n0_geneo"], "pcg_iters": info["iters"],
                     "trained_net_subspace_loss": loss}
        found = s.export("geneo_found")
        out[name]["_found"] = found
        s.close()
    same = bool(np.array_equal(out["cold"].pop("_found"), out["warm"].pop("_found")))
    line = {"metric": "GenEO set-up time with the learned warm start (s)",
            "value": out["warm"]["setup_s"], "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "higher_is_better": False, "vs_baseline": None, "dtype": "f64 (network bf16)",
            "data": "synthetic",
            "config": {"workload": WARM_WORKLOAD, "train_draws": [100, 101, 102, 103],
                       "train_steps_per_draw": 150, "train_seconds": t_train,
                       "train_loss_first_last": losses, "held_out_seed": 5},
            "cold": out["cold"], "warm": out["warm"], "same_geneo_counts": same}
    print(json.dumps(line), flush=True)
    net.close()


# Table "homogeneous_beam_both" (Sec. 4), N = 8: right-preconditioned GMRES
# iterations to a relative residual of 1e-6 on the (N/2) x 1 x 1 beam at
# h = 1/16, tau = 10, and the GenEO size (0 for every N and both BCs)
PAPER_BEAM_N8 = {"dirichlet": {"AS": 12, "AS-SNK": 14, "AS-SNK-GenEO": 14, "AS-NK": 14,
                               "AS-NK-GenEO": 14},
                 "mixed": {"AS": 20, "AS-SNK": 15, "AS-SNK-GenEO": 15, "AS-NK": 19,
                           "AS-NK-GenEO": 19}}


def run_paper_beam(args):
    """The paper's weak-scaling beam at N = 8 (64 x 16 x 16 cells, h = 1/16,
    8 boxes, one overlap layer, mu = eps = 1, f = (1, 1, 1), gamma = 1e-3,
    lambda > 10), Dirichlet on all faces and mixed (Neumann on the two y
    faces), every coarse variant of Sec. 4 except AMS, solved with
    right-preconditioned GMRES to 1e-6 as in Table "homogeneous_beam_both";
    the paper's iteration counts are printed beside ours (context: the
    paper penalises boundary dofs in FreeFEM, this library eliminates them,
    and the partitions of unity differ)."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import workloads as W
    import paper_2311_18783_gb300 as pkg
    variants = {"AS": dict(coarse=pkg.COARSE_NONE, geneo=0),
                "AS-SNK": dict(coarse=pkg.COARSE_SNK, geneo=0),
                "AS-SNK-GenEO": dict(coarse=pkg.COARSE_SNK, geneo=1),
                "AS-NK": dict(coarse=pkg.COARSE_NK, geneo=0),
                "AS-NK-GenEO": dict(coarse=pkg.COARSE_NK, geneo=1)}
    out = {}
    for bc in ("dirichlet", "mixed"):
        w = W.paper_beam(8)
        if bc == "mixed":
            w.natural = W.natural_faces(w, sides=((1, 0), (1, 1)))
        out[bc] = {}
        for name, kw in variants.items():
            t0 = time.perf_counter()
            s = pkg.Solver.from_workload(w, **kw)
            setup = time.perf_counter() - t0
            b = torch.empty(s.n, dtype=torch.float64, device="cuda")
            s.assemble_rhs(w.f_slot[0], b)
            x = torch.zeros_like(b)
            g = s.solve_gmres(b, x, tol=1e-6, maxit=500, restart=100)
            x2 = torch.zeros_like(b)
            c = s.solve(b, x2, tol=1e-6, maxit=500)
            out[bc][name] = {"gmres_iters": g["iters"], "paper_gmres_iters": PAPER_BEAM_N8[bc][name],
                             "gmres_relres": g["relres"], "gmres_s": g["seconds"],
                             "pcg_iters": c["iters"], "n0": s.sizes["n0"],
                             "n0_geneo": s.sizes["n0_geneo"], "setup_s": setup}
            out[bc]["dofs_unknown"] = s.n
            s.close()
            print(json.dumps({bc: {name: out[bc][name]}}), file=sys.stderr, flush=True)
    line = {"metric": "GMRES iterations to 1e-6 on the paper's N = 8 beam", "value": None,
            "unit": "iterations", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "paper_beam_N8", "cells": [64, 16, 16], "h": 1 / 16,
                       "gamma": 1e-3, "tau_paper": 10, "krylov": "right-preconditioned GMRES(100)",
                       "paper_table": "homogeneous_beam_both, N = 8"},
            "results": out}
    print(json.dumps(line), flush=True)


def time_spmv(s, reps=50):
    """Mean device time of one geneo_spmv launch (the SELL SpMV kernel alone)
    over `reps` back-to-back launches on the current stream, after 5 warm-up
    launches, and its algorithmic bytes: 12 B per stored nonzero of A (value
    and column index) plus 20 B per row (x read, y written, row pointer)."""
    import torch
    n, nnz = s.n, s.sizes["nnz"]
    x = torch.randn(n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(5):
        s.spmv(x, y)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        s.spmv(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / reps * 1e-3
    nbytes = 12 * nnz + 20 * n
    peaks, src = load_peaks()
    return {"kernel": "k_spmv_sell (SELL-32-256, float64)", "bound": "hbm",
            "achieved": nbytes / t / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": nbytes / t / 1e9 / peaks["hbm_gbs"], "peak_source": f"hbm_gbs of {src}",
            "algorithmic_bytes_per_launch": nbytes, "launch_us": t * 1e6, "nnz": nnz, "n": n}


def run_spmv(args):
    """SpMV roofline on the 48^3 blocks matrix (12.1 M nonzeros, 146 MB of
    values and indices: larger than the 129 MB L2), set up without coarse
    space or GenEO (only A and the local inverses are built)."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import workloads as W
    import paper_2311_18783_gb300 as pkg
    w = W.cube48_blocks()
    s = pkg.Solver.from_workload(w, coarse=pkg.COARSE_NONE, geneo=0)
    r = time_spmv(s, reps=max(20, args.steps))
    line = {"metric": "SpMV achieved HBM bandwidth", "value": r["achieved"], "unit": "GB/s",
            "n_gpus": 1, "steps": max(20, args.steps), "warmup": 5, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cube48_blocks (matrix only)",
                       "l2": "inputs larger than L2 (A 146 MB)"},
            "roofline": r}
    print(json.dumps(line), flush=True)
    s.close()


def run_many(args):
    """The batching configuration: independent problems of
    workloads.many_problems (seed 3) in one context (geneo_setup_batch), float32
    split local factors, one segmented PCG per problem in the same launches
    (the iteration replayed as a CUDA graph), balanced form, autotuned SYMV.
    The 256 problems need 309 GB of float64 local inverses (sum n_i^2 =
    7.7e10), more than one GPU holds, so the largest prefix of the list whose
    float64 and float32 factors fit in --many-gb is set up (the count is in
    the line).  A step is one segmented solve of all of them to 1e-8."""
    import numpy as np
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    import workloads as W
    import paper_2311_18783_gb300 as pkg
    ps = W.many_problems(256, seed=3)
    for w in ps:
        w.f_slot = W.box(w.nx, w.ny, w.nz, h=w.hx, f='random', seed=w.nx).f_slot
    budget, used, take = args.many_gb * 1e9, 0.0, []
    for w in ps:
        t = pkg.Solver.topology(w, geneo=0)
        ni = np.diff(t.export("N_off")).astype(np.float64)
        t.close()
        need = float(((np.ceil(ni / 64) * 64) ** 2).sum()) / 2 * 12
        if used + need > budget:
            break
        used += need
        take.append(w)
    comp = pkg.compose(take)
    t0 = time.perf_counter()
    # the default LOBPCG mode misses GenEO vectors on the 2-3-cell boxes of
    # this workload (PCG then stalls); the Neumann mode finds the oracle's
    s = pkg.Solver.batch(take, precision=pkg.PREC_FP32, balanced=1, autotune=1,
                         lobpcg_neumann=1, lobpcg_block=16)
    setup_s = time.perf_counter() - t0
    b = torch.empty(s.n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(comp["f_slot"][0], b)
    x = torch.zeros_like(b)
    for _ in range(args.warmup):
        s.solve_segments(b, x, tol=TOL, maxit=1000)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.3)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.profile(True)
    s.profile_read()
    e0.record(stream)
    for _ in range(args.steps):
        st, infos = s.solve_segments(b, x, tol=TOL, maxit=1000)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = s.profile_read()
    s.profile(False)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    its = [i["iters"] for i in infos]
    stages = [float(v) for v in s.export("setup_stages")]
    line = {"metric": METRIC + ", all problems of the batch", "value": ms / 1e3, "unit": "s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "many_problems (seed 3)", "problems": len(take),
                       "of": len(ps), "n": s.n, "nsub": s.sizes["nsub"],
                       "n0": s.sizes["n0"], "n0_geneo": s.sizes["n0_geneo"],
                       "local_factor_gb": s.sizes["local_factor_bytes"] / 1e9,
                       "memory_budget_gb": args.many_gb, "tol": TOL, "setup_s": setup_s,
                       "setup_stages_s": stages,
                       "l2": "inputs larger than L2 (local factors "
                             f"{s.sizes['local_factor_bytes'] / 1e9:.0f} GB)"},
            "status": st, "problems_per_s": len(take) / (ms / 1e3),
            "pcg_iters": {"min": min(its), "median": float(np.median(its)), "max": max(its)},
            "clocks": clk, "gpu_launches": prof["launches"]}
    print(json.dumps(line), flush=True)
    s.close()


def coarse_single_launch(s):
    """Whether the autotuner kept the single-launch shape of the coarse
    solve (its row of the "autotune" export, target 2)."""
    rows = s.export("autotune").reshape(-1, 12)
    rows = rows[rows[:, 0] == 2]
    return bool(len(rows) and rows[-1][2] == 1)


def load_oracle_solution(workload, n):
    """The oracle's accurate solution of the benchmark workload, stored by
    tests/golden/make_cube32_solution.py (a file read, no oracle code run),
    or None."""
    if workload != WORKLOAD:
        return None
    path = os.path.join(ROOT, "tests", "golden", "cube32_solution.npy")
    if not os.path.exists(path):
        return None
    import numpy as np
    x = np.load(path)
    return x if x.shape == (n,) else None


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload in (BLOCK_WORKLOAD, "beam128_mild", "beam64_layered"):
        run_block(args)
        return
    if args.workload == WARM_WORKLOAD:
        run_warm(args)
        return
    if args.workload == "paper_beam":
        run_paper_beam(args)
        return
    if args.workload == "spmv_cube48":
        run_spmv(args)
        return
    if args.workload == "many_problems":
        run_many(args)
        return
    import torch
    import torch.distributed as dist
    import numpy as np
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import workloads as W
    import paper_2311_18783_gb300 as pkg
    w = getattr(W, args.workload)()
    prec = pkg.PREC_FP32 if args.precision == "mixed" else pkg.PREC_FP64
    t0 = time.perf_counter()
    s = pkg.Solver.from_workload(w, precision=prec, balanced=1, autotune=1)
    setup_s = time.perf_counter() - t0
    stage_names = ["assembly", "local_inverses", "split_factors", "geneo_eigensolves",
                   "geneo_filter", "coarse_factor", "autotune", "total"]
    stages = dict(zip(stage_names, [float(v) for v in s.export("setup_stages")]))
    tuned = []
    for row in s.export("autotune").reshape(-1, 12):
        ncand = pkg.Solver.symv_config_count(int(row[1])) if row[0] < 2 else 2
        tuned.append({"target": ["local factors", "S_j^-1 blocks",
                                 "coarse solve (0 per level and phase, 1 one launch)"][int(row[0])],
                      "precision": "f64" if int(row[1]) == pkg.PREC_FP64 else "f32",
                      "chosen": int(row[2]), "from_cache": bool(row[3]),
                      "ms_per_candidate": [float(v) for v in row[4:4 + ncand]]})
    n = s.n
    if prec == pkg.PREC_FP32:
        # mixed precision: C_j and S_j^-1 of the split local inverse in float32
        s.use_gradient_precision(pkg.PREC_FP32)
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    s.assemble_rhs(w.f_slot[0], b)
    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()
    xo = load_oracle_solution(args.workload, n)

    def err_vs_oracle(v):
        if xo is None:
            return None
        return float(np.linalg.norm(v.cpu().numpy() - xo) / np.linalg.norm(xo))

    def timed_variant(p, bal, steps, warmup, prof=False):
        """Mean device time of `steps` PCG solves to TOL with local factors p
        in the balanced (bal) or literal form, after `warmup` untimed ones."""
        s.use_precision(p)
        s.use_balanced(bal)
        for _ in range(warmup):
            s.solve(b, x, tol=TOL, maxit=1000)
        torch.cuda.synchronize()
        if prof:
            s.profile(True)
            s.profile_read()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its = []
        for _ in range(steps):
            info = s.solve(b, x, tol=TOL, maxit=1000)
            its.append(info["iters"])
        e1.record(stream)
        torch.cuda.synchronize()
        out = {"value": e0.elapsed_time(e1) / steps / 1e3, "unit": "s", "pcg_iters": its[-1],
               "err_vs_oracle_fp64": err_vs_oracle(x)}
        pr = None
        if prof:
            pr = s.profile_read()
            s.profile(False)
        return out, its, pr

    def timed_refined(p, nref=2):
        s.use_precision(p)
        s.use_balanced(True)
        xr = torch.zeros_like(b)
        s.solve_refined(b, xr, tol=TOL, maxit=1000, nref=nref)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = s.solve_refined(b, xr, tol=TOL, maxit=1000, nref=nref)
        e1.record(stream)
        torch.cuda.synchronize()
        return {"value": e0.elapsed_time(e1) / 1e3, "unit": "s", "nref": nref,
                "pcg_iters_total": info["iters"], "accurate_relres": info["relres"],
                "err_vs_oracle_fp64": err_vs_oracle(xr)}

    side = max(1, min(args.steps, 5))
    variants = {}
    coarse_other_ms = coarse_other_shape = coarse_steps = None
    fp64_side = None
    if prec == pkg.PREC_FP32:
        # plain float64 factors on the same GPU, same problem and form
        v64, _, p64 = timed_variant(pkg.PREC_FP64, True, side, max(1, min(args.warmup, 2)), True)
        l64 = p64["local_symv_ms"] / max(1, p64["local_symv_launches"]) * 1e-3
        v64["local_symv_tflops"] = p64["local_symv_flops"] / l64 / 1e12
        v64["local_symv_frac_of_fp64_peak"] = p64["local_symv_flops"] / l64 / 1e9 / FP64_PEAK_GFLOPS
        fp64_side = v64
        variants["fp64_literal"], _, _ = timed_variant(pkg.PREC_FP64, False, side, 1)
        variants["mixed_literal"], _, _ = timed_variant(pkg.PREC_FP32, False, side, 1)
        # the split's gradient part with S_j^-1 in float64 (the headline keeps
        # it in float32 as well)
        s.use_gradient_precision(pkg.PREC_FP64)
        variants["mixed_grad64_balanced"], _, _ = timed_variant(pkg.PREC_FP32, True, side, 1)
        s.use_gradient_precision(pkg.PREC_FP32)
        # the coarse solve in the shape the autotuner did not keep (one
        # cooperative launch, or one launch per level and phase; identical
        # results), with the per-step profile of the single launch
        kept = coarse_single_launch(s)
        s.use_persistent_coarse(not kept)
        other, _, pcl = timed_variant(pkg.PREC_FP32, True, side, 1, True)
        if not kept:
            cs = np.asarray(s.export("coarse_steps"), dtype=np.float64).reshape(-1, 5)
            coarse_steps = [[int(r[0]), int(r[1]), int(r[2]), round(r[3] / 1e6, 3),
                             round(r[4] / 2070.0, 2)] for r in cs]
        s.use_persistent_coarse(kept)
        variants["mixed_coarse_single_launch" if not kept else "mixed_coarse_per_level"] = other
        if pcl["coarse_symv_launches"]:
            coarse_other_ms = pcl["coarse_symv_ms"] / pcl["coarse_symv_launches"]
            coarse_other_shape = "one cooperative launch" if not kept else "per level and phase"
    # headline: balanced form with the precision asked for, clocks sampled
    s.use_precision(prec)
    s.use_balanced(True)
    for _ in range(args.warmup):
        s.solve(b, x, tol=TOL, maxit=1000)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    head, iters, prof = timed_variant(prec, True, args.steps, 0, True)
    torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(head["value"] * 1e3, world, "cuda")
    clk = clocks.stop()
    # end to end through the host-buffer entry point (copies inside)
    bh = b.cpu().pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    s.solve_host(bh, tol=TOL, maxit=1000, out=xh)
    torch.cuda.synchronize()
    te = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        s.solve_host(bh, tol=TOL, maxit=1000, out=xh)
        te.append(time.perf_counter() - t1)
    e2e_s = statistics.mean(te)
    # the sparse coarse solve (multifrontal tile GEMVs), timed by the
    # library's event pair around every solve in the headline's timed region
    coarse_roof = None
    if prof["coarse_symv_launches"] and prof["coarse_solve_bytes"]:
        tc = prof["coarse_symv_ms"] / prof["coarse_symv_launches"] * 1e-3
        cb = prof["coarse_solve_bytes"]
        single = coarse_single_launch(s)
        coarse_roof = {"kernel": ("k_mf_solve_persistent (one coarse solve, one cooperative "
                                  "launch)") if single else
                                 "k_mf_tiles<0..3> + k_mf_gather (one coarse solve)",
                       "bound": "hbm", "achieved": cb / tc / 1e9, "peak": peaks_hbm(),
                       "unit": "GB/s", "frac": cb / tc / 1e9 / peaks_hbm(),
                       "algorithmic_bytes_per_solve": cb, "solve_ms": tc * 1e3,
                       "solves": prof["coarse_symv_launches"],
                       "other_shape": coarse_other_shape, "other_shape_solve_ms": coarse_other_ms}
    if coarse_roof is not None:
        # per step of the last profiled single-launch coarse solve: kind (0
        # permutation in, 1 gather, 2..5 tile phase 0..3, 6 permutation out),
        # tree level, items, MB of factor tiles, microseconds (SM cycles of
        # the first CTA at 2070 MHz)
        if coarse_steps is None and coarse_roof["kernel"].startswith("k_mf_solve_persistent"):
            cs = np.asarray(s.export("coarse_steps"), dtype=np.float64).reshape(-1, 5)
            coarse_steps = [[int(r[0]), int(r[1]), int(r[2]), round(r[3] / 1e6, 3),
                             round(r[4] / 2070.0, 2)] for r in cs]
        coarse_roof["single_launch_steps"] = coarse_steps
    spmv_roof = time_spmv(s)
    spmv_roof["l2"] = ("A, x and y take about 45 MB; the value and index loads carry an "
                       "evict-first hint, so back-to-back launches re-read A; bench.py "
                       "--workload spmv_cube48 measures a 146 MB matrix")
    refined = {}
    if prec == pkg.PREC_FP32:
        refined["mixed"] = timed_refined(pkg.PREC_FP32)
    refined["fp64"] = timed_refined(pkg.PREC_FP64)
    s.use_precision(prec)
    # roofline of the dominant kernel: the local-factor SYMV
    peaks, peak_src = load_peaks()
    launches = max(1, prof["local_symv_launches"])
    t_launch = prof["local_symv_ms"] / launches * 1e-3
    if prec == pkg.PREC_FP64:
        achieved = prof["local_symv_flops"] / t_launch / 1e12
        peak = FP64_PEAK_GFLOPS / 1e3
        roof = {"kernel": "k_symv_strips<double> (local A_i^-1 apply)", "bound": "alu",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": "FP64 FMA rate derived from unit counts and the 2070 MHz clock",
                "traffic": None, "algorithmic_flops_per_launch": prof["local_symv_flops"],
                "launch_ms": t_launch * 1e3}
    else:
        achieved = prof["local_symv_bytes"] / t_launch / 1e9
        peak = peaks["hbm_gbs"]
        roof = {"kernel": "k_symv_strips<float> (local split factors)", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"hbm_gbs of {peak_src}",
                "traffic": (None if SYMV_F32_TRAFFIC_RATIO is None else
                            SYMV_F32_TRAFFIC_RATIO * prof["local_symv_bytes"]),
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum on "
                                  "cube16_hole_channels (autotuned configuration there), "
                                  "scaled by stored tiles",
                "algorithmic_bytes_per_launch": prof["local_symv_bytes"],
                "launch_ms": t_launch * 1e3}
    applies_per_s = aggregate_rate(sum(iters) + len(iters), ms * args.steps / 1e3, world)
    line = {"metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == pkg.PREC_FP64 else "f32+f64",
            "plain_fp64": fp64_side,
            "err_vs_oracle_fp64": head["err_vs_oracle_fp64"],
            "variants": variants, "refined": refined,
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "nsub": s.sizes["nsub"],
                       "n0": s.sizes["n0"], "n0_geneo": s.sizes["n0_geneo"], "tol": TOL,
                       "form": "balanced (x0 = Z E^-1 Z^T b, one coarse solve per iteration)",
                       "local_factors": ("float32 C_j and S_j^-1, float64 PCG and coarse solve"
                                         if prec == pkg.PREC_FP32 else "float64"),
                       "coarse_factor_gb": s.sizes["coarse_factor_bytes"] / 1e9,
                       "pcg_iters": iters[-1], "precision": args.precision,
                       "l2": "inputs larger than L2 (local factors "
                             f"{s.sizes['local_factor_bytes'] / 1e9:.1f} GB)",
                       "oracle_solution": None if xo is None else
                       "tests/golden/cube32_solution.npy (sparse LU + extended-precision "
                       "refinement, written by tests/golden/make_cube32_solution.py)",
                       "setup_s": setup_s, "setup_stages_s": stages,
                       "autotuned_symv": tuned},
            "applies_per_s": applies_per_s,
            "roofline": roof, "spmv_roofline": spmv_roof, "coarse_roofline": coarse_roof,
            "clocks": clk,
            "gpu_launches": prof["launches"],
            "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": n * 8,
                    "d2h_bytes_per_step": n * 8}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == WORKLOAD:
        o = OracleSample()
        o.step()
        per_iter, oinfo = statistics.median([o.step() for _ in range(2)]), o.info
        oit, src = oracle_iterations(iters[-1])
        line["cpu_baseline"] = {"value": per_iter * oit, "unit": "s", "cores": oinfo["cores"],
                                "cpu": oinfo["cpu"], "kind": "oracle",
                                "sample": oinfo["sample"] + f"; x {oit} iterations ({src})"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
