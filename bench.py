#!/usr/bin/env python
"""Benchmark of the space-angle sawtooth multigrid hot path on GB300.

One step = one sawtooth cycle (Fig. multi_grid_it) over every group of the
workload: fine PG residual, restriction to every level, upwind Jacobi on
every level with UpSamp, update, fine PG Jacobi, scalar flux and the FP64
residual norm.  Default workload: 256 x 256 nodes, 16 x 32 directions (512),
one group, seeded 8 x 8 checkerboard of sigma_t ~ logU[0.1, 10], scattering
ratio 0.9, source 1, vacuum, quadratic ConvFEM with PG, psi in FP32.

Metric: MG unknown-updates/s = (unknowns x cycles) / seconds, all ranks;
the timed cycles run as the library's captured CUDA graph (btmg_solve with
a fixed cycle count), the per-kernel shares come from an eager, event-timed
run of the same cycles.  Multi-GPU runs are independent replicas (one
problem per rank, no collective on the data path; the path does not need
one).

The second half of the metric, time to a 1e-6 relative residual (learned vs
plain multigrid), is reported under "time_to_1e-6" for the learned-
correction evaluation workload (512 x 512 nodes, 32 x 32 directions, the
checkerboard family at held-out seed 5000) and for a scattering-dominated
case (256 x 256, 16 x 32, domain side 30, c = 0.99): plain FP32 multigrid,
FP64-refined FP32 and BF16 inner cycles, and FP64-refined FP32 with the
learned correction every 4th cycle.

--impl reference times the FP64 CPU oracle (the slow reference program of
this repository) on the host cores, on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2301_09991_gb300 import inputs as I  # noqa: E402

METRIC = "MG unknown-updates/s"
UNIT = "unknown-updates/s"
WORKLOADS = {
    # name: (builder, description)
    "checker256": (lambda: I.checkerboard(n=256, n_polar=16, n_azim=32, blocks=8, seed=2, c=0.9),
                   "256x256 nodes, 16x32 dirs (512), 1 group, 8x8 checkerboard sigma_t~logU[0.1,10] "
                   "seed 2, c=0.9, q=1, vacuum, quadratic ConvFEM + anisotropic PG"),
    "checker64": (lambda: I.checkerboard(n=64, n_polar=8, n_azim=16, blocks=8, seed=2, c=0.9),
                  "64x64 nodes, 8x16 dirs (128), small case of the same family"),
}
# Algorithmic work per unknown of the fused PG operator:
PG_FLOPS_PER_UNKNOWN = 250.0  # separable evaluation of Eq. Petrov + Sec. 2.6 on interior nodes
SM_COUNT, FP32_LANES_PER_SM, SM_MAX_MHZ = 152, 128, 2070.0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": SM_MAX_MHZ}, "fallback"


def fp32_peak_tflops(sm_mhz):
    # FFMA: 128 lanes/SM x 2 flops x 152 SMs x clock
    return SM_COUNT * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def job_throughput(ms_local, units_per_rank, steps, ws, device="cpu"):
    """Whole-job (max-over-ranks ms, unknown-updates/s): every rank processes
    units_per_rank unknowns per step; the job takes as long as its slowest
    rank.  Replicas only: the one collective is this MAX of the elapsed time."""
    ms = float(ms_local)
    if ws > 1:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms, units_per_rank * steps * ws / (ms / 1000.0)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_from_profiles(kernel):
    """dram bytes per launch from the committed ncu summary of `kernel`, or
    None when the kernel source changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        for line in fh:
            m = re.match(r"\s*(\w+)\s+bytes_per_launch=(\S+)\s+src=(\S+):(\w+)", line)
            if not m or m.group(1) != kernel:
                continue
            src = os.path.join(ROOT, "paper_2301_09991_gb300", "csrc", m.group(3))
            if not os.path.exists(src):
                return None
            with open(src, "rb") as f:
                if hashlib.sha256(f.read()).hexdigest()[:len(m.group(4))] != m.group(4):
                    return None
            return float(m.group(2))
    return None


def cpu_baseline(workload, sample_cycles=1):
    """FP64 oracle: sample_cycles sawtooth cycles of the full workload on all
    host cores (OpenMP over direction planes)."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    prob = WORKLOADS[workload][0]()
    op = O.OracleProblem(prob)
    psi = op.zeros()
    N = int(np.prod(op.shape))
    t0 = time.perf_counter()
    for _ in range(sample_cycles):
        psi, _, _ = op.mg_cycle(psi)
    dt = time.perf_counter() - t0
    return {"value": N * sample_cycles / dt, "unit": UNIT, "cores": O.omp_threads(), "kind": "oracle",
            "sample": "%d FP64 oracle cycle(s) of the full %s workload (%d unknowns), %.1f s"
                      % (sample_cycles, workload, N, dt)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle as O
    # the full workload of the GPU line (about 2 s per FP64 cycle on 16 host
    # cores), so both arms time the same configuration
    prob = WORKLOADS[args.workload][0]()
    op = O.OracleProblem(prob)
    psi = op.zeros()
    N = int(np.prod(op.shape))
    for _ in range(args.warmup):
        psi, _, _ = op.mg_cycle(psi)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        psi, _, _ = op.mg_cycle(psi)
    dt = time.perf_counter() - t0
    value = N * args.steps / dt
    sample = ("%d FP64 oracle cycles of the full %s workload (%d unknowns per step), after %d warm-up cycles"
              % (args.steps, args.workload, N, args.warmup))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload][1],
                       "unknowns_per_gpu": N},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.omp_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def sweep_rooflines(btmg, torch, prob, pk, peak_src, cycles=10):
    """HBM roofline of the multigrid sweeps with the upwind fine scheme
    (pg = 0; the operator of the converged solves and of the refinement) on
    the same workload, FP32: the fine residual and Jacobi sweep (8 B per
    unknown: psi in, r or psi out) and the finest nu-sweep upwind Jacobi
    with the update (12 B per unknown: r1 and psi in, psi out), each
    event-timed per launch in eager cycles."""
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=0)
    psi = gp.zeros()
    for _ in range(3):
        gp.mg_cycle(psi, want_residual=False)
    gp.profile(True)
    for _ in range(cycles):
        gp.mg_cycle(psi, want_residual=False)
    torch.cuda.synchronize()
    prof = gp.profile_read()
    gp.profile(False)
    n = gp.num_unknowns() // gp.G
    peak = float(pk["hbm_gbs"])
    out = {"workload": "same as the metric, pg = 0 (upwind fine scheme), FP32", "peak": peak, "unit": "GB/s",
           "peak_source": "%s copy bandwidth" % peak_src}
    for cls, key, bpu, kernel in (("pg_residual", "k_upres_resid", 8, "fine residual (k_upres_tma)"),
                                  ("pg_jacobi", "k_upres_jacobi", 8, "fine Jacobi (k_upres_tma)"),
                                  ("upwind_fine", "k_upwind_fine", 12, "finest nu-sweep upwind Jacobi (k_upwind)")):
        ms, cnt = prof[cls]
        avg_s = ms / max(cnt, 1) / 1000.0
        ach = n * bpu / avg_s / 1e9
        out[cls] = {"kernel": kernel, "bytes_per_unknown": bpu, "ms": round(avg_s * 1e3, 4),
                    "achieved": ach, "frac": ach / peak, "traffic": traffic_from_profiles(key)}
    out["cycle_ms"] = round(sum(v[0] for v in prof.values()) / cycles, 4)
    del gp, psi
    # the scattering smoother on every level (scat_levels = 2): the finest
    # level's nu sweeps (J and the source in, J out: 12 B per unknown each),
    # and the final pass (J and psi in, psi out: 12 B), per cycle
    gp = btmg.Problem(prob, dtype=btmg.F32, pg=0, scat_levels=2)
    psi = gp.zeros()
    for _ in range(3):
        gp.mg_cycle(psi, want_residual=False)
    gp.profile(True)
    for _ in range(cycles):
        gp.mg_cycle(psi, want_residual=False)
    torch.cuda.synchronize()
    prof = gp.profile_read()
    gp.profile(False)
    nu = 3
    bpu = 12 * (nu + 1)
    fine_s = prof["upwind_fine"][0] / cycles / 1000.0
    ach = n * bpu / fine_s / 1e9
    out["scatter_fine"] = {"kernel": "finest-level scattering smoother (k_scat_sweep x 3, k_scat_corr x 3, "
                                     "k_scat_final)", "bytes_per_unknown_per_cycle": bpu,
                           "ms_per_cycle": round(fine_s * 1e3, 4), "achieved": ach, "frac": ach / peak,
                           "launches_per_cycle": prof["upwind_fine"][1] // cycles,
                           "coarse_ms_per_cycle": round(prof["upwind_coarse"][0] / cycles, 4),
                           "cycle_ms": round(sum(v[0] for v in prof.values()) / cycles, 4)}
    del gp, psi
    # cubic ConvFEM order (7 x 7 filters, halo 9), PG on: the fine PG
    # residual and Jacobi in three direct passes (k_pgd_grad, k_pgd_k,
    # k_pgd_apply), per launch of the operator
    prob3 = dict(prob, order=3)
    gp = btmg.Problem(prob3, dtype=btmg.F32, pg=1)
    psi = gp.zeros()
    for _ in range(3):
        gp.mg_cycle(psi, want_residual=False)
    gp.profile(True)
    for _ in range(cycles):
        gp.mg_cycle(psi, want_residual=False)
    torch.cuda.synchronize()
    prof = gp.profile_read()
    gp.profile(False)
    out["cubic_pg"] = {"kernel": "cubic PG operator (k_pgd_grad, k_pgd_k, k_pgd_apply)",
                       "resid_ms": round(prof["pg_residual"][0] / max(prof["pg_residual"][1], 1), 4),
                       "jacobi_ms": round(prof["pg_jacobi"][0] / max(prof["pg_jacobi"][1], 1), 4),
                       "cycle_ms": round(sum(v[0] for v in prof.values()) / cycles, 4)}
    del gp, psi
    return out


def time_to_residual(btmg, torch, rtol=1e-6):
    """Seconds (wall, synchronised) and cycles to a relative residual of rtol
    for plain FP32 multigrid, FP64-refined FP32 / BF16 inner cycles (32
    cycles per FP64 outer step: the FP64 residual is the costly part of a
    step on this GPU, whose FP64 rate is a small fraction of its FP32 rate) and
    FP64-refined FP32 with the learned correction (upwind fine operator,
    pg = 0, for which the FP64 refinement is defined), and FP64-refined FP32 /
    BF16 with the scattering smoother on every level (scat_levels = 2, arbitrated
    by plain multigrid: an outer residual above 1.5 times the best drops it
    for the rest of the solve)."""
    from paper_2301_09991_gb300 import learned as LN
    net = LN.load_net(os.path.join(ROOT, "paper_2301_09991_gb300", "weights", "unet_thick.npy"))
    cases = {
        "checker512_32x32_seed5000": (I.checkerboard(n=512, n_polar=32, n_azim=32, blocks=8, seed=5000, c=0.9),
                                      "512x512 nodes, 32x32 dirs, unit square, c=0.9 (held-out seed)"),
        "thick256_16x32_L30_c0.99": (LN.training_problem(5010, n=256, n_polar=16, n_azim=32, c=0.99, length=30.0),
                                     "256x256 nodes, 16x32 dirs, side 30, c=0.99 (held-out seed)"),
        # the same regime at full size, refined FP32 with and without the smoother only
        "thick512_32x32_L30_c0.99": (LN.training_problem(5011, n=512, n_polar=32, n_azim=32, c=0.99, length=30.0),
                                     "512x512 nodes, 32x32 dirs, side 30, c=0.99 (held-out seed)",
                                     ("refined_f32", "refined_f32_scatter")),
    }
    out = {}
    for name, case in cases.items():
        prob, desc = case[0], case[1]
        only = case[2] if len(case) > 2 else None
        row = {"description": desc}

        def timed(fn):
            fn()  # warm-up: workspaces, graphs, twin problem
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = fn()
            torch.cuda.synchronize()
            return r, time.perf_counter() - t0

        if only is None or "plain_f32" in only:
            gp = btmg.Problem(prob, dtype=btmg.F32, pg=0)
            psi = gp.zeros()

            def plain():
                psi.zero_()
                return gp.solve(psi, rtol=rtol, max_cycles=600, check_every=10, history=False)
            r, sec = timed(plain)
            row["plain_f32"] = {"seconds": round(sec, 4), "cycles": r["cycles"], "rel_resid": r["rel_resid"],
                                "reached": bool(r["rel_resid"] <= rtol)}
            del gp, psi
        for key, dt, nt, scat, inner in (("refined_f32", btmg.F32, None, 0, 32),
                                         ("refined_bf16", btmg.BF16, None, 0, 32),
                                         ("refined_f32_learned", btmg.F32, net, 0, 32),
                                         ("refined_f32_scatter", btmg.F32, None, 2, 32),
                                         ("refined_bf16_scatter", btmg.BF16, None, 2, 32)):
            if only is not None and key not in only:
                continue
            gp = btmg.Problem(prob, dtype=dt, pg=0, scat_levels=scat)
            if nt is not None:
                gp.set_learned(nt, every=4)
            psi64 = torch.zeros(gp.shape, dtype=torch.float64, device="cuda")

            def refined():
                psi64.zero_()
                return gp.solve_refined(psi64, rtol=rtol, max_outer=300, inner_cycles=inner)
            r, sec = timed(refined)
            row[key] = {"seconds": round(sec, 4), "cycles": r["cycles"], "rel_resid": r["rel_resid"],
                        "reached": bool(r["rel_resid"] <= rtol)}
            if nt is not None:
                st = gp.learn_stats()
                row[key].update({"learned_steps": st[0], "fallbacks": st[3]})
            if scat:
                row[key]["fallbacks"] = gp.scatter_fallbacks()
            del gp, psi64
        out[name] = row
    return out


def multigroup(btmg, torch, cycles=3, rtol=1e-6):
    """The 4-group downscatter workload at full size (512^2 nodes, 32 x 32
    directions, 1.07 G unknowns): psi in BF16 with FP32 accumulation and the
    upwind fine scheme.  Throughput of `cycles` graph cycles (one btmg_solve
    call, groups in order, block Gauss-Seidel over groups), and the wall time
    of the FP64-refined solve to rtol (32 inner cycles per outer step)."""
    prob = I.multigroup(n=512, n_polar=32, n_azim=32, G=4, seed=3)
    gp = btmg.Problem(prob, dtype=btmg.BF16, pg=0)
    psi = gp.zeros()
    gp.solve(psi, rtol=0.0, max_cycles=2, check_every=2, history=False)  # warm-up, graph capture
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gp.solve(psi, rtol=0.0, max_cycles=cycles, check_every=cycles, history=False)
    torch.cuda.synchronize()
    t_cyc = time.perf_counter() - t0
    del psi
    psi64 = torch.zeros(gp.shape, dtype=torch.float64, device="cuda")
    gp.solve_refined(psi64, rtol=1e-2, max_outer=2, inner_cycles=4)  # warm-up: twin problem, workspaces
    psi64.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = gp.solve_refined(psi64, rtol=rtol, max_outer=100, inner_cycles=32)
    torch.cuda.synchronize()
    t_sol = time.perf_counter() - t0
    n = gp.num_unknowns()
    del gp, psi64
    torch.cuda.empty_cache()
    pg_on = multigroup_pg(btmg, torch, prob, cycles)
    return {"workload": "512x512 nodes, 32x32 dirs, 4 downscatter groups (seed 3), BF16 storage, FP32 compute, "
                        "upwind fine scheme", "unknowns": n, "pg_on": pg_on,
            "cycle_value": n * cycles / t_cyc, "unit": UNIT, "cycle_ms": 1000 * t_cyc / cycles,
            "refined_to": rtol, "refined_seconds": round(t_sol, 4), "refined_inner_cycles": r["cycles"],
            "refined_rel_resid": r["rel_resid"], "reached": bool(r["rel_resid"] <= rtol)}


def multigroup_pg(btmg, torch, prob, cycles):
    """The same 4-group workload on the full hot path (PG on the finest level,
    psi in BF16, FP32 accumulation): throughput of `cycles` graph cycles,
    per-kernel shares of one eager cycle, and the algorithmic HBM bytes of
    the cycle against its time.  Bytes per fine unknown and group: PG
    residual psi in + r out; restriction r in; finest upwind sweeps r and
    psi in, psi out; PG Jacobi psi in and out; the coarse corrections add
    about one sixteenth of the restriction's and the sweep's words."""
    gp = btmg.Problem(prob, dtype=btmg.BF16, pg=1)
    psi = gp.zeros()
    gp.solve(psi, rtol=0.0, max_cycles=2, check_every=2, history=False)  # warm-up, graph capture
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gp.solve(psi, rtol=0.0, max_cycles=cycles, check_every=cycles, history=False)
    torch.cuda.synchronize()
    t_cyc = (time.perf_counter() - t0) / cycles
    gp.profile(True)
    gp.mg_cycle(psi, want_residual=False)
    torch.cuda.synchronize()
    prof = gp.profile_read()
    gp.profile(False)
    n = gp.num_unknowns()
    s, c = psi.element_size(), 4  # storage and compute bytes
    bpu = (s + c) + c + (c + s + s) + (s + s) + (c + c) / 16.0
    pk, _ = peaks()
    gbs = n * bpu / t_cyc / 1e9
    tot = sum(v[0] for v in prof.values())
    del gp, psi
    torch.cuda.empty_cache()
    return {"workload": "the same, PG on, BF16 psi", "cycle_value": n / t_cyc, "unit": UNIT,
            "cycle_ms": round(1000 * t_cyc, 3), "bytes_per_unknown": bpu, "achieved_gbs": gbs,
            "hbm_frac": gbs / float(pk["hbm_gbs"]),
            "kernel_share": {k: round(v[0] / tot, 4) for k, v in prof.items()}}


def batched(btmg, torch, cycles=4, probs=None, label=None):
    """Batched workload: 64 independent one-group Voronoi problems (seed 4),
    N uniform over the multiples of 16 in [64, 512], direction grids uniform
    over {8x16, 16x16, 16x32, 32x32}, PG on, FP32.  Throughput of `cycles`
    cycles of btmg_solve_batch (autotuned chunks, the coarse corrections of
    all problems in one persistent launch with an autotuned tile width and
    grid; one eager cycle, graph cycles, final residuals) against the same
    cycles run problem by problem (btmg_solve, graph path)."""
    probs = I.batch() if probs is None else probs
    N = sum(p["nx"] * p["ny"] * p["n_polar"] * p["n_azim"] for p in probs)
    t0 = time.perf_counter()
    b = btmg.Batch(probs, dtype=btmg.F32, pg=1, autotune=True)
    torch.cuda.synchronize()
    t_tune = time.perf_counter() - t0
    psis = b.zeros()
    b.solve(psis, rtol=0.0, max_cycles=2, check_every=1)  # warm-up, graph capture
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.solve(psis, rtol=0.0, max_cycles=cycles, check_every=cycles)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    chunks = [b.chunks(i) for i in range(len(probs))]
    persistent, tile, ctas, coarse_ms = b.coarse()
    b.close()
    del psis, b
    torch.cuda.empty_cache()
    gps = [btmg.Problem(p, dtype=btmg.F32, pg=1) for p in probs]
    xs = [g.zeros() for g in gps]
    for g, x in zip(gps, xs):
        g.solve(x, rtol=0.0, max_cycles=3, check_every=3, history=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g, x in zip(gps, xs):
        g.solve(x, rtol=0.0, max_cycles=cycles, check_every=cycles, history=False)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    del gps, xs
    torch.cuda.empty_cache()
    return {"workload": label or ("64 Voronoi problems, N in 64..512 (step 16), dirs in {8x16,16x16,16x32,32x32}, "
                                  "seed 4, PG on, FP32"),
            "problems": len(probs), "persistent_coarse": {"used": persistent, "tile": tile, "ctas_per_sm": ctas,
                                                          "ms_per_launch": round(coarse_ms, 4)},
            "unknowns": N, "cycles": cycles, "value": N * cycles / t_batch, "unit": UNIT,
            "seconds": round(t_batch, 4), "sequential_value": N * cycles / t_seq,
            "sequential_seconds": round(t_seq, 4), "autotune_seconds": round(t_tune, 2),
            "chunks_tuned_vs_auto": sum(1 for c in chunks if c[0] != c[1])}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="btmg", choices=["btmg", "reference"])
    ap.add_argument("--workload", default="checker256", choices=sorted(WORKLOADS))
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64", "bf16", "f16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-cycles", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-ttr", action="store_true", help="skip the time-to-1e-6 section")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-workload section")
    ap.add_argument("--no-sweeps", action="store_true", help="skip the upwind-scheme sweep rooflines")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2301_09991_gb300 import btmg
    import __graft_entry__

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    __graft_entry__.build()

    code = {"f32": btmg.F32, "f64": btmg.F64, "bf16": btmg.BF16, "f16": btmg.F16}[args.dtype]
    prob = WORKLOADS[args.workload][0]()
    gp = btmg.Problem(prob, dtype=code, pg=1)
    N = gp.num_unknowns()
    psi = gp.zeros()
    stream = torch.cuda.current_stream()
    # warm-up: its first cycle runs eagerly, the second captures the cycle
    # graph for this psi and stream, which the timed call then replays
    gp.solve(psi, rtol=0.0, max_cycles=args.warmup, check_every=args.warmup, history=False)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    out = gp.solve(psi, rtol=0.0, max_cycles=args.steps, check_every=args.steps, history=False)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    assert out["cycles"] == args.steps, out
    ms, value = job_throughput(ms, N, args.steps, ws, "cuda")

    # per-kernel device times: the same cycles eagerly, each launch bracketed
    # by CUDA events on the launching stream
    n_prof = min(args.steps, 10)
    gp.profile(True)
    n0 = gp.launch_count()
    for _ in range(n_prof):
        gp.mg_cycle(psi, want_residual=False)
    torch.cuda.synchronize()
    prof = gp.profile_read()
    gp.profile(False)
    per_cycle = (gp.launch_count() - n0) / n_prof
    # the timed solve: the cycles' kernels plus one final residual evaluation
    # (phi partials, source, norm sums and the residual kernel)
    launches = int(round(per_cycle * args.steps)) + 4 * gp.G + gp.G

    # end to end through the C-ABI call with host buffers
    # (btmg_mg_cycle_host): every step copies psi in from pinned memory,
    # runs one cycle, and copies psi back (overlapping the cycle's last
    # kernel) with the FP64 residual norms and the error word
    hpsi = torch.zeros(gp.shape, dtype=gp.torch_dtype).pin_memory()
    hpsi.copy_(psi.cpu())
    gp.mg_cycle_host(hpsi, want_residual=True)  # first call: the device buffer and side streams
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        gp.mg_cycle_host(hpsi, want_residual=True)  # returns once hpsi holds the result
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    nbytes = psi.numel() * psi.element_size()
    e2e = {"value": N * args.e2e_steps * ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nbytes,
           "d2h_bytes_per_step": nbytes + 16 * gp.G + 4}

    # roofline of the dominant kernel class (most device time in the timed region)
    pk, src = peaks()
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    avg_s = dom_ms / max(dom_n, 1) / 1000.0
    per_launch_unknowns = N // gp.G
    if dom in ("pg_residual", "pg_jacobi"):
        sm_mhz = float(pk.get("sm_max_mhz", SM_MAX_MHZ))
        achieved = PG_FLOPS_PER_UNKNOWN * per_launch_unknowns / avg_s / 1e12
        peak = fp32_peak_tflops(sm_mhz)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": traffic_from_profiles("k_pg_resid" if dom == "pg_residual" else "k_pg_jacobi"),
                "kernel": "k_pg (%s)" % dom,
                "peak_source": "FP32 FFMA: 152 SMs x 128 lanes x 2 flops x %.0f MHz" % sm_mhz,
                # the derivation checked by measurement: independent fmaf chains on every SM
                "fma_rate_measured": btmg.fp32_fma_rate(5)}
    else:
        # upwind fine: reads src + psi (+ coarse delta), writes psi
        esz = psi.element_size()
        byts = per_launch_unknowns * (4 + 2 * esz)
        achieved = byts / avg_s / 1e9
        peak = float(pk["hbm_gbs"])
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic_from_profiles("k_upwind_fine"), "kernel": "k_upwind (%s)" % dom,
                "peak_source": "%s copy bandwidth" % src}
    roof["kernel_ms"] = {k: round(v[0] / max(v[1], 1), 4) for k, v in prof.items()}
    roof["kernel_share"] = {k: round(v[0] / sum(x[0] for x in prof.values()), 4) for k, v in prof.items()}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload][1],
                       "unknowns_per_gpu": N, "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "inputs larger than L2 (psi, psi_tmp and r_1 are %d MB each)"
                             % (nbytes // 2 ** 20)},
            "roofline": roof, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk}
    if rank == 0 and not args.no_sweeps:
        line["sweeps"] = sweep_rooflines(btmg, torch, prob, pk, src)
    if rank == 0 and not args.no_ttr:
        line["time_to_1e-6"] = time_to_residual(btmg, torch)
    if rank == 0 and not args.no_batch:
        del psi, gp, hpsi
        torch.cuda.empty_cache()
        line["batched"] = batched(btmg, torch)
        # many small problems: the coarse levels are latency-bound
        small = I.batch(count=256, seed=44, n_lo=32, n_hi=128, step=16, grids=((4, 8), (8, 8), (8, 16)))
        line["batched_small"] = batched(btmg, torch, cycles=8, probs=small,
                                        label="256 Voronoi problems, N in 32..128 (step 16), dirs in {4x8,8x8,8x16}, "
                                              "seed 44, PG on, FP32")
        line["multigroup"] = multigroup(btmg, torch)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_cycles)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
