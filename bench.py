"""Benchmark: unknowns solved per second to relative residual 1e-10 with the GB300 HOMG solver.

Workload: 2-D Poisson, 5-point stencil, 4097^2 nodes (h = 1/4096), 12 levels, FP64, f iid
uniform[-1, 1] over the interior from numpy default_rng(0), u0 = 0, MFMG cycles with MaxI = 32,
restarted until ||f - A u|| / ||f|| <= 1e-10. One step = one complete solve (zeroing u, then
``homg_solve``). The working set (about 0.8 GB) exceeds the 126 MB L2, so no flush is needed.

Prints one JSON line (rank 0). ``--impl reference`` times the CPU oracle instead (the reference arm
of this benchmark, since the paper publishes no code).
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

METRIC = "unknowns solved/sec to 1e-10 rel residual"
UNIT = "unknowns/s"
N_SIDE = 4096
LEVELS = 12
TOL = 1e-10
MAX_I = 32
MAX_CYCLES = 60
WORKLOAD = ("2-D Poisson -Lap u = f, 5-point, 4097x4097 nodes, 12 levels, FP64, f iid uniform[-1,1] "
            "(default_rng(0)), u0 = 0, HOMG MFMG MaxI=32, to relative residual 1e-10")

# Peaks for the roofline (denominators).
FALLBACK_HBM_GBS = 6800.0
# Nominal FP64 issue rate, for context only: 1.25 TFLOP/s (FMA = 2 flops) = 0.625e12 FP64
# instructions/s. The denominator of the FP64 ALU fraction is measured live (measure_fp64_peak).
FP64_NOMINAL_OPS = 0.625e12


FALLBACK_BF16_TFLOPS = 1900.0
LEVEL0_FP64_DRAM_BYTES = 384.30e6  # k_jacobi2d2<0, 0> on 4097^2, one launch at 16 rows per thread
# k_jacobi2_x2<float> (two fused sweeps) on 4097^2, one captured launch: 134.8 MB read + 38.2 MB written
LEVEL0_FP32_DRAM_BYTES = 173.01e6


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, device=None):
    """Largest value of x over all ranks (x itself in a single process)."""
    import torch

    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, elapsed_s, device=None):
    """Whole-job throughput of independent replicas: every rank's units over the slowest rank's time.

    Replicas only (the solve does not shard across GPUs): the sole collectives are this max and a
    barrier; no data crosses ranks."""
    import torch

    world = torch.distributed.get_world_size() if torch.distributed.is_initialized() else 1
    return units_per_rank * world / max_over_ranks(elapsed_s, device)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def oracle_cpu_baseline(f_np, full=True):
    """The oracle as it stands, single-threaded on one host core: the complete benchmark solve
    (u0 = 0 to relres 1e-10) on the 4097^2 grid, timed in full; or (full=False) one cycle of it,
    scaled by the oracle's own cycle count at 1025^2."""
    import oracle

    oracle.build()
    t0 = time.perf_counter()
    if full:
        _, status, cycles, hist = oracle.solve(f_np, LEVELS, tol=TOL, max_cycles=MAX_CYCLES, max_i=MAX_I)
        dt = time.perf_counter() - t0
        if status != oracle.OK:
            raise RuntimeError("oracle solve did not converge (status %d)" % status)
        return {"value": (N_SIDE - 1) ** 2 / dt, "unit": UNIT, "cores": 1, "host_cores": host_cores(), "kind": "oracle",
                "sample": "the full oracle solve of the 4097^2 workload, u0 = 0 to relres 1e-10 "
                          "(%d cycles, final relres %.2e, %.1f s, one thread)" % (cycles, hist[-1], dt),
                "ms_per_solve": 1e3 * dt, "cycles": cycles}
    oracle.solve(f_np, LEVELS, tol=0.0, max_cycles=1, max_i=MAX_I)
    dt = time.perf_counter() - t0
    _, _, cycles, _ = oracle.solve(inputs_uniform(1024), 10, tol=TOL, max_cycles=MAX_CYCLES, max_i=MAX_I)
    return {"value": (N_SIDE - 1) ** 2 / (dt * cycles), "unit": UNIT, "cores": 1, "host_cores": host_cores(),
            "kind": "oracle",
            "sample": "one oracle cycle on the 4097^2 grid (%.1f s), scaled by the %d cycles the oracle needs at "
                      "1025^2" % (dt, cycles)}


def inputs_uniform(n):
    from paper_1108_2045_gb300 import inputs

    return inputs.uniform_rhs(n, 2, seed=0)


def measure_fp64_peak(homg, stream, dev, clocks_index):
    """The FP64 instruction issue rate of this GPU, measured now: the library's probe kernel (8
    independent chains of dependent FP64 fused multiply-adds, or additions, per thread; 8 blocks of
    256 threads per SM) launched 20 times back to back after 3 warm-up launches, each launch timed
    with CUDA events on the stream. Returns the mean and best rates per op and the SM clock seen."""
    import torch

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = 8 * sms
    sink = torch.empty(blocks * homg.HOMG_PROBE_THREADS, dtype=torch.float64, device=dev)
    out = {"kernel": "homg_fp64_issue_probe (k_fp64_issue)", "blocks": blocks,
           "threads_per_block": homg.HOMG_PROBE_THREADS}
    iters = 2048
    with ClockSampler(clocks_index) as clk:
        for op, name in ((0, "fma"), (1, "add")):
            for _ in range(3):
                instr = homg.homg_fp64_issue_probe(op, blocks, iters, sink, stream)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(21)]
            ev[0].record(stream)
            for i in range(20):
                homg.homg_fp64_issue_probe(op, blocks, iters, sink, stream)
                ev[i + 1].record(stream)
            torch.cuda.synchronize(dev)
            ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(20)]
            out[name] = {"instructions_per_launch": instr, "launch_ms_mean": sum(ms) / len(ms),
                         "mean_tinstr_per_s": instr / (sum(ms) / len(ms) * 1e-3) / 1e12,
                         "best_tinstr_per_s": instr / (min(ms) * 1e-3) / 1e12}
    out["clocks"] = clk.summary()
    out["peak_tinstr_per_s"] = max(out["fma"]["mean_tinstr_per_s"], out["add"]["mean_tinstr_per_s"])
    return out


def run_cfg2_sine(args, homg, inputs, stream, barrier, pending):
    """The manufactured right-hand side of the 4097^2 workload, f = 2 pi^2 sin(pi x) sin(pi y), whose
    discrete solution is c_h sin(pi x) sin(pi y) with c_h = pi^2 h^2 / (4 sin^2(pi h / 2)). The FP64
    rounding of that exact solution alone leaves a relative residual (the floor, measured here with the
    library's residual of the rounded closed form, and by the oracle in the CPU leg) above 1e-10 at
    this size, so HOMG and the classic V(2,2) cycle solve to tol = max(1e-10, 4 x floor), FP64 cycles.
    Reports cycles, time, the attained relres and the error against the closed form."""
    import numpy as np
    import torch

    n, L = N_SIDE, LEVELS
    h = 1.0 / n
    ch = np.pi ** 2 * h ** 2 / (4 * np.sin(np.pi * h / 2) ** 2)
    f_np = inputs.sine_rhs(n, 2)
    exact_np = ch * inputs.sine_solution(n, 2)
    f = torch.from_numpy(f_np).cuda()
    exact = torch.from_numpy(exact_np).cuda()
    u = torch.zeros_like(f)
    with homg.Solver(2, n + 1, L) as s:
        s.set_stream(stream)
        floor = s.residual_norm(f, exact)
    tol = max(TOL, 4.0 * floor)
    out = {"workload": "2-D Poisson, 4097^2 nodes, 12 levels, f = 2 pi^2 sin(pi x) sin(pi y), u0 = 0, FP64 cycles",
           "floor_relres": floor, "tol": tol}
    for name, kw in (("homg", dict(max_i=MAX_I)), ("v22", dict(cycle="v"))):
        with homg.Solver(2, n + 1, L, **kw) as s:
            s.set_stream(stream)
            u.zero_()
            s.solve(f, u, tol=tol, max_cycles=MAX_CYCLES)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.cfg2_sine_steps):
                u.zero_()
                st, cyc, rr = s.solve(f, u, tol=tol, max_cycles=MAX_CYCLES)
            e1.record(stream)
            barrier()
            ms = e0.elapsed_time(e1) / args.cfg2_sine_steps
        r = {"status": st, "cycles": cyc, "relres": rr, "ms_per_solve": ms, "unknowns_per_s": (n - 1) ** 2 / (ms * 1e-3),
             "rel_err_vs_discrete_exact": float(torch.linalg.vector_norm(u - exact) / torch.linalg.vector_norm(exact))}
        if name == "homg":
            pending.append((r, "poisson", None, f_np, u.cpu().numpy()))
        out[name] = r
    out["homg_ms_over_v22_ms"] = out["homg"]["ms_per_solve"] / out["v22"]["ms_per_solve"]
    pending.append((out, "floor", None, f_np, exact_np))
    del f, u, exact
    torch.cuda.empty_cache()
    return out


CFG3_SIDE = 512


def run_cfg3(args, homg, inputs, stream, barrier, pending):
    """3-D Poisson, 7-point stencil, 513^3 nodes, 9 levels: FP64 cycles against FP32 and bfloat16
    cycles (FP64 residual, update and norms; iterative refinement) to relative residual 1e-10, for
    f = 3 pi^2 sin sin sin and for f iid N(0, 1) (seed 0). Reports time to 1e-10, cycles, the error
    against the FP64 solution and, for the sine case, against the closed-form discrete solution
    c_h prod sin(pi x_k), c_h = pi^2 h^2 / (4 sin^2(pi h / 2))."""
    import numpy as np
    import torch

    n = args.cfg3_side
    levels = n.bit_length() - 1
    out = {"workload": "3-D Poisson -Lap u = f, 7-point, %d^3 nodes, %d levels, MaxI=32, to relres 1e-10" % (n + 1, levels)}
    h = 1.0 / n
    ch = np.pi ** 2 * h ** 2 / (4 * np.sin(np.pi * h / 2) ** 2)
    for rhs in ("sine", "normal"):
        f_np = inputs.sine_rhs(n, 3) if rhs == "sine" else inputs.normal_rhs(n, 3, seed=0)
        f = torch.from_numpy(f_np).cuda()
        del f_np
        u = torch.zeros_like(f)
        ref = None
        res = {}
        for prec in ("fp64", "fp32", "bf16"):
            with homg.Solver(3, n + 1, levels, max_i=MAX_I, precision=prec, launch_mode=args.launch) as s3:
                s3.set_stream(stream)
                u.zero_()
                s3.solve(f, u, tol=TOL, max_cycles=MAX_CYCLES)
                barrier()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.cfg3_steps):
                    u.zero_()
                    st, cyc, rr = s3.solve(f, u, tol=TOL, max_cycles=MAX_CYCLES)
                e1.record(stream)
                barrier()
                ms = e0.elapsed_time(e1) / args.cfg3_steps
                stats = s3.stats()
            r = {"status": st, "cycles": cyc, "relres": rr, "ms_per_solve": ms,
                 "unknowns_per_s": (n - 1) ** 3 / (ms * 1e-3),
                 "fine_launch_us": 1e3 * stats["fine_ms"] / max(1, stats["cycles"] * stats["fine_launches_per_cycle"])}
            if prec == "fp64":
                ref = u.clone()
            else:
                r["rel_diff_vs_fp64"] = float(torch.linalg.vector_norm(u - ref) / torch.linalg.vector_norm(ref))
                r["speedup_vs_fp64"] = res["fp64"]["ms_per_solve"] / ms
            if rhs == "sine":
                x = torch.arange(n + 1, dtype=torch.float64, device=u.device) / n
                sx = torch.sin(np.pi * x)
                exact = ch * sx[:, None, None] * sx[None, :, None] * sx[None, None, :]
                r["rel_err_vs_discrete_exact"] = float(torch.linalg.vector_norm(u - exact) / torch.linalg.vector_norm(exact))
                del exact
            if rhs == "normal" and prec == "fp32" and args.cfg3_oracle_check:
                # checked later, by the oracle's own FP64 residual (CPU leg)
                pending.append((r, "poisson", None, f.cpu().numpy(), u.cpu().numpy()))
            res[prec] = r
        out[rhs] = res
        del f, u, ref
        torch.cuda.empty_cache()
    return out


def run_cfg4(args, homg, stream, barrier, pending):
    """1024 independent 2-D Poisson problems of uneven sizes in one batched solve to relres 1e-10
    each: FP32 cycles with FP64 refinement (FP64 cycles beside it). Per-problem solve times are
    device-clock times from a problem's initial residual test to its convergence. Sampled problems
    (two per size) are checked with the oracle's own FP64 residual; the oracle's time for the whole
    batch is extrapolated from one timed oracle solve per size (both in the CPU leg)."""
    import numpy as np
    import torch

    from paper_1108_2045_gb300 import inputs

    ks, fs_np = inputs.uneven_batch(1024, seed=1)
    ks_arr = np.array(ks)
    fs = [torch.from_numpy(f).cuda() for f in fs_np]
    us = [torch.zeros_like(f) for f in fs]
    sides = [2 ** k + 1 for k in ks]
    unknowns = float(sum((s - 2) ** 2 for s in sides))
    sample = [i for k in range(6, 11) for i in np.flatnonzero(ks_arr == k)[:2]]
    out = {"workload": "1024 2-D Poisson problems, 5-point, sides 2^k+1 with k ~ U{6..10} (seed 1), f iid N(0,1), "
                       "each to relres 1e-10, one batched solve",
           "problems_per_k": {str(k): int((ks_arr == k).sum()) for k in range(6, 11)}, "unknowns": unknowns}
    # FP32 and FP64 cycles with the per-group graphs; FP32 cycles in one persistent launch
    for name, prec, mode in (("fp32", "fp32", "graph"), ("fp64", "fp64", "graph"), ("fp32_persistent", "fp32", "persistent")):
        with homg.BatchSolver(sides, precision=prec, launch_mode=mode) as b:
            b.set_stream(stream)
            for u in us:
                u.zero_()
            b.solve(fs, us, tol=TOL, max_cycles=MAX_CYCLES)
            runs = []
            for _ in range(args.cfg4_steps):
                for u in us:
                    u.zero_()
                barrier()
                rc, status, cycles, relres, ms = b.solve(fs, us, tol=TOL, max_cycles=MAX_CYCLES)
                runs.append((b.stats()["solve_ms"], ms, status, cycles, relres))
            st = b.stats()
        batch_ms = min(r[0] for r in runs)
        per = np.array(runs[-1][1])
        r = {"batch_ms": batch_ms, "value": unknowns / (batch_ms * 1e-3), "unit": UNIT, "launch": mode,
             "all_converged": all(x == 0 for x in runs[-1][2]), "max_relres": max(runs[-1][4]),
             "cycles_min_max": [min(runs[-1][3]), max(runs[-1][3])],
             "solve_ms_p50": float(np.percentile(per, 50)), "solve_ms_p99": float(np.percentile(per, 99)),
             "tuned_rows_level0": dict(zip([str(x) for x in st["sides"]], st["rows"])),
             "tuned_sweep_us_level0": dict(zip([str(x) for x in st["sides"]], st["tuned_us"]))}
        if prec == "fp32" and args.cfg4_oracle_check:
            r["oracle_sample"] = "two problems per k (the first of each size in batch order)"
            for i in sample:  # checked later by the oracle's own FP64 residual (CPU leg)
                pending.append((r, "poisson_max", None, fs_np[i], us[i].cpu().numpy()))
        out[name] = r
    out["persistent_over_graph_ms"] = out["fp32_persistent"]["batch_ms"] / out["fp32"]["batch_ms"]
    del fs, us
    torch.cuda.empty_cache()
    if args.cfg4_oracle_time:
        # problems timed per size (the first ones of each size in batch order), bounded CPU time
        nsample = {6: 8, 7: 8, 8: 4, 9: 2, 10: 1}
        per_k = {k: ([fs_np[int(i)] for i in np.flatnonzero(ks_arr == k)[:nsample[k]]], int((ks_arr == k).sum()))
                 for k in range(6, 11)}
        pending.append((out, "batch_time", None, per_k, unknowns))
    return out


CFG5_SIDE = 2048
CFG5_LEVELS = 11


def run_cfg5(args, homg, stream, barrier, pending):
    """Variable-coefficient diffusion -div(k grad u) = f on 2049^2 nodes, 11 levels, k = exp(g) with g
    a Gaussian random field (sigma 1, squared-exponential correlation length 0.05, seed 2), f iid
    N(0, 1) (seed 0), to relres 1e-10: plain HOMG (FP64 and FP32 cycles) against the learned
    corrector ahead of every cycle. Two networks are trained here, from scratch, on the same 20,000
    64 x 64 patches of error/residual pairs the solver produces on four other right-hand sides (seeds
    100-103; iterates after 2, 3 and 4 cycles): one on the mean squared error against the scaled true
    error, one on the residual its proposal leaves. The learned solves run with the judge on the
    proposal's own residual and, for the error-trained network, with the judge after the following
    cycle. Training time is reported, not timed as a solve."""
    import numpy as np
    import torch

    from paper_1108_2045_gb300 import inputs, learned

    n, L = CFG5_SIDE, CFG5_LEVELS
    kc = inputs.grf_coefficient(n, sigma=1.0, ell=0.05, seed=2)
    f_np = inputs.normal_rhs(n, 2, seed=0)
    k = torch.from_numpy(kc).cuda()
    f = torch.from_numpy(f_np).cuda()
    u = torch.zeros_like(f)
    unknowns = float((n - 1) ** 2)
    out = {"workload": "2-D -div(k grad u) = f, 5-point flux form with harmonic-mean faces, 2049^2 nodes, 11 levels, "
                       "k = exp(GRF sigma 1, ell 0.05, seed 2), f iid N(0,1) seed 0, to relres 1e-10",
           "k_range": [float(kc.min()), float(kc.max())]}

    def timed(fn, steps):
        fn()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            res = fn()
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1) / steps, res

    plain = {}
    for prec in ("fp64", "fp32"):
        with homg.Solver(2, n + 1, L, max_i=MAX_I, precision=prec) as s:
            s.set_stream(stream)
            s.set_coefficient(k)

            def solve():
                u.zero_()
                return s.solve(f, u, tol=TOL, max_cycles=MAX_CYCLES)

            ms, (st, cyc, rr) = timed(solve, args.cfg5_steps)
        plain[prec] = {"status": st, "cycles": cyc, "relres": rr, "ms_per_solve": ms, "unknowns_per_s": unknowns / (ms * 1e-3)}
    out["plain"] = plain
    with homg.Solver(2, n + 1, L, max_i=MAX_I, precision="fp32") as s, homg.Net() as net, homg.Net() as net_r:
        s.set_stream(stream)
        net.set_stream(stream)
        net_r.set_stream(stream)
        s.set_coefficient(k)
        net.set_params(learned.init_params(args.cfg5_seed))
        net_r.set_params(learned.init_params(args.cfg5_seed))
        net_r.set_loss("residual")
        t0 = time.perf_counter()
        fs_train = [torch.from_numpy(inputs.normal_rhs(n, 2, seed=100 + i)).cuda() for i in range(4)]
        X, T = learned.make_training_set(s, net, fs_train, cycles=(2, 3, 4), patches=args.cfg5_patches, seed=1)
        data_s = time.perf_counter() - t0
        target_ms = float((T.double() ** 2).mean())
        del fs_train
        losses, train_s = learned.train(net, X, T, epochs=args.cfg5_epochs, seed=2)
        losses_r, train_r_s = learned.train(net_r, X, T, epochs=args.cfg5_epochs, seed=2)
        del X, T
        out["training"] = {"patches": args.cfg5_patches, "patch": 64, "epochs": args.cfg5_epochs, "batch": 64,
                           "iterates_after_cycles": [2, 3, 4],
                           "data_seconds": data_s, "train_seconds": train_s, "loss_per_epoch": losses,
                           "target_mean_square": target_ms, "variance_explained": 1.0 - losses[-1] / target_ms,
                           "residual_loss": {"train_seconds": train_r_s, "loss_per_epoch": losses_r,
                                             "note": "same patches; loss = mean square of the residual the proposal "
                                                     "leaves (inputs have unit mean square: 1.0 = no reduction)"}}
        # the network alone on the full grid: tensor-core convolution throughput
        x_img = torch.zeros(1, n + 1, 2, n + 1, 8, dtype=torch.bfloat16, device="cuda")
        y_img = torch.zeros(1, n + 1, n + 1, dtype=torch.float32, device="cuda")
        u.zero_()
        homg.homg_features(s.handle, f, u, x_img)
        fwd_ms, _ = timed(lambda: net.forward(x_img, y_img), 5)
        px = float((n + 1) ** 2)
        flop_real = px * 2 * 9 * (2 * 32 + 32 * 32 * 2 + 32 * 1)
        flop_exec = px * 2 * 9 * (16 * 32 + 32 * 32 * 2 + 32 * 16)
        peaks, psrc = measured_peaks()
        bf16_peak = peaks.get("bf16_tflops", FALLBACK_BF16_TFLOPS)
        out["network"] = {"forward_ms": fwd_ms, "algorithmic_tflops": flop_real / (fwd_ms * 1e-3) / 1e12,
                          "executed_tflops": flop_exec / (fwd_ms * 1e-3) / 1e12,
                          "bf16_peak_tflops": bf16_peak, "peak_source": psrc,
                          "frac_of_bf16_peak": flop_exec / (fwd_ms * 1e-3) / 1e12 / bf16_peak,
                          "note": "4 tcgen05 convolution launches; executed FLOPs count the zero-padded channels "
                                  "(2 -> 16 inputs of layer 1, 1 -> 16 outputs of layer 4)"}
        del x_img, y_img
        learned_res = {}
        # (name, cycle precision, network, judge): the error-trained network judged on its own residual
        # (FP32 and FP64 cycles) and after the following cycle; the residual-trained network
        variants = [("fp32", "fp32", net, "proposal"), ("fp64", "fp64", net, "proposal"),
                    ("fp32_judge_after_cycle", "fp32", net, "after_cycle"),
                    ("fp32_residual_loss", "fp32", net_r, "proposal")]
        for name, prec, nw, judge in variants:
            with homg.Solver(2, n + 1, L, max_i=MAX_I, precision=prec) as s2:
                s2.set_stream(stream)
                s2.set_coefficient(k)
                homg.homg_set_learned_judge(s2.handle, judge)

                def lsolve():
                    u.zero_()
                    return homg.homg_solve_learned(s2.handle, nw, f, u, tol=TOL, max_cycles=MAX_CYCLES)

                ms, (st, cyc, rr, acc) = timed(lsolve, args.cfg5_steps)
            r = {"status": st, "cycles": cyc, "relres": rr, "ms_per_solve": ms, "unknowns_per_s": unknowns / (ms * 1e-3),
                 "judge": judge, "loss": "residual" if nw is net_r else "error",
                 "proposals_kept": int(sum(acc)), "decisions": [int(a) for a in acc],
                 "speedup_vs_plain_fp64": plain["fp64"]["ms_per_solve"] / ms,
                 "speedup_vs_plain_same_precision": plain[prec]["ms_per_solve"] / ms}
            if name == "fp32" and args.cfg5_oracle_check:
                pending.append((r, "vc", kc, f_np, u.cpu().numpy()))
            learned_res[name] = r
        out["learned"] = learned_res
    if args.cfg5_oracle_time:
        pending.append((out, "vc_time", kc, f_np, plain["fp64"]["cycles"]))
    del f, u, k
    torch.cuda.empty_cache()
    return out


def run_cfg1(args, homg, stream, barrier, pending):
    """cfg1: 129^2 nodes, 7 levels, f = 2 pi^2 sin(pi x) sin(pi y), to relres 1e-10 (the small case
    the oracle solves in full, timed beside it in the CPU leg); and T-paper: one cycle on the Sec. 4
    polynomial problem at 129^2 with MaxI 2, 4 and 32, the normalised L1 error against the analytic
    solution (the quantity of Fig. 4; the paper prints 5 % and 1.6 % for MaxI 4 and 32)."""
    import numpy as np
    import torch

    from paper_1108_2045_gb300 import inputs

    n, L = 128, 7
    f_np = inputs.sine_rhs(n, 2)
    f = torch.from_numpy(f_np).cuda()
    u = torch.zeros_like(f)
    out = {"workload": "2-D Poisson, 129^2 nodes, 7 levels, f = 2 pi^2 sin sin, to relres 1e-10"}
    with homg.Solver(2, n + 1, L, max_i=MAX_I) as s:
        s.set_stream(stream)
        u.zero_()
        s.solve(f, u, tol=TOL, max_cycles=MAX_CYCLES)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.cfg1_steps):
            u.zero_()
            st, cyc, rr = s.solve(f, u, tol=TOL, max_cycles=MAX_CYCLES)
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1) / args.cfg1_steps
    out.update(status=st, cycles=cyc, relres=rr, ms_per_solve=ms, unknowns_per_s=(n - 1) ** 2 / (ms * 1e-3))
    if args.cfg1_oracle_time:
        pending.append((out, "full_solve_time", None, f_np, L))
    fp = torch.from_numpy(inputs.paper_poly_rhs(n)).cuda()
    ue = inputs.paper_poly_solution(n)
    tp = {}
    for maxi in (2, 4, 32):
        with homg.Solver(2, n + 1, L, max_i=maxi) as s:
            s.set_stream(stream)
            up = torch.zeros_like(fp)
            s.solve(fp, up, tol=0.0, max_cycles=1)
            got = up.cpu().numpy()
        tp["max_i_%d" % maxi] = float(np.abs(got - ue).sum() / np.abs(ue).sum())
    out["tpaper_l1_error_one_cycle"] = tp
    return out


def run_pow2(args, homg, stream, barrier, pending):
    """Power-of-two grids (Sec. 3): 4096^2 nodes (boundary included), 12 levels, f iid uniform[-1, 1]
    over the interior (seed 0), whole-grid form, to relres 1e-10, FP64 and FP32 cycles."""
    import numpy as np
    import torch

    N, L = 4096, 12
    f_np = np.zeros((N, N))
    f_np[1:-1, 1:-1] = np.random.default_rng(0).uniform(-1, 1, (N - 2, N - 2))
    f = torch.from_numpy(f_np).cuda()
    u = torch.zeros_like(f)
    out = {"workload": "2-D Poisson, power-of-two grid of 4096^2 nodes (Sec. 3 quadrant lattices), 12 levels, "
                       "f iid uniform[-1,1] seed 0, whole-grid HOMG form, to relres 1e-10"}
    for prec in ("fp64", "fp32"):
        with homg.Solver(2, N, L, max_i=MAX_I, precision=prec, geometry="pow2") as s:
            s.set_stream(stream)
            u.zero_()
            s.solve(f, u, tol=TOL, max_cycles=MAX_CYCLES)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.pow2_steps):
                u.zero_()
                st, cyc, rr = s.solve(f, u, tol=TOL, max_cycles=MAX_CYCLES)
            e1.record(stream)
            barrier()
            ms = e0.elapsed_time(e1) / args.pow2_steps
            stats = s.stats()
        r = {"status": st, "cycles": cyc, "relres": rr, "ms_per_solve": ms,
             "unknowns_per_s": (N - 2) ** 2 / (ms * 1e-3), "iterations_per_cycle": stats["iterations_per_cycle"],
             "kernel_launches": stats["kernel_launches"]}
        if prec == "fp64" and args.pow2_oracle_check:
            pending.append((r, "poisson", None, f_np, u.cpu().numpy()))
        out[prec] = r
    del f, u
    torch.cuda.empty_cache()
    return out


def cpu_leg(pending):
    """Everything the oracle does in a bench run (the CPU-baseline leg): its own FP64 residual of
    results the GPU legs kept, and its timing on samples of their workloads."""
    import numpy as np

    import oracle

    oracle.build()
    for target, kind, kc, a, b in pending:
        if kind in ("poisson", "poisson_max"):
            rr = oracle.norm_interior(oracle.residual(a, b)) / oracle.norm_interior(a)
            key = "oracle_relres" if kind == "poisson" else "oracle_relres_max_sampled"
            target[key] = max(rr, target.get(key, 0.0))
        elif kind == "floor":
            target["oracle_floor_relres"] = oracle.norm_interior(oracle.residual(a, b)) / oracle.norm_interior(a)
        elif kind == "vc":
            target["oracle_relres"] = oracle.norm_interior(oracle.residual_vc(kc, a, b)) / oracle.norm_interior(a)
        elif kind == "batch_time":
            est, per_k = 0.0, {}
            for kk, (fks, cnt) in a.items():
                times, cycs = [], []
                for fk in fks:
                    t0 = time.perf_counter()
                    _, status, cyc, _ = oracle.solve_mixed(fk, kk, precision="fp32", tol=TOL, max_cycles=MAX_CYCLES)
                    times.append(time.perf_counter() - t0)
                    cycs.append(cyc)
                mean = sum(times) / len(times)
                per_k[str(kk)] = {"sampled": len(fks), "mean_seconds": mean, "cycles": cycs}
                est += mean * cnt
            target["cpu_oracle"] = {"value": b / est, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": "FP32-cycle oracle solves of 8/8/4/2/1 problems of sides 65..1025, mean time "
                                              "per size times the problems of that size (%.0f s estimated for the batch)" % est,
                                    "per_k": per_k}
        elif kind == "full_solve_time":
            t0 = time.perf_counter()
            _, status, cyc, _ = oracle.solve(a, b, tol=TOL, max_cycles=MAX_CYCLES, max_i=MAX_I)
            dt = time.perf_counter() - t0
            n = a.shape[0] - 1
            target["cpu_oracle"] = {"value": (n - 1) ** 2 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": "the full oracle solve (%d cycles, %.2f s)" % (cyc, dt),
                                    "ms_per_solve": 1e3 * dt}
        elif kind == "vc_time":
            t0 = time.perf_counter()
            oracle.cycle_vc(kc, a, CFG5_LEVELS)
            dt = time.perf_counter() - t0
            n = kc.shape[0] - 1
            target["cpu_oracle"] = {"value": (n - 1) ** 2 / (dt * b), "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": "one FP64 variable-coefficient oracle cycle on the 2049^2 grid (%.1f s), "
                                              "scaled by the %d cycles plain HOMG takes" % (dt, b)}


def run_reference(args):
    """The reference arm: the oracle (the paper publishes no code) on the benchmark workload, one
    thread of the host. A step is one MFMG cycle of the restarted oracle solve (restriction, 286
    HOMG iterations over the 4097^2 grid, update and residual); consecutive steps continue the same
    solve from u0 = 0, so the run itself observes how many cycles reach relres 1e-10 (cycles are
    added, untimed, if warm-up plus timed steps end first). ms_per_step is the measured mean time of
    a timed step; value = unknowns / (that time x the observed cycle count)."""
    world, rank, local = dist_setup(args)
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_1108_2045_gb300 import inputs

    oracle.build()
    f = inputs.uniform_rhs(N_SIDE, 2, seed=0)
    u = np.zeros_like(f)
    times, relres, converged_after = [], None, None
    cycles_done = 0

    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        u_next, _, _, hist = oracle.solve(f, LEVELS, u0=u, tol=0.0, max_cycles=1, max_i=MAX_I)
        dt = time.perf_counter() - t0
        u = u_next
        cycles_done += 1
        relres = hist[-1]
        if converged_after is None and relres <= TOL:
            converged_after = cycles_done
        if step >= args.warmup:
            times.append(dt)
    while converged_after is None and cycles_done < MAX_CYCLES:  # untimed: only to count cycles
        u, _, _, hist = oracle.solve(f, LEVELS, u0=u, tol=0.0, max_cycles=1, max_i=MAX_I)
        cycles_done += 1
        relres = hist[-1]
        if relres <= TOL:
            converged_after = cycles_done
    if converged_after is None:
        raise RuntimeError("the oracle solve did not reach relres %g" % TOL)
    step_s = sum(times) / len(times)
    value = (N_SIDE - 1) ** 2 / (step_s * converged_after)
    sample = ("each step: one MFMG cycle of the oracle's restarted solve on the 4097^2 grid (one thread), steps "
              "continuing one solve from u0 = 0; relres 1e-10 after %d cycles (observed in this run); "
              "value = unknowns / (mean step time %.1f s x %d)" % (converged_after, step_s, converged_after))
    cpu = {"value": value, "unit": UNIT, "cores": 1, "host_cores": host_cores(), "kind": "oracle", "sample": sample}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * step_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config("fp64", args.gpus),
            "run": {"step": "one oracle MFMG cycle", "cycles_to_tol": converged_after},
            "impl": "reference", "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(precision, n_gpus):
    """The benchmarked workload, identical in both arms (the run's own results go under "run")."""
    return {"workload": WORKLOAD, "precision": precision, "grid": N_SIDE + 1, "levels": LEVELS, "max_i": MAX_I,
            "tol": TOL, "l2": "working set ~0.8 GB > 126 MB L2; no flush",
            "parallelism": "replicas" if n_gpus > 1 else "single GPU"}


def legs_digest(line):
    """Compact summary of every leg of the line (ms per solve, cycles, checks), kept short so that it
    fits at the end of the printed line."""
    def r3(x):
        return None if x is None else float("%.4g" % x)

    prec = line["config"]["precision"]  # the headline leg's cycle precision (fp64 by default)
    d = {prec + "_ms": r3(line["ms_per_step"]), prec + "_cyc": line["run"]["cycles"],
         "roof_hbm": r3(line["roofline"]["frac"])}
    alu = line["roofline"].get("alu", {})
    if "frac" in alu:
        d["roof_fp64pipe"] = r3(alu["frac"])
        d["fp64_peak_T"] = r3(alu["peak"])
    if "e2e" in line:
        d["e2e_Mps"] = r3(line["e2e"]["value"] / 1e6)
    for k, v in line.get("mixed_precision", {}).items():
        d[k + "_ms"] = [r3(v["ms_per_step"]), v["cycles"], r3(v["fine_hbm_frac"])]
    for k, v in line.get("vcycle_v22", {}).items():
        d["v22_" + k + "_ms"] = [r3(v["ms_per_step"]), v["cycles"]]
    if "wholegrid" in line:
        d["wg_ms"] = r3(line["wholegrid"]["ms_per_step"])
    c = line.get("cfg2_manufactured")
    if c:
        d["sine4097"] = {"floor": r3(c["floor_relres"]), "homg": [r3(c["homg"]["ms_per_solve"]), c["homg"]["cycles"]],
                         "v22": [r3(c["v22"]["ms_per_solve"]), c["v22"]["cycles"]],
                         "orc_rr": r3(c["homg"].get("oracle_relres"))}
    c = line.get("cfg1_small")
    if c:
        d["cfg1"] = [r3(c["ms_per_solve"]), c["cycles"], r3(c.get("cpu_oracle", {}).get("ms_per_solve"))]
    c = line.get("cfg3_3d")
    if c:
        d["cfg3"] = {rhs: {p: [r3(v["ms_per_solve"]), v["cycles"]] for p, v in c[rhs].items()}
                     for rhs in ("sine", "normal") if rhs in c}
    c = line.get("cfg4_batched")
    if c:
        d["cfg4"] = {p: [r3(c[p]["batch_ms"]), r3(c[p]["solve_ms_p50"]), r3(c[p]["solve_ms_p99"]), c[p]["all_converged"]]
                     for p in ("fp32", "fp64", "fp32_persistent") if p in c}
    c = line.get("cfg5_learned")
    if c:
        d["cfg5"] = {"plain": {p: r3(v["ms_per_solve"]) for p, v in c["plain"].items()},
                     "learned": {p.replace("fp32_", ""): [r3(v["ms_per_solve"]), v["cycles"], v["proposals_kept"]]
                                 for p, v in c.get("learned", {}).items()}}
    c = line.get("pow2_grid")
    if c:
        d["pow2"] = {p: [r3(c[p]["ms_per_solve"]), c[p]["cycles"]] for p in ("fp64", "fp32") if p in c}
    if "cpu_baseline" in line:
        d["cpu_Mps"] = r3(line["cpu_baseline"]["value"] / 1e6)
    return d


def run(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__

    __graft_entry__.build()
    from paper_1108_2045_gb300 import homg, inputs

    dev = torch.device("cuda", local)
    f_np = inputs.uniform_rhs(N_SIDE, 2, seed=0)
    f = torch.from_numpy(f_np).to(dev)
    u = torch.zeros_like(f)
    stream = torch.cuda.current_stream(dev)
    solver = homg.Solver(2, N_SIDE + 1, LEVELS, max_i=MAX_I, exec_mode=args.exec, launch_mode=args.launch,
                         precision=args.precision)
    solver.set_stream(stream)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def step():
        u.zero_()
        status, cycles, relres = solver.solve(f, u, tol=TOL, max_cycles=MAX_CYCLES)
        if status != homg.HOMG_OK:
            raise RuntimeError("solve did not converge: status %d after %d cycles (relres %.3e)" % (status, cycles, relres))
        return cycles, relres

    for _ in range(args.warmup):
        step()
    # timed region: K device-resident solves
    stats = []
    barrier()
    with ClockSampler(local) as clocks:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            cycles, relres = step()
            stats.append(solver.stats())
        t1.record(stream)
        barrier()
    unknowns = (N_SIDE - 1) ** 2
    value = replica_throughput(unknowns * args.steps, t0.elapsed_time(t1) * 1e-3, dev)
    elapsed_ms = max_over_ranks(t0.elapsed_time(t1), dev)

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    f_host = torch.from_numpy(f_np).pin_memory()
    u_host = torch.zeros_like(f_host).pin_memory()
    solver.solve_host(f_host, u_host, tol=TOL, max_cycles=MAX_CYCLES)
    barrier()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        u_host.zero_()
        st, _, _ = solver.solve_host(f_host, u_host, tol=TOL, max_cycles=MAX_CYCLES)
        if st != homg.HOMG_OK:
            raise RuntimeError("host solve did not converge")
    barrier()
    e2e_value = replica_throughput(unknowns * args.steps, time.perf_counter() - e0, dev)
    grid_bytes = f_np.nbytes

    # whole-grid form of the same iterates (the paper's one-launch-per-iteration layout), for contrast
    wg = None
    if args.wholegrid_steps > 0:
        with homg.Solver(2, N_SIDE + 1, LEVELS, max_i=MAX_I, exec_mode="wholegrid") as s2:
            s2.set_stream(stream)
            u.zero_()
            s2.solve(f, u, tol=TOL, max_cycles=MAX_CYCLES)
            ws = []
            barrier()
            w0 = torch.cuda.Event(enable_timing=True)
            w1 = torch.cuda.Event(enable_timing=True)
            w0.record(stream)
            for _ in range(args.wholegrid_steps):
                u.zero_()
                s2.solve(f, u, tol=TOL, max_cycles=MAX_CYCLES)
                ws.append(s2.stats())
            w1.record(stream)
            barrier()
            wms = w0.elapsed_time(w1) / args.wholegrid_steps
            iters = sum(s["cycles"] * (s["iterations_per_cycle"] - s["fine_iterations_per_cycle"]) for s in ws)
            coarse_ms = sum(s["coarse_ms"] for s in ws)
            wg = {"value": unknowns / (wms * 1e-3), "ms_per_step": wms,
                  "coarse_iteration_us": 1e3 * coarse_ms / iters if iters else None}

    # mixed precision (FP32 / bfloat16 cycles inside the FP64 restart loop) on the same workload
    mixed = {}
    peaks, peak_src = measured_peaks()
    hbm_peak_mp = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
    for prec in ([] if args.mixed_steps <= 0 else ["fp32", "bf16"]):
        with homg.Solver(2, N_SIDE + 1, LEVELS, max_i=MAX_I, precision=prec) as s3:
            s3.set_stream(stream)
            for _ in range(3):
                u.zero_()
                s3.solve(f, u, tol=TOL, max_cycles=MAX_CYCLES)
            ms_list, sts = [], []
            barrier()
            m0 = torch.cuda.Event(enable_timing=True)
            m1 = torch.cuda.Event(enable_timing=True)
            m0.record(stream)
            for _ in range(args.mixed_steps):
                u.zero_()
                st3, c3, r3 = s3.solve(f, u, tol=TOL, max_cycles=MAX_CYCLES)
                if st3 != homg.HOMG_OK:
                    raise RuntimeError("%s solve did not converge" % prec)
                sts.append(s3.stats())
            m1.record(stream)
            barrier()
            mms = m0.elapsed_time(m1) / args.mixed_steps
            # level 0: consecutive plain sweeps run fused (two per launch), each launch moving the
            # algorithmic bytes of one sweep
            fl = sum(x["cycles"] * x["fine_launches_per_cycle"] for x in sts)
            fi = sum(x["cycles"] * x["fine_iterations_per_cycle"] for x in sts)
            fine_total_ms = sum(x["fine_ms"] for x in sts)
            fus = 1e3 * fine_total_ms / fl
            fb = sts[0]["fine_bytes_per_iteration"]
            mixed[prec] = {"value": unknowns / (mms * 1e-3), "ms_per_step": mms, "cycles": c3, "final_relres": r3,
                           "speedup_vs_fp64": (elapsed_ms / args.steps) / mms,
                           "fine_launches_per_cycle": sts[0]["fine_launches_per_cycle"],
                           "fine_sweep_us": 1e3 * fine_total_ms / fi,
                           "fine_launch_us": fus, "fine_hbm_gbs": fb / (fus * 1e-6) / 1e9,
                           "fine_hbm_frac": fb / (fus * 1e-6) / 1e9 / hbm_peak_mp,
                           "time_split_ms_per_step": {k: sum(x[k] for x in sts) / len(sts)
                                                      for k in ("coarse_ms", "fine_ms", "residual_ms", "setup_ms")}}

    # classic V(2,2) cycle on the same workload and GPU (the comparator named by the benchmark config)
    vcyc = {}
    for prec in ([] if args.vcycle_steps <= 0 else ["fp64", "fp32"]):
        with homg.Solver(2, N_SIDE + 1, LEVELS, cycle="v", precision=prec) as s4:
            s4.set_stream(stream)
            for _ in range(3):
                u.zero_()
                s4.solve(f, u, tol=TOL, max_cycles=MAX_CYCLES)
            sts = []
            barrier()
            v0 = torch.cuda.Event(enable_timing=True)
            v1 = torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            for _ in range(args.vcycle_steps):
                u.zero_()
                st4, c4, r4 = s4.solve(f, u, tol=TOL, max_cycles=MAX_CYCLES)
                if st4 != homg.HOMG_OK:
                    raise RuntimeError("V-cycle solve did not converge")
                sts.append(s4.stats())
            v1.record(stream)
            barrier()
            vms = v0.elapsed_time(v1) / args.vcycle_steps
            homg_ms = (elapsed_ms / args.steps) if prec == "fp64" else mixed.get("fp32", {}).get("ms_per_step")
            vcyc[prec] = {"value": unknowns / (vms * 1e-3), "ms_per_step": vms, "cycles": c4, "final_relres": r4,
                          "homg_ms_over_v_ms": (homg_ms / vms) if homg_ms else None,
                          "time_split_ms_per_step": {k: sum(x[k] for x in sts) / len(sts)
                                                     for k in ("coarse_ms", "fine_ms", "residual_ms", "setup_ms")}}
    # the FP64 pipe's issue rate on this GPU, now (denominator of the FP64 ALU fraction)
    fp64_peak = measure_fp64_peak(homg, stream, dev, local) if args.fp64_probe else None
    pending = []  # oracle work of the CPU leg (rank 0, one GPU only)
    cfg2s = run_cfg2_sine(args, homg, inputs, stream, barrier, pending) if (args.cfg2_sine_steps > 0 and world == 1) else None
    cfg1 = run_cfg1(args, homg, stream, barrier, pending) if (args.cfg1_steps > 0 and world == 1) else None
    cfg3 = run_cfg3(args, homg, inputs, stream, barrier, pending) if (args.cfg3_steps > 0 and world == 1) else None
    cfg4 = run_cfg4(args, homg, stream, barrier, pending) if (args.cfg4_steps > 0 and world == 1) else None
    cfg5 = run_cfg5(args, homg, stream, barrier, pending) if (args.cfg5_steps > 0 and world == 1) else None
    pow2 = run_pow2(args, homg, stream, barrier, pending) if (args.pow2_steps > 0 and world == 1) else None
    hbm_peak = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
    # dominant kernel: the level-0 HOMG iteration (damped Jacobi over every interior node)
    # (binary32 cycles fuse consecutive plain sweeps: a launch then does two sweeps' arithmetic on one
    # sweep's traffic)
    launches = sum(s["cycles"] * s["fine_launches_per_cycle"] for s in stats)
    fine_ms = sum(s["fine_ms"] for s in stats)
    per_launch_s = fine_ms * 1e-3 / launches
    sweeps_per_launch = stats[0]["fine_iterations_per_cycle"] / stats[0]["fine_launches_per_cycle"]
    ops = stats[0]["fine_flops_per_iteration"] * sweeps_per_launch
    bts = stats[0]["fine_bytes_per_iteration"]
    alu_achieved = ops / per_launch_s / 1e12
    hbm_achieved = bts / per_launch_s / 1e9
    clk = clocks.summary()
    # FP64 instructions the level-0 sweep issues per interior node: one shared neighbour pair and
    # three FMAs per node, on warps of 63 output columns out of 64 (k_jacobi2d2)
    fp64_issued_per_node = 4.0 * 64 / 63
    kname = ("k_jacobi2d2 (level-0 HOMG iteration: damped Jacobi on every interior node, shared neighbour pairs)"
             if args.precision == "fp64" else
             "k_jacobi2 (level-0 HOMG iteration: damped Jacobi on every interior node)" if sweeps_per_launch == 1 else
             "k_jacobi2_x2 / k_jacobi2 (level-0 HOMG iterations, consecutive plain sweeps fused two per launch; "
             "average over the level's launches)")
    # DRAM bytes (read + write) per launch of this kernel from ncu: the FP64 sweep
    # (profiles/k_jacobi2d2_fp64_4097.md) and the fused FP32 pair (profiles/k_jacobi2_x2_fp32_4097.md;
    # the level's two single FP32 sweeps move the same bytes); the bfloat16 build was not captured
    traffic, traffic_src = {"fp64": (LEVEL0_FP64_DRAM_BYTES, "profiles/k_jacobi2d2_fp64_4097.md"),
                            "fp32": (LEVEL0_FP32_DRAM_BYTES, "profiles/k_jacobi2_x2_fp32_4097.md")}.get(
        args.precision, (None, None))
    common = {"kernel": kname, "launch_us": per_launch_s * 1e6, "launches": launches,
              "algorithmic_flops_per_launch": ops, "algorithmic_bytes_per_launch": bts, "traffic": traffic,
              "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, " + traffic_src if traffic else None}
    # The roofline is the HBM one (algorithmic bytes per launch / launch time / measured copy
    # bandwidth). An FP64 sweep is bound on GB300 by the FP64 pipe instead (4.06 FP64 instructions
    # issued per 24 bytes): its ALU fraction, against the issue rate measured in this run, is carried
    # beside it, counted in the instructions the kernel issues (the method's own count, 5 per node
    # as one FMA per neighbour, centre and source, is given as well).
    roofline = dict(common, bound="hbm", achieved=hbm_achieved, peak=hbm_peak, unit="GB/s",
                    frac=hbm_achieved / hbm_peak, peak_source=peak_src + " (MEASURED_PEAKS.json hbm_gbs)")
    if fp64_peak:
        p_meas = fp64_peak["peak_tinstr_per_s"]
        instr_unit = "T FP64 instr/s" if args.precision == "fp64" else "T FP32 instr/s"
        roofline["alu"] = {"binding": args.precision == "fp64", "achieved": alu_achieved, "unit": instr_unit,
                           "instructions_per_launch": ops}
        if args.precision == "fp64":
            issued = ops / 5.0 * fp64_issued_per_node
            alu_achieved = issued / per_launch_s / 1e12
            roofline["alu"].update(achieved=alu_achieved, instructions_per_launch=issued,
                                   instructions_per_node=fp64_issued_per_node, method_instructions_per_launch=ops,
                                   peak=p_meas, frac=alu_achieved / p_meas,
                                   peak_source="measured in this run: homg_fp64_issue_probe, mean of 20 back-to-back "
                                               "launches (FMA %.3f, ADD %.3f T instr/s; SM clock median %s MHz)" % (
                                                   fp64_peak["fma"]["mean_tinstr_per_s"],
                                                   fp64_peak["add"]["mean_tinstr_per_s"],
                                                   fp64_peak["clocks"].get("sm_mhz")),
                                   nominal_peak=FP64_NOMINAL_OPS / 1e12, frac_of_nominal=alu_achieved / (FP64_NOMINAL_OPS / 1e12))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32 cycles, f64 residual/update", "bf16": "bf16 cycles, f64 residual/update"}[args.precision],
        "data": "synthetic",
        "config": workload_config(args.precision, world),
        "run": {"exec": args.exec, "exec_used": {1: "wholegrid", 2: "lattice"}[stats[0]["exec_mode"]],
                "cycles": stats[-1]["cycles"], "final_relres": relres,
                "iterations_per_cycle": stats[0]["iterations_per_cycle"], "launch": args.launch},
        "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": 2 * grid_bytes, "d2h_bytes_per_step": grid_bytes},
        "gpu_launches": int(sum(s["kernel_launches"] for s in stats)),
        "clocks": clk,
        "time_split_ms_per_step": {k: sum(s[k] for s in stats) / len(stats)
                                   for k in ("coarse_ms", "fine_ms", "residual_ms", "setup_ms", "solve_ms")},
    }
    if fp64_peak:
        line["fp64_issue_probe"] = fp64_peak
    if wg:
        line["wholegrid"] = wg
    if cfg2s:
        line["cfg2_manufactured"] = cfg2s
    if mixed:
        line["mixed_precision"] = mixed
    if vcyc:
        line["vcycle_v22"] = vcyc
    if args.cfg3_steps > 0 and world == 1:
        line["cfg3_3d"] = cfg3
    if cfg1:
        line["cfg1_small"] = cfg1
    if cfg4:
        line["cfg4_batched"] = cfg4
    if cfg5:
        line["cfg5_learned"] = cfg5
    if pow2:
        line["pow2_grid"] = pow2
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_cpu_baseline(f_np, full=args.cpu_baseline == "full")
        cpu_leg(pending)
    # last key: a compact digest of every leg, so that the end of the printed line carries them all
    line["legs"] = legs_digest(line)
    solver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    p = argparse.ArgumentParser(description=__doc__)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="homg", choices=["homg", "reference"])
    p.add_argument("--exec", default="auto", choices=["auto", "lattice", "wholegrid"])
    p.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "bf16"],
                   help="precision of the timed solver's cycles (the FP64 workload is the headline)")
    p.add_argument("--wholegrid-steps", type=int, default=2)
    p.add_argument("--launch", default="graph", choices=["graph", "stream"],
                   help="stream: enqueue kernels directly (for profilers that cannot see inside conditional graphs)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-baseline", default="full", choices=["full", "cycle"],
                   help="full: time the oracle's complete 4097^2 solve (about 2 minutes on one core); cycle: one cycle, scaled")
    p.add_argument("--no-fp64-probe", dest="fp64_probe", action="store_false")
    p.add_argument("--cfg2-sine-steps", type=int, default=2,
                   help="timed solves per cycle type of the 4097^2 manufactured right-hand side (0: skip)")
    p.add_argument("--mixed-steps", type=int, default=3, help="timed solves per mixed-precision variant (0: skip)")
    p.add_argument("--cfg3-steps", type=int, default=2, help="timed 513^3 solves per precision and RHS (0: skip)")
    p.add_argument("--cfg3-side", type=int, default=CFG3_SIDE, choices=[64, 128, 256, 512],
                   help="intervals per side of the 3-D leg (512: the 513^3 workload; smaller for profiling)")
    p.add_argument("--vcycle-steps", type=int, default=3, help="timed V(2,2) comparator solves (0: skip)")
    p.add_argument("--cfg4-steps", type=int, default=2, help="timed batched solves of the 1024-problem batch (0: skip)")
    p.add_argument("--no-cfg4-oracle-check", dest="cfg4_oracle_check", action="store_false")
    p.add_argument("--no-cfg4-oracle-time", dest="cfg4_oracle_time", action="store_false")
    p.add_argument("--cfg5-steps", type=int, default=2, help="timed solves per form of the 2049^2 variable-coefficient workload (0: skip)")
    p.add_argument("--cfg5-epochs", type=int, default=6, help="training epochs of the learned corrector")
    p.add_argument("--cfg5-patches", type=int, default=20000)
    p.add_argument("--cfg5-seed", type=int, default=0, help="seed of the network's initial parameters")
    p.add_argument("--no-cfg5-oracle-check", dest="cfg5_oracle_check", action="store_false")
    p.add_argument("--no-cfg5-oracle-time", dest="cfg5_oracle_time", action="store_false")
    p.add_argument("--cfg1-steps", type=int, default=5, help="timed solves of the 129^2 case (0: skip)")
    p.add_argument("--no-cfg1-oracle-time", dest="cfg1_oracle_time", action="store_false")
    p.add_argument("--pow2-steps", type=int, default=2, help="timed solves on the 4096^2 power-of-two grid (0: skip)")
    p.add_argument("--no-pow2-oracle-check", dest="pow2_oracle_check", action="store_false")
    p.add_argument("--no-cfg3-oracle-check", dest="cfg3_oracle_check", action="store_false")
    args = p.parse_args()
    if args.warmup < 3:
        p.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
