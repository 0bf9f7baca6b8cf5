"""Benchmark of the triangular solve on GB300.

Workload (one "step"): Left/Lower/NoTrans/NonUnit solve with m = n = 16384,
alpha = 1.5, synthetic well-conditioned inputs (diagonal U[1,2), off-diagonal
U(-1,1)/m, B ~ N(0,1), seed 0), through the library's C entry point, solved
to FP64-level error by the mixed-precision path (BF16 tensor-core solve plus
split-precision refinement); the plain FP64 solve of the same problem is
timed after it on the same GPU for comparison (--path fp64 makes the plain
solve the timed step).  Inputs (A 2 GiB + B 2 GiB in FP64) are larger than
L2, and B is re-copied from a pristine device copy before every step (outside
the timed events), which also evicts L2.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TRSM TFLOP/s at FP64-level error: mixed+refine vs plain FP64, same GB300"
UNIT = "TFLOP/s"
# FP64 arithmetic peak used for the roofline: 152 SMs x 2 DFMA/clk/SM x 2 flop
# x 2.07 GHz (maximum SM clock); a DFMA throughput probe measured 1.196 TF/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


MEASURED_PEAKS = _measured_peaks()


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--m", type=int, default=16384)
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--path", default="mixed", choices=["mixed", "fp64", "batched", "potrf"])
    p.add_argument("--dtype", default="f64", choices=["f64", "f32"], help="batched path precision")
    p.add_argument("--prec", default="bf16", choices=["bf16", "fp8"], help="mixed path low precision")
    p.add_argument("--count", type=int, default=4096, help="batched path: number of problems")
    p.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison leg")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the other configurations (FP8 mixed, 32768 x 4096, the 16 plain FP64 forms)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-cols", type=int, default=0,
                   help="right-hand sides in the oracle sample (0 = auto, ~10-30 s)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- clocks ------

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
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
        self.t.join(timeout=2)
        sm, smax, power, reasons = [], None, [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": ["no samples"]}
        under = [s for s, p in zip(sm, power)] if not power else \
            [s for s, p in zip(sm, power) if p > 0.25 * max(power)]
        under = under or sm
        return {"sm_mhz": float(np.median(under)), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


# -------------------------------------------------------------- oracle arm ----

_ORACLE_INPUTS = {}


def oracle_sample(m, n_sample, seed=0, nthreads=0):
    """Time the CPU oracle on n_sample right-hand sides of the workload
    (the triangle A is generated once per (m, seed) and reused).
    Returns (seconds, flops, threads)."""
    import oracle
    from paper_2305_19917_gb300 import inputs
    key = (m, seed)
    if key not in _ORACLE_INPUTS:
        _ORACLE_INPUTS.clear()
        _ORACLE_INPUTS[key] = inputs.make_problem(0, 0, 0, 0, m, 1, seed)[0]
    A = _ORACLE_INPUTS[key]
    B = np.random.default_rng(seed + 1).standard_normal((m, n_sample))
    X = np.asfortranarray(B)
    threads = nthreads if nthreads > 0 else (os.cpu_count() or 1)
    t0 = time.perf_counter()
    oracle.dtrsm_inplace(0, 0, 0, 0, 1.5, A, X, nthreads=threads)
    dt = time.perf_counter() - t0
    return dt, float(m) * m * n_sample, threads


def auto_sample_cols(m, target_s=15.0):
    """Pick a column count giving roughly target_s seconds of oracle work."""
    probe = 16
    dt, _, _ = oracle_sample(m, probe)
    cols = int(probe * target_s / max(dt, 1e-3))
    return max(16, min(cols, 4096)), dt


def cpu_baseline(m, cols):
    dt, flops, threads = oracle_sample(m, cols)
    return {"value": flops / dt / 1e12, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"FP64 substitution (C, OpenMP over right-hand sides) on {cols} of the "
                      f"{m}x{m} Left/Lower/N solve's right-hand sides, {dt:.1f} s; TFLOP/s = "
                      f"m^2*cols/time"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    m = args.m
    cols = args.cpu_sample_cols or auto_sample_cols(m, target_s=max(3.0, 60.0 / max(1, args.steps + args.warmup)))[0]
    for _ in range(args.warmup):
        oracle_sample(m, max(16, cols // 8))
    times = []
    for _ in range(args.steps):
        dt, flops, threads = oracle_sample(m, cols)
        times.append(dt)
    t = float(np.mean(times))
    value = float(m) * m * cols / t / 1e12
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"Left/Lower/N/NonUnit TRSM m={m}, sample of {cols} right-hand sides "
                                   f"(CPU oracle), alpha=1.5, seed 0"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{cols} right-hand sides of the m={m} solve per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm ---

def _timed_steps(solve, reset, steps, stream):
    """Run `steps` solves, each bracketed by CUDA events on `stream` (the B
    reset copy before each one is outside the events)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    out = []
    for i in range(steps):
        reset()
        ev[i][0].record(stream)
        out.append(solve())
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], out


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2305_19917_gb300 import api, inputs
    from paper_2305_19917_gb300 import dist as gdist

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    api.lib()
    m, n = args.m, args.n
    side, uplo, trans, diag, alpha = 0, 0, 0, 0, 1.5
    tol, max_iter = 1e-11, 60
    prec = api.PREC_FP8 if args.prec == "fp8" else api.PREC_BF16

    # One problem with world * n right-hand sides, sharded over the ranks
    # (n per GPU, no exchange): every rank holds A and its own block of B.
    # Host inputs (seeded; rank 0's block is the single-GPU workload's B),
    # device copies.
    A_h, B_h = inputs.make_problem(side, uplo, trans, diag, m, n, seed=0)
    if rank > 0:
        B_h = np.asfortranarray(np.random.default_rng(10_000 + rank).standard_normal((m, n)))
    A = api.to_device_colmajor(A_h, torch.float64)
    B0 = api.to_device_colmajor(B_h, torch.float64)
    B = api.colmajor_empty(m, n, torch.float64)
    stream = torch.cuda.current_stream()
    flops = float(m) * m * n
    mixed = args.path == "mixed"

    def reset():
        B.copy_(B0)

    def solve_mixed():
        _, _, st, it, est = gdist.solve_sharded(side, uplo, trans, diag, alpha, A, B, rank=rank, world=world,
                                                total=world * n, path="mixed", tol=tol, prec=prec,
                                                max_iter=max_iter, stream=stream)
        if st < 0 or st in (api.STATUS_CUDA_ERROR, api.STATUS_TIMEOUT):
            raise api.GbError("gb_dtrsm_mixed", st)
        return st, it, est, api.gb_mixed_history()

    def solve_fp64():
        gdist.solve_sharded(side, uplo, trans, diag, alpha, A, B, rank=rank, world=world, total=world * n,
                            path="plain", stream=stream)
        return None

    solve = solve_mixed if mixed else solve_fp64
    for _ in range(max(3, args.warmup)):
        reset()
        solve()
    torch.cuda.synchronize()

    # ---- timed region: K steps ----
    clocks = ClockSampler(dev)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    api.gb_profile_enable(1)
    launches0 = api.gb_kernel_launches()
    wall0 = time.perf_counter()
    ms, outs = _timed_steps(solve, reset, args.steps, stream)
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    launches = api.gb_kernel_launches() - launches0
    clk = clocks.stop()
    prof = {k: api.gb_profile_read(i) for i, k in enumerate(api.KERNEL_KINDS)}
    api.gb_profile_enable(0)
    ms_step = float(np.sum(ms) / args.steps)
    if world > 1:
        t = torch.tensor([ms_step], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = world * flops / (ms_step * 1e-3) / 1e12

    # accuracy on sampled right-hand sides (oracle, CPU) -- not timed
    acc = None
    if rank == 0:
        import oracle
        cols = [0, n // 3, n - 1]
        Xs = B[:, cols].cpu().numpy()
        Xo = oracle.dtrsm(side, uplo, trans, diag, alpha, A_h, B_h[:, cols])
        acc = {"fwd_err_sampled": float(np.linalg.norm(Xs - Xo) / np.linalg.norm(Xo)), "columns": cols}
        if mixed:
            acc["refinement_steps"] = [o[1] for o in outs]
            acc["est_err"] = [o[2] for o in outs]
            acc["status"] = [o[0] for o in outs]
            acc["history_rho_levels"] = outs[-1][3]

    # ---- e2e: host buffers, H2D + solve + D2H inside the timed region ----
    # the mixed path goes through the library's host-buffer entry point (it
    # copies A's referenced triangle and B in, overlaps B's copy with the
    # A-only kernels, and copies X back); the plain path copies A and B in
    # and X out around the device call
    A_pin = torch.empty((m, m), dtype=torch.float64, pin_memory=True).t()
    A_pin.copy_(A)
    B_pin = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
    B_host0 = B0.cpu()
    e2e_ms = []
    if mixed:
        h2d, d2h = api.gb_mixed_host_bytes(side, uplo, m, n)
    else:
        A_e = api.colmajor_empty(m, m, torch.float64)
        h2d, d2h = (m * m + m * n) * 8, m * n * 8
    if mixed:
        # two untimed calls: the host entry point solves in column blocks, whose
        # low-precision solve graph is captured and whose buffers are mapped on first use
        for _ in range(2):
            B_pin.copy_(B_host0)
            api.trsm_mixed_host(side, uplo, trans, diag, alpha, A_pin, B_pin, tol=tol, prec=prec,
                                max_iter=max_iter, stream=stream)
    for _ in range(max(1, min(args.steps, 10))):
        B_pin.copy_(B_host0)  # fresh right-hand sides (host copy, not timed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        if mixed:
            api.trsm_mixed_host(side, uplo, trans, diag, alpha, A_pin, B_pin, tol=tol, prec=prec,
                                max_iter=max_iter, stream=stream)
        else:
            A_e.copy_(A_pin, non_blocking=True)
            B.copy_(B_pin, non_blocking=True)
            api.trsm(side, uplo, trans, diag, alpha, A_e, B, stream=stream)
            B_pin.copy_(B, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_t = float(np.mean(e2e_ms))
    if world > 1:
        t = torch.tensor([e2e_t], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_t = float(t.item())
    if mixed:
        # the host solution's own error, and its distance from the device-resident one
        if acc:
            Xe = B_pin[:, cols].numpy()
            acc["e2e_fwd_err_sampled"] = float(np.linalg.norm(Xe - Xo) / np.linalg.norm(Xo))
            acc["e2e_max_abs_diff_vs_device"] = float(np.abs(Xe - Xs).max())
    del A_pin, B_pin

    # ---- plain FP64 on the same GPU, same workload (the comparison) ----
    plain = None
    if mixed and not args.no_plain:
        for _ in range(1):
            reset()
            solve_fp64()
        pms, _ = _timed_steps(solve_fp64, reset, 2, stream)
        pt = float(np.mean(pms))
        plain = {"value": flops / (pt * 1e-3) / 1e12, "unit": UNIT, "ms_per_step": pt, "steps": 2,
                 "speedup_of_mixed": pt / ms_step}

    # ---- roofline of the dominant kernel (largest share of device time) ----
    # (a "graph" record is a whole captured sequence of kernels, not one kernel)
    dom = max((k for k in prof if k != "graph"), key=lambda k: prof[k]["ms"])
    p = prof[dom]
    achieved = p["flops"] / (p["ms"] * 1e-3) / 1e12 if p["ms"] > 0 else 0.0
    if dom in ("gemm_tc", "residual"):
        peak = MEASURED_PEAKS.get("bf16_tflops_sustained") or 1700.0
        bound, src = "tensor", "MEASURED_PEAKS.json bf16_tflops_sustained (kernel timed inside a long step)"
    else:
        peak, bound = FP64_PEAK_TFLOPS, "alu"
        src = ("derived: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz (not in MEASURED_PEAKS.json; "
               "probe measured 1.196 TF/s DFMA)")
    traffic = RESIDUAL_DRAM_BYTES.get((m, n, args.prec)) if (mixed and dom == "residual") else None
    roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": src,
                "launches": p["launches"], "ms_total": p["ms"],
                "share": p["ms"] / max(1e-9, sum(v["ms"] for v in prof.values()))}

    extras = None
    if mixed and not args.no_extras:
        # free the headline workload's buffers first (the extras need up to ~20 GB)
        del A, B0, B
        torch.cuda.empty_cache()
        extras = run_extras(stream, rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cols = args.cpu_sample_cols or auto_sample_cols(m)[0]
        cpu = cpu_baseline(m, cols)

    if rank == 0:
        if mixed:
            wl = (f"mixed {args.prec.upper()} + refinement TRSM Left/Lower/N/NonUnit m=n={m} to FP64-level error "
                  f"(tol {tol:g} on ||D||/||X||; forward error vs FP64 oracle <= 1e-10), alpha=1.5, "
                  f"diag U[1,2), offdiag U(-1,1)/m, B~N(0,1), seed 0")
        else:
            wl = (f"plain FP64 TRSM Left/Lower/N/NonUnit m=n={m}, alpha=1.5, diag U[1,2), "
                  f"offdiag U(-1,1)/m, B~N(0,1), seed 0, planner default plan")
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": (args.prec + "+f64") if mixed else "f64", "data": "synthetic",
                "config": {"workload": wl, "global_batch": world,
                           "sharding": (f"one problem with {world} x {n} right-hand sides split over {world} "
                                        f"GPU(s), {n} per GPU (columns of B; no collective on the data path)"),
                           "l2": "inputs larger than L2 (4 GiB); B re-copied before each step"},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": world * flops / (e2e_t * 1e-3) / 1e12, "unit": UNIT,
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                        "ms_per_step": [round(float(x), 3) for x in e2e_ms],
                        "ms_mean": e2e_t, "ms_median": float(np.median(e2e_ms)),
                        "value_at_median": world * flops / (float(np.median(e2e_ms)) * 1e-3) / 1e12},
                "gpu_launches": int(launches), "clocks": clk, "accuracy": acc,
                "plain_fp64": plain, "wall_s_timed": wall, "other_configs": extras,
                "kernels": {k: {"launches": v["launches"], "ms": v["ms"],
                                "tflops": (v["flops"] / (v["ms"] * 1e-3) / 1e12 if v["ms"] > 0 else 0.0)}
                            for k, v in prof.items() if v["launches"]}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def _time_calls(fn, reset, steps, warm, stream):
    import torch
    for _ in range(warm):
        reset()
        fn()
    torch.cuda.synchronize()
    ms, outs = _timed_steps(fn, reset, steps, stream)
    return float(np.mean(ms)), outs


def run_extras(stream, rank):
    """The other configurations, timed briefly on the same GPU (device-
    resident inputs, CUDA events, B reset outside the events):
      * mixed FP8 E4M3 (per-block power-of-two scales) at m = n = 16384;
      * mixed BF16 at m = n = 16384 on two more seeds (the headline's is 0);
      * mixed BF16 and FP8 at m = 32768, n = 4096, with plain FP64 beside them;
      * plain FP64 at m = n = 8192 in all 16 side/uplo/trans/diag forms and at
        m = n = 16384 in two more forms (Right/Upper/T/Unit, Left/Upper/T/NonUnit),
        alpha = 1.5;
      * the Cholesky factorisation on this TRSM, FP64, n = 16384;
      * the 4096-instance uneven batch in FP64 and FP32 (tile autotuned).
    Inputs come from the seeded device generator (same distributions as the
    headline's); accuracy is checked on sampled columns (rows for side Right)
    against the CPU oracle."""
    import torch

    import oracle
    from paper_2305_19917_gb300 import api, inputs

    out = {}
    alpha, tol = 1.5, 1e-11

    def sampled_err(side, uplo, trans, diag, A, B_orig, X):
        m, n = X.shape
        if side == 0:
            idx = [0, n // 2, n - 1]
            Bs, Xs = B_orig[:, idx], X[:, idx]
        else:
            idx = [0, m // 2, m - 1]
            Bs, Xs = B_orig[idx, :], X[idx, :]
        Ah = A.cpu().numpy()
        Xo = oracle.dtrsm(side, uplo, trans, diag, alpha, Ah, Bs.cpu().numpy())
        return float(np.linalg.norm(Xs.cpu().numpy() - Xo) / np.linalg.norm(Xo))

    def mixed_leg(name, A, B0, prec, seed_note):
        m, n = B0.shape
        B = api.colmajor_empty(m, n, torch.float64)
        reset = lambda: B.copy_(B0)  # noqa: E731
        p = api.PREC_FP8 if prec == "fp8" else api.PREC_BF16
        fn = lambda: api.trsm_mixed(0, 0, 0, 0, alpha, A, B, tol=tol, prec=p, max_iter=60,  # noqa: E731
                                    stream=stream)
        t, outs = _time_calls(fn, reset, 2, 1, stream)
        err = sampled_err(0, 0, 0, 0, A, B0, B) if rank == 0 else None
        out[name] = {"workload": f"mixed {prec.upper()} + refinement Left/Lower/N/NonUnit m={m} n={n}, "
                                 f"alpha=1.5, tol 1e-11, {seed_note}",
                     "ms_per_step": t, "tflops": float(m) * m * n / (t * 1e-3) / 1e12,
                     "refinement_steps": outs[-1][1], "status": outs[-1][0], "est_err": outs[-1][2],
                     "history_rho_levels": api.gb_mixed_history(), "fwd_err_sampled": err}
        del B

    def plain_leg(name, side, uplo, trans, diag, A, B0, steps=1):
        m, n = B0.shape
        B = api.colmajor_empty(m, n, torch.float64)
        reset = lambda: B.copy_(B0)  # noqa: E731
        fn = lambda: api.trsm(side, uplo, trans, diag, alpha, A, B, stream=stream)  # noqa: E731
        t, _ = _time_calls(fn, reset, steps, 1, stream)
        err = sampled_err(side, uplo, trans, diag, A, B0, B) if rank == 0 else None
        fl = float(m) * m * n if side == 0 else float(m) * n * n
        out[name] = {"workload": f"plain FP64 side={side} uplo={uplo} trans={trans} diag={diag} m={m} n={n}, "
                                 f"alpha=1.5, planner default plan",
                     "ms_per_step": t, "tflops": fl / (t * 1e-3) / 1e12, "fwd_err_sampled": err}
        del B

    # mixed FP8 at 16384^2 (BF16 is the headline)
    A, B0 = inputs.make_problem_device(0, 0, 0, 0, 16384, 16384, seed=0)
    mixed_leg("mixed_fp8_16384", A, B0, "fp8", "device generator seed 0")
    del A, B0
    # the headline configuration (BF16, 16384^2) on two more seeds
    for sd in (1, 2):
        A, B0 = inputs.make_problem_device(0, 0, 0, 0, 16384, 16384, seed=sd)
        mixed_leg(f"mixed_bf16_16384_seed{sd}", A, B0, "bf16", f"device generator seed {sd}")
        del A, B0
    # 32768 x 4096: BF16, FP8 and plain FP64
    A, B0 = inputs.make_problem_device(0, 0, 0, 0, 32768, 4096, seed=1)
    mixed_leg("mixed_bf16_32768x4096", A, B0, "bf16", "device generator seed 1")
    mixed_leg("mixed_fp8_32768x4096", A, B0, "fp8", "device generator seed 1")
    plain_leg("plain_fp64_32768x4096", 0, 0, 0, 0, A, B0)
    for nm in ("mixed_bf16_32768x4096", "mixed_fp8_32768x4096"):
        out[nm]["speedup_vs_plain_fp64"] = out["plain_fp64_32768x4096"]["ms_per_step"] / out[nm]["ms_per_step"]
    del A, B0
    torch.cuda.empty_cache()
    # plain FP64, all 16 forms at 8192^2
    for uplo in (0, 1):
        A, B0 = inputs.make_problem_device(0, uplo, 0, 0, 8192, 8192, seed=2 + uplo)
        for side in (0, 1):
            for trans in (0, 1):
                for diag in (0, 1):
                    plain_leg(f"plain_fp64_8192_s{side}u{uplo}t{trans}d{diag}", side, uplo, trans, diag, A, B0)
        del A, B0
    # two more forms at 16384^2
    A, B0 = inputs.make_problem_device(1, 1, 1, 1, 16384, 16384, seed=4)
    plain_leg("plain_fp64_16384_s1u1t1d1", 1, 1, 1, 1, A, B0)
    plain_leg("plain_fp64_16384_s0u1t1d0", 0, 1, 1, 0, A, B0)
    del A, B0
    torch.cuda.empty_cache()
    # Cholesky on this TRSM (FP64, lower, n = 16384): n^3/3 flops per factorisation
    nc = 16384
    S0 = inputs.make_spd_device(nc, seed=5)
    S = torch.empty_like(S0)
    reset = lambda: S.copy_(S0)  # noqa: E731
    infos = []
    t, _ = _time_calls(lambda: infos.append(api.potrf(0, S, stream=stream)), reset, 1, 1, stream)
    err = None
    if rank == 0:
        cols = [0, nc // 2, nc - 1]
        L = torch.tril(S).cpu().numpy()
        R = L @ L[cols, :].T
        Acols = S0[:, cols].cpu().numpy()
        err = float(np.linalg.norm(R - Acols) / np.linalg.norm(Acols))
    for dt, nm in ((0, "batched_fp64_4096uneven"), (1, "batched_fp32_4096uneven")):
        r = batched_measure(dt, 4096, 3, 3, stream)
        r.pop("cpu_baseline", None)
        out[nm] = r
    out["potrf_fp64_16384"] = {"workload": "Cholesky A = L L^T (gb_dpotrf, lower), n = 16384, FP64, symmetric "
                                           "diagonally dominant SPD (device generator seed 5)",
                               "ms_per_step": t, "tflops": float(nc) ** 3 / 3 / (t * 1e-3) / 1e12,
                               "info": infos[-1], "backward_err_sampled_cols": err}
    del S0, S
    torch.cuda.empty_cache()
    return out


# DRAM bytes (read + write) per launch of the residual kernel, from one ncu
# capture of the full-size workload (dram__bytes_read.sum + dram__bytes_write.sum,
# mean of the two launches of one solve).  Only valid for the kernel as it was
# when captured; drop the entry when the kernel changes.
RESIDUAL_DRAM_BYTES = {(16384, 16384, "bf16"): 20.42e9}

# FP32 ALU peak for the batched FP32 roofline: 152 SMs x 128 FFMA/clk x 2
# flop x 2.07 GHz (an FFMA probe measured 69.8 TFLOP/s).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def batched_measure(dtype, count, steps, warmup, stream, cpu_baseline_on=False):
    """The uneven batch on the current GPU: `count` problems, m log-uniform
    in [16, 512], n in [1, 256], side/uplo uniform (seeded); the kernel's tile
    shape picked by the library's autotuner (untimed), then one plan (work
    queue + CUDA graph) replayed per step; all A in one device pool, all B in
    another, so the per-step reset of B is a single copy outside the timed
    events.  Returns a dict of the measurements."""
    import torch

    import oracle
    from paper_2305_19917_gb300 import api, inputs

    dt = dtype
    tdt = torch.float64 if dt == 0 else torch.float32
    items = inputs.make_batch(count, seed=0)
    a_sizes = [it["A"].size for it in items]
    b_sizes = [it["B"].size for it in items]
    Apool = torch.empty(int(sum(a_sizes)) + 16, dtype=tdt, device="cuda")
    Bpool = torch.empty(int(sum(b_sizes)) + 16, dtype=tdt, device="cuda")
    descs, oa, ob = [], 0, 0
    for it, sa, sb in zip(items, a_sizes, b_sizes):
        m, n = it["B"].shape
        k = it["A"].shape[0]
        Apool[oa:oa + sa].copy_(torch.as_tensor(np.asfortranarray(it["A"]).ravel(order="F")).to(tdt))
        Bpool[ob:ob + sb].copy_(torch.as_tensor(np.asfortranarray(it["B"]).ravel(order="F")).to(tdt))
        descs.append(dict(side=it["side"], uplo=it["uplo"], trans=it["trans"], diag=it["diag"], m=m, n=n,
                          alpha=it["alpha"], A_ptr=Apool.data_ptr() + oa * Apool.element_size(), lda=k,
                          B_ptr=Bpool.data_ptr() + ob * Bpool.element_size(), ldb=m))
        oa += sa
        ob += sb
    B0 = Bpool.clone()
    tile, tile_ms = api.gb_batched_autotune(dt, descs, reps=3, stream=stream.cuda_stream)
    plan = api.BatchedPlan(dt, descs, stream.cuda_stream, tile=tile)
    info = plan.info()
    flops = info["flops"]
    esz = Apool.element_size()

    def reset():
        Bpool.copy_(B0)

    def solve():
        plan.run(stream.cuda_stream)

    for _ in range(max(3, warmup)):
        reset()
        solve()
    torch.cuda.synchronize()
    api.gb_profile_enable(1)
    l0 = api.gb_kernel_launches()
    ms, _ = _timed_steps(solve, reset, steps, stream)
    launches = api.gb_kernel_launches() - l0
    prof = api.gb_profile_read(api.KERNEL_KINDS.index("batched"))
    api.gb_profile_enable(0)
    ms_step = float(np.mean(ms))
    errs = []
    for idx in range(0, len(items), max(1, len(items) // 32)):
        it = items[idx]
        off = int(sum(b_sizes[:idx]))
        X = Bpool[off:off + b_sizes[idx]].double().cpu().numpy().reshape(it["B"].shape, order="F")
        Xo = oracle.dtrsm(it["side"], it["uplo"], it["trans"], it["diag"], it["alpha"], it["A"], it["B"])
        errs.append(float(np.linalg.norm(X - Xo) / max(np.linalg.norm(Xo), 1e-300)))
    # e2e: host pools in pinned memory, copied in and X copied out each step
    A_pin = Apool.cpu().pin_memory()
    B_pin = B0.cpu().pin_memory()
    X_pin = torch.empty_like(B_pin).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    Apool.copy_(A_pin, non_blocking=True)
    Bpool.copy_(B_pin, non_blocking=True)
    solve()
    X_pin.copy_(Bpool, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    peak = FP64_PEAK_TFLOPS if dt == 0 else FP32_PEAK_TFLOPS
    achieved = prof["flops"] / (prof["ms"] * 1e-3) / 1e12 if prof["ms"] > 0 else 0.0
    hbm = prof["bytes"] / (prof["ms"] * 1e-3) / 1e9 if prof["ms"] > 0 else 0.0
    cpu = None
    if cpu_baseline_on:
        t0 = time.perf_counter()
        sample = items[: max(1, len(items) // 16)]
        fl = 0.0
        for it in sample:
            oracle.dtrsm(it["side"], it["uplo"], it["trans"], it["diag"], it["alpha"], it["A"], it["B"])
            k = it["A"].shape[0]
            fl += float(k) * k * (it["B"].size // k)
        dtc = time.perf_counter() - t0
        cpu = {"value": fl / dtc / 1e12, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"first {len(sample)} of the {len(items)} problems, FP64 oracle, {dtc:.1f} s"}
    out = {"workload": f"batched uneven TRSM ({'FP64' if dt == 0 else 'FP32'}): {len(items)} problems, m log-uniform "
                       f"[16,512], n uniform [1,256], side/uplo uniform, seed 0; one persistent launch (device work "
                       f"queue, CUDA graph)",
           "ms_per_step": ms_step, "tflops": flops / (ms_step * 1e-3) / 1e12, "units": info["units"],
           "grid": info["grid"], "tile": tile, "tile_autotune_ms": tile_ms, "launches": int(launches),
           "roofline": {"kernel": "batched", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                        "frac": achieved / peak, "traffic": None,
                        "peak_source": "derived from SM count x FMA units x 2.07 GHz",
                        "hbm_gbs": hbm, "hbm_frac": hbm / MEASURED_PEAKS.get("hbm_gbs", 6797.2),
                        "launches": prof["launches"], "ms_total": prof["ms"]},
           "e2e": {"value": flops / (e2e_ms * 1e-3) / 1e12, "unit": UNIT,
                   "h2d_bytes_per_step": int((Apool.numel() + Bpool.numel()) * esz),
                   "d2h_bytes_per_step": int(Bpool.numel() * esz)},
           "cpu_baseline": cpu, "fwd_err_max_sampled": max(errs), "instances_checked": len(errs),
           "pool_mb": (Apool.numel() + Bpool.numel()) * esz / 1e6}
    plan.close()
    return out


def run_batched(args):
    """--path batched: the uneven batch as the timed step."""
    import torch

    from paper_2305_19917_gb300 import api

    rank, world, local = dist_env()
    torch.cuda.set_device(local if world > 1 else 0)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    api.lib()
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(dev)
    clocks.start()
    r = batched_measure(0 if args.dtype == "f64" else 1, args.count, args.steps, args.warmup, stream,
                        cpu_baseline_on=(not args.no_cpu_baseline and world == 1))
    clk = clocks.stop()
    ms_step = r["ms_per_step"]
    if world > 1:
        from paper_2305_19917_gb300 import dist as gdist
        ms_step = gdist.max_over_ranks(ms_step, device="cuda")
    value = world * r["tflops"] * r["ms_per_step"] / ms_step
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
                "config": {"workload": r["workload"], "units": r["units"], "grid": r["grid"], "tile": r["tile"],
                           "tile_autotune_ms": r["tile_autotune_ms"],
                           "l2": f"B reset by one copy before each step; A+B pools exceed L2 ({r['pool_mb']:.0f} MB)"},
                "roofline": r["roofline"], "cpu_baseline": r["cpu_baseline"], "e2e": r["e2e"],
                "gpu_launches": r["launches"], "clocks": clk,
                "accuracy": {"fwd_err_max_sampled": r["fwd_err_max_sampled"],
                             "instances_checked": r["instances_checked"]}}
        print(json.dumps(line), flush=True)
    return 0


def run_potrf(args):
    """--path potrf: the Cholesky factorisation on this TRSM (gb_dpotrf,
    FP64, lower) of an n x n symmetric diagonally dominant SPD matrix as the
    timed step (A re-copied from a pristine device copy before each step,
    outside the events); TFLOP/s of n^3/3."""
    import torch

    from paper_2305_19917_gb300 import api, inputs

    torch.cuda.set_device(0)
    api.lib()
    n = args.n
    stream = torch.cuda.current_stream()
    S0 = inputs.make_spd_device(n, seed=5)
    S = torch.empty_like(S0)
    infos = []
    t, _ = _time_calls(lambda: infos.append(api.potrf(0, S, stream=stream)), lambda: S.copy_(S0), args.steps,
                       max(1, args.warmup), stream)
    cols = [0, n // 2, n - 1]
    L = torch.tril(S).cpu().numpy()
    err = float(np.linalg.norm(L @ L[cols, :].T - S0[:, cols].cpu().numpy()) / np.linalg.norm(S0[:, cols].cpu().numpy()))
    line = {"metric": "Cholesky TFLOP/s (n^3/3) on this TRSM", "value": float(n) ** 3 / 3 / (t * 1e-3) / 1e12,
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"gb_dpotrf lower, n = {n}, symmetric diagonally dominant SPD (device seed 5)"},
            "accuracy": {"info": infos[-1], "backward_err_sampled_cols": err}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.path == "batched":
        return run_batched(args)
    if args.path == "potrf":
        return run_potrf(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
