"""Autotuner data collection: time every candidate plan on sampled shapes.

    python -m paper_2305_19917_gb300.autotune --shapes 420 --out DB.jsonl
    python -m paper_2305_19917_gb300.autotune --kind components --shapes 420 --out COMP.jsonl
    python -m paper_2305_19917_gb300.autotune --kind precision --shapes 150 --seed 1 --out PREC.jsonl

``--kind components`` measures, for the same shapes, the task times of the
paper's analytic model (Section V): TS(order) of every leaf / block order it
needs and gemm(M, K) of every update shape (see time_components).
``--kind precision`` times, on FP64 shapes up to k^2 ncols = 4e11, the plain
FP64 solve against the mixed BF16 / FP8 candidates (time_precision).

Shapes: m and n log-uniform in [64, 32768], dtype FP64 or FP32, side, uplo,
trans uniform, diag NonUnit; a shape is redrawn while m^2 n (k^2 ncols)
exceeds the per-dtype work cap that keeps one solve within a few ms (the
candidate sweep times 48 plans x 3 repetitions per shape).  Inputs are
generated on the GPU with a seeded generator (diagonal U[1,2), strict
triangle U(-1,1)/k, B ~ N(0,1)); only times are recorded.  Each shape
appends 48 JSON rows (dtype, side, uplo, trans, m, n, driver, nb, depth,
ms) to the database; shapes already in it are skipped, so an interrupted
collection resumes where it stopped.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

from . import api

WORK_CAP = {0: 1.5e9, 1: 3.0e10}   # flops (k^2 ncols) per solve, FP64 / FP32


def sample_shapes(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        dtype = int(rng.integers(0, 2))
        m = int(round(np.exp(rng.uniform(np.log(64), np.log(32768)))))
        n = int(round(np.exp(rng.uniform(np.log(64), np.log(32768)))))
        side, uplo, trans = (int(x) for x in rng.integers(0, 2, 3))
        k, ncols = (m, n) if side == 0 else (n, m)
        if float(k) * k * ncols > WORK_CAP[dtype]:
            continue
        out.append(dict(dtype=dtype, side=side, uplo=uplo, trans=trans, m=m, n=n))
    return out


def make_inputs(s, seed):
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    tdt = torch.float64 if s["dtype"] == 0 else torch.float32
    k = s["m"] if s["side"] == 0 else s["n"]
    A = (torch.rand((k, k), generator=g, device="cuda", dtype=tdt) * 2 - 1) / k
    A.diagonal().copy_(torch.rand(k, generator=g, device="cuda", dtype=tdt) + 1)
    A = A.t().contiguous().t()  # column-major view
    B = torch.randn((s["n"], s["m"]), generator=g, device="cuda", dtype=tdt).t()
    return A, B


def time_shape(s, cands, seed, reps=3):
    import torch
    A, B = make_inputs(s, seed)
    k = A.shape[0]
    ms = api.gb_autotune_time(s["dtype"], s["side"], s["uplo"], s["trans"], 0, s["m"], s["n"], 1.0,
                              A.data_ptr(), k, B.data_ptr(), s["m"], cands, reps,
                              torch.cuda.current_stream().cuda_stream)
    return [dict(s, driver=c["driver"], nb=c["nb"], depth=c["depth"], ms=float(t)) for c, t in zip(cands, ms)]


def collect(out, count, seed=0, budget_s=1e9, verbose=True):
    import torch
    torch.cuda.set_device(0)
    api.lib()
    done = set()
    if os.path.exists(out):
        with open(out) as f:
            for line in f:
                if line.strip():
                    r = json.loads(line)
                    done.add((r["dtype"], r["side"], r["uplo"], r["trans"], r["m"], r["n"]))
    cands = api.gb_plan_candidates(0)
    shapes = sample_shapes(count, seed)
    t0 = time.time()
    with open(out, "a") as f:
        for i, s in enumerate(shapes):
            key = (s["dtype"], s["side"], s["uplo"], s["trans"], s["m"], s["n"])
            if key in done:
                continue
            if time.time() - t0 > budget_s:
                break
            rows = time_shape(s, cands, seed * 100003 + i)
            for r in rows:
                f.write(json.dumps(r) + "\n")
            f.flush()
            done.add(key)
            if verbose and i % 20 == 0:
                print(f"[{i}/{len(shapes)}] {s} best {min(r['ms'] for r in rows):.3f} ms "
                      f"({time.time() - t0:.0f} s)", flush=True)
    return out


# ---- component timings of the paper's analytic model (Section V) ---------------

COMP_NBS = (16, 32, 64, 128, 256, 512)
COMP_DEPTHS = 6


def _time_events(fn, reps=3):
    """Median of `reps` CUDA-event timings of fn() (one untimed call first)."""
    import torch
    st = torch.cuda.current_stream()
    fn()
    out = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return float(np.median(out))


def component_orders(k):
    """Orders of the TS tasks the analytic model needs for an order-k
    triangle: the recursive model's leaves ceil(k / 2^i), i = 0..6, and the
    blocked / iterative block sizes nb <= k."""
    o = {max(1, -(-k // (2 ** i))) for i in range(COMP_DEPTHS + 1)}
    o |= {nb for nb in COMP_NBS if nb <= k}
    return sorted(o)


def component_gemms(k):
    """(M, K) shapes of the gemm tasks the analytic model needs: recursive
    level j, M = K = ceil(k / 2^(j+1)) (j = 0..5); blocked, one nb x nb
    block; iterative, block row of nb against c solved blocks, K = c nb for
    c in a doubling grid up to r - 1 (r = ceil(k / nb)) -- times in between
    are interpolated linearly in K."""
    g = set()
    for j in range(COMP_DEPTHS):
        h = -(-k // (2 ** (j + 1)))
        if h >= 1 and h < k:
            g.add((h, h))
    for nb in COMP_NBS:
        if nb >= k:
            continue
        r = -(-k // nb)
        c = 1
        while c < r - 1:
            g.add((nb, c * nb))
            c *= 2
        g.add((nb, (r - 1) * nb))
    return sorted(g)


def time_components(s, seed, reps=3):
    """Measured TS(order) and gemm(M, K) times (ms) for one shape: TS as the
    library's blocked solve (nb = min(64, order)) of an order x ncols
    sub-problem in the shape's own form, gemm as gb_gemm_update with N = ncols."""
    import torch
    A, B = make_inputs(s, seed)
    k = A.shape[0]
    ncols = s["n"] if s["side"] == 0 else s["m"]
    dt = torch.float64 if s["dtype"] == 0 else torch.float32
    stream = torch.cuda.current_stream().cuda_stream
    ts = {}
    for o in component_orders(k):
        Ao = A[:o, :o]
        Bo = B[:o, :] if s["side"] == 0 else B[:, :o]
        mo, no = (o, ncols) if s["side"] == 0 else (ncols, o)
        plan = dict(driver=api.DRIVER_BLOCKED, nb=min(64, max(16, 1 << (max(o, 1) - 1).bit_length()))
                    if o < 64 else 64, depth=0)
        ms = api.gb_autotune_time(s["dtype"], s["side"], s["uplo"], s["trans"], 0, mo, no, 1.0, Ao.data_ptr(),
                                  k, Bo.data_ptr(), s["m"], [plan], reps, stream)
        ts[str(o)] = ms[0]
    gm = {}
    for M, K in component_gemms(k):
        Ag = torch.randn((K, M), device="cuda", dtype=dt).t()
        Bg = torch.randn((ncols, K), device="cuda", dtype=dt).t()
        Cg = torch.randn((ncols, M), device="cuda", dtype=dt).t()
        fn = lambda: api.gb_gemm_update(s["dtype"], M, ncols, K, Ag.data_ptr(), M, Bg.data_ptr(), K,  # noqa: E731
                                        Cg.data_ptr(), M, 1.0, stream)
        gm[f"{M},{K}"] = _time_events(fn, reps)
    return dict(s, ts=ts, gemm=gm)


def collect_components(out, count=420, seed=0, verbose=True):
    """Component timings for the plan database's shapes (same sampling)."""
    import torch
    torch.cuda.set_device(0)
    api.lib()
    done = set()
    if os.path.exists(out):
        with open(out) as f:
            for line in f:
                if line.strip():
                    r = json.loads(line)
                    done.add((r["dtype"], r["side"], r["uplo"], r["trans"], r["m"], r["n"]))
    t0 = time.time()
    with open(out, "a") as f:
        for i, s in enumerate(sample_shapes(count, seed)):
            key = (s["dtype"], s["side"], s["uplo"], s["trans"], s["m"], s["n"])
            if key in done:
                continue
            f.write(json.dumps(time_components(s, seed * 100003 + i)) + "\n")
            f.flush()
            done.add(key)
            if verbose and i % 50 == 0:
                print(f"[components {i}/{count}] {s} ({time.time() - t0:.0f} s)", flush=True)
    return out


# ---- the precision decision: plain FP64 vs mixed BF16 / FP8 ---------------------

PREC_WORK_CAP = 4.0e11  # k^2 ncols of the plain FP64 solve (about 0.35 s)


def sample_precision_shapes(count, seed):
    """FP64-accuracy shapes for the precision decision: m and n log-uniform
    in [256, 32768], side / uplo / trans uniform, k^2 ncols <= PREC_WORK_CAP."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        m = int(round(np.exp(rng.uniform(np.log(256), np.log(32768)))))
        n = int(round(np.exp(rng.uniform(np.log(256), np.log(32768)))))
        side, uplo, trans = (int(x) for x in rng.integers(0, 2, 3))
        k, ncols = (m, n) if side == 0 else (n, m)
        if float(k) * k * ncols > PREC_WORK_CAP:
            continue
        out.append(dict(dtype=0, side=side, uplo=uplo, trans=trans, m=m, n=n))
    return out


def time_precision(s, seed, reps=2, tol=1e-11):
    """One shape: the plain FP64 solve with the built-in default plan and
    every mixed candidate of gb_plan_mixed_candidates (gb_dtrsm_mixed_leaf),
    each timed with CUDA events; mixed rows carry their status, refinement
    steps and normwise distance from the plain FP64 solution."""
    import torch
    from . import inputs
    k = s["m"] if s["side"] == 0 else s["n"]
    A, B0 = inputs.make_problem_device(s["side"], s["uplo"], s["trans"], 0, s["m"], s["n"], seed)
    B = api.colmajor_empty(s["m"], s["n"], torch.float64)
    stream = torch.cuda.current_stream().cuda_stream
    st, plan, _ = api.gb_plan_choose(0, s["side"], s["uplo"], s["trans"], s["m"], s["n"])
    rows = []

    def plain():
        B.copy_(B0)
        api.gb_dtrsm(s["side"], s["uplo"], s["trans"], 0, s["m"], s["n"], 1.0, A.data_ptr(), k, B.data_ptr(),
                     s["m"], stream)
    t_plain = _time_events(plain, reps)
    torch.cuda.synchronize()
    Xp = B.clone()
    xn = float(torch.linalg.norm(Xp))
    rows.append(dict(s, prec=-1, leaf=0, driver=plan["driver"], nb=plan["nb"], depth=plan["depth"], ms=t_plain,
                     status=0, iters=0, err_vs_fp64=0.0))
    for prec, leaf, cp in api.gb_plan_mixed_candidates(k):
        res = {}

        def mixed():
            B.copy_(B0)
            res["r"] = api.gb_dtrsm_mixed_leaf(s["side"], s["uplo"], s["trans"], 0, s["m"], s["n"], 1.0,
                                               A.data_ptr(), k, B.data_ptr(), s["m"], tol, prec, 60, leaf, stream)
        t = _time_events(mixed, reps)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(B - Xp)) / max(xn, 1e-300)
        st_, it, _ = res["r"]
        rows.append(dict(s, prec=prec, leaf=leaf, driver=cp["driver"], nb=cp["nb"], depth=cp["depth"], ms=t,
                         status=st_, iters=it, err_vs_fp64=err))
    return rows


def collect_precision(out, count=150, seed=1, verbose=True):
    import torch
    torch.cuda.set_device(0)
    api.lib()
    done = set()
    if os.path.exists(out):
        with open(out) as f:
            for line in f:
                if line.strip():
                    r = json.loads(line)
                    done.add((r["side"], r["uplo"], r["trans"], r["m"], r["n"]))
    t0 = time.time()
    with open(out, "a") as f:
        for i, s in enumerate(sample_precision_shapes(count, seed)):
            key = (s["side"], s["uplo"], s["trans"], s["m"], s["n"])
            if key in done:
                continue
            for r in time_precision(s, seed * 100003 + i):
                f.write(json.dumps(r) + "\n")
            f.flush()
            done.add(key)
            if verbose and i % 10 == 0:
                print(f"[precision {i}/{count}] {s} ({time.time() - t0:.0f} s)", flush=True)
    return out


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--shapes", type=int, default=420)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--out", required=True)
    p.add_argument("--budget-s", type=float, default=1e9)
    p.add_argument("--kind", default="plans", choices=["plans", "components", "precision"])
    a = p.parse_args(argv)
    if a.kind == "components":
        collect_components(a.out, a.shapes, a.seed)
    elif a.kind == "precision":
        collect_precision(a.out, a.shapes, a.seed)
    else:
        collect(a.out, a.shapes, a.seed, a.budget_s)
    return 0


if __name__ == "__main__":
    sys.exit(main())
