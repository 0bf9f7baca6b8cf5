"""Autotuner data collection: time every candidate plan on sampled shapes.

    python -m paper_2305_19917_gb300.autotune --shapes 420 --out DB.jsonl

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


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--shapes", type=int, default=420)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--out", required=True)
    p.add_argument("--budget-s", type=float, default=1e9)
    a = p.parse_args(argv)
    collect(a.out, a.shapes, a.seed, a.budget_s)
    return 0


if __name__ == "__main__":
    sys.exit(main())
