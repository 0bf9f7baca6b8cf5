"""Learned cost model: training / inference driver for the library's CUDA MLP
kernels, plus the plan-choice policies it is compared with.

The network maps the 17 plan features of ``gb_plan_features`` to the log of
the measured solve time.  It replaces the paper's analytical performance
models (Section V: ``Comp(i) = r(i) TS(i) + sum r(j) gemm(j)`` for the
recursive model and its iterative / blocked counterparts, with the stop rule
``2 TS(i+1) < TS(i)``).  Those models, evaluated with task times measured on
the GPU (PaperAnalyticPolicy), are "the method without the network" that it
is compared with, beside a fitted-rates variant (AnalyticPolicy) and a
fixed plan.  The same network also predicts the mixed-precision solves, so
the planner chooses the precision (plain FP64, BF16- or FP8-mixed, and the
mixed solve's leaf order) for a request of FP64-level accuracy.

All arithmetic of training and inference runs in the CUDA kernels
(gb_mlp_forward / backward / loss / adam); torch only provides device
buffers.
"""
import json
import os
import struct

import numpy as np

from . import api

HIDDEN = 64


def features(rows):
    """Feature matrix (float32, n x 17) of timing rows (dicts with dtype,
    side, uplo, trans, m, n, driver, nb, depth)."""
    return np.array([api.gb_plan_features(r["dtype"], r["side"], r["uplo"], r["trans"], r["m"], r["n"],
                                          dict(driver=r["driver"], nb=r["nb"], depth=r["depth"]))
                     for r in rows], dtype=np.float32)


class MLP:
    """3 x 64 GELU network trained with the library's CUDA kernels."""

    def __init__(self, in_dim=api.N_FEATURES, seed=0, device="cuda"):
        import torch
        self.D = in_dim
        self.np = api.gb_mlp_param_count(in_dim)
        rng = np.random.default_rng(seed)
        p = np.zeros(self.np, dtype=np.float32)
        off = 0
        for fan_in, fan_out in ((in_dim, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN)):
            p[off:off + fan_in * fan_out] = rng.normal(0, np.sqrt(2.0 / fan_in), fan_in * fan_out)
            off += fan_in * fan_out + fan_out
        p[off:off + HIDDEN] = rng.normal(0, np.sqrt(1.0 / HIDDEN), HIDDEN)
        self.dev = device
        self.params = torch.as_tensor(p, device=device)
        self.mean, self.scale = 0.0, 1.0

    def _buf(self, n, cols=1):
        import torch
        return torch.zeros((n, cols) if cols > 1 else n, dtype=torch.float32, device=self.dev)

    def predict_norm(self, X):
        import torch
        Xd = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float32), device=self.dev)
        Y = self._buf(len(X))
        st = api.gb_mlp_forward(self.params.data_ptr(), self.D, Xd.data_ptr(), len(X), Y.data_ptr(), 0, 0)
        assert st == 0, st
        torch.cuda.synchronize()
        return Y.cpu().numpy()

    def predict_log_ms(self, X):
        return self.predict_norm(X) * self.scale + self.mean

    def loss_and_grad(self, X, T):
        """(loss, gradient) of the MSE on a batch, via the CUDA kernels."""
        import torch
        n = len(X)
        Xd = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float32), device=self.dev)
        Td = torch.as_tensor(np.ascontiguousarray(T, dtype=np.float32), device=self.dev)
        Y, Z, dY = self._buf(n), self._buf(n, 3 * HIDDEN), self._buf(n)
        G = torch.zeros(self.np, dtype=torch.float32, device=self.dev)
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        assert api.gb_mlp_forward(self.params.data_ptr(), self.D, Xd.data_ptr(), n, Y.data_ptr(), Z.data_ptr()) == 0
        assert api.gb_mlp_loss(Y.data_ptr(), Td.data_ptr(), n, dY.data_ptr(), loss.data_ptr()) == 0
        assert api.gb_mlp_backward(self.params.data_ptr(), self.D, Xd.data_ptr(), Z.data_ptr(), dY.data_ptr(), n,
                                   G.data_ptr()) == 0
        torch.cuda.synchronize()
        return float(loss.item()), G.cpu().numpy()

    def fit(self, X, logt, epochs=400, batch=512, lr=2e-3, seed=0, verbose=False):
        """Adam on mean squared error of the normalised log time."""
        import torch
        X = np.ascontiguousarray(X, dtype=np.float32)
        logt = np.asarray(logt, dtype=np.float64)
        self.mean = float(logt.mean())
        self.scale = float(logt.std() or 1.0)
        T = ((logt - self.mean) / self.scale).astype(np.float32)
        n = len(X)
        Xd = torch.as_tensor(X, device=self.dev)
        Td = torch.as_tensor(T, device=self.dev)
        M = torch.zeros(self.np, dtype=torch.float32, device=self.dev)
        V = torch.zeros_like(M)
        G = torch.zeros_like(M)
        Yb, Zb, dYb = self._buf(batch), self._buf(batch, 3 * HIDDEN), self._buf(batch)
        rng = np.random.default_rng(seed)
        step = 0
        hist = []
        for ep in range(epochs):
            perm = torch.as_tensor(rng.permutation(n), device=self.dev)
            lr_e = lr * (0.5 * (1 + np.cos(np.pi * ep / epochs)))  # cosine decay
            for s0 in range(0, n, batch):
                idx = perm[s0:s0 + batch]
                nb = len(idx)
                xb = Xd[idx].contiguous()
                tb = Td[idx].contiguous()
                G.zero_()
                api.gb_mlp_forward(self.params.data_ptr(), self.D, xb.data_ptr(), nb, Yb.data_ptr(), Zb.data_ptr())
                api.gb_mlp_loss(Yb.data_ptr(), tb.data_ptr(), nb, dYb.data_ptr(), 0)
                api.gb_mlp_backward(self.params.data_ptr(), self.D, xb.data_ptr(), Zb.data_ptr(), dYb.data_ptr(),
                                    nb, G.data_ptr())
                step += 1
                api.gb_mlp_adam(self.params.data_ptr(), G.data_ptr(), M.data_ptr(), V.data_ptr(), self.np,
                                float(lr_e), 0.9, 0.999, 1e-8, step)
            if verbose and (ep % 50 == 0 or ep == epochs - 1):
                pred = self.predict_norm(X)
                hist.append(float(np.mean((pred - T) ** 2)))
                print(f"epoch {ep} mse {hist[-1]:.4f}")
        torch.cuda.synchronize()
        return hist

    def save(self, path):
        p = self.params.cpu().numpy().astype(np.float32)
        with open(path, "wb") as f:
            f.write(b"GBMLP001")
            f.write(struct.pack("<iii", self.D, HIDDEN, p.size))
            f.write(struct.pack("<ff", self.mean, self.scale))
            f.write(p.tobytes())

    @classmethod
    def load(cls, path, device="cuda"):
        import torch
        with open(path, "rb") as f:
            assert f.read(8) == b"GBMLP001"
            D, hid, npar = struct.unpack("<iii", f.read(12))
            mean, scale = struct.unpack("<ff", f.read(8))
            p = np.frombuffer(f.read(4 * npar), dtype=np.float32)
        m = cls(D, device=device)
        m.params = torch.as_tensor(p.copy(), device=device)
        m.mean, m.scale = mean, scale
        return m


# ---- timing database ----------------------------------------------------------

def load_db(path):
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line:
                rows.append(json.loads(line))
    return rows


def shape_key(r):
    return (r["dtype"], r["side"], r["uplo"], r["trans"], r["m"], r["n"])


def group_by_shape(rows):
    g = {}
    for r in rows:
        g.setdefault(shape_key(r), []).append(r)
    return g


def split_shapes(rows, frac=0.8, seed=0):
    keys = sorted(group_by_shape(rows))
    rng = np.random.default_rng(seed)
    rng.shuffle(keys)
    cut = int(round(frac * len(keys)))
    train = set(keys[:cut])
    return [r for r in rows if shape_key(r) in train], [r for r in rows if shape_key(r) not in train]


# ---- policies -------------------------------------------------------------------

def plan_work(r):
    """(launches, TS flops, gemm flops) of a row's plan, from the schedule
    counts of the paper's model (gb_plan_counts)."""
    k = r["m"] if r["side"] == 0 else r["n"]
    ncols = r["n"] if r["side"] == 0 else r["m"]
    c = api.gb_plan_counts(dict(driver=r["driver"], nb=r["nb"], depth=r["depth"]), k)
    gemm_f = 2.0 * c["gemm_madds_per_col"] * ncols
    ts_f = float(k) * k * ncols - gemm_f
    # TS tasks larger than the 64-row kernel are blocked again inside
    leaf_ts = c["n_diag"] * max(1, int(np.ceil((k / max(1, c["n_diag"])) / 64)))
    return c["n_diag"] + c["n_gemm"] + 2 * leaf_ts, ts_f, gemm_f


class AnalyticPolicy:
    """Section V-style model: t = a * launches + TS flops / r_ts + gemm
    flops / r_gemm per dtype, coefficients by non-negative least squares."""

    def fit(self, rows):
        from scipy.optimize import nnls
        self.coef = {}
        for dt in sorted({r["dtype"] for r in rows}):
            sub = [r for r in rows if r["dtype"] == dt]
            A = np.array([plan_work(r) for r in sub], dtype=np.float64)
            t = np.array([r["ms"] for r in sub])
            scale = A.max(axis=0)
            scale[scale == 0] = 1
            x, _ = nnls(A / scale / t[:, None], np.ones(len(t)))  # relative error
            self.coef[dt] = x / scale
        return self

    def predict(self, r):
        return float(np.dot(self.coef[r["dtype"]], plan_work(r)))


class PaperAnalyticPolicy:
    """The paper's analytic computation models (Section V) with measured task
    times, as the planner without the network:

      recursive (V-A):  Comp(i) = r(i) TS(i) + sum_{j<i} r(j) gemm(j)
      iterative (V-B):  Comp(i) = r(i) TS(i) + sum_{j=0}^{r(i)-2} gemm(i, j)
      blocked   (V-C):  Comp(i) = r(i) TS(i) + ((r(i) - 1) r(i) / 2) gemm(i)

    with r(i) = 2^i (Eq. 1) for the recursive model and r = ceil(k / nb) for
    the fixed-granularity ones.  TS(order) and gemm(M, K) are the times the
    autotuner measured for the shape (component database): TS as one
    diagonal task of that order (the library's blocked solve with nb <= 64,
    i.e. the leaf method every plan uses), gemm(j) as one update of
    ceil(k/2^(j+1)) rows x ncols x ceil(k/2^(j+1)), gemm(i) as one nb x nb
    block, gemm(i, j) as block row j+1 against the j+1 solved blocks (left
    looking, K = (j+1) nb; times between measured K interpolated linearly).
    mode "argmin": the candidate with the least Comp among the plans the
    models describe (recursive with nb = 64 leaves' inner blocking, blocked
    and iterative with every nb).  mode "stop_rule": the recursive model with
    the refinement level of Section V-A's rule -- refine from i to i+1 only
    while 2 TS(i+1) < TS(i)."""

    def __init__(self, components, mode="argmin"):
        self.comp = components
        self.mode = mode

    @staticmethod
    def _k_ncols(r):
        return (r["m"], r["n"]) if r["side"] == 0 else (r["n"], r["m"])

    def _ts(self, c, order):
        return c["ts"][str(order)]

    def _gemm(self, c, M, K):
        key = f"{M},{K}"
        if key in c["gemm"]:
            return c["gemm"][key]
        # interpolate in K among the measured (M, K') of the same M
        pts = sorted((int(k2.split(",")[1]), v) for k2, v in c["gemm"].items() if int(k2.split(",")[0]) == M)
        ks = np.array([p[0] for p in pts], dtype=float)
        ts = np.array([p[1] for p in pts], dtype=float)
        return float(np.interp(K, ks, ts))

    def comp_plan(self, r):
        """Comp of a candidate row's plan, or inf for plans the models do not
        describe."""
        c = self.comp.get(shape_key(r))
        if c is None:
            return float("inf")
        k, _ = self._k_ncols(r)
        nb, d = r["nb"], r["depth"]
        if r["driver"] == 1:  # recursive
            if nb != 64:
                return float("inf")
            t = 2 ** d * self._ts(c, max(1, -(-k // 2 ** d)))
            for j in range(d):
                h = -(-k // 2 ** (j + 1))
                if h >= k:
                    continue
                t += 2 ** j * self._gemm(c, h, h)
            return t
        rr = -(-k // nb)
        if rr <= 1:
            return self._ts(c, k)
        ts = self._ts(c, nb)
        if r["driver"] == 0:  # blocked
            return rr * ts + (rr - 1) * rr / 2 * self._gemm(c, nb, nb)
        return rr * ts + sum(self._gemm(c, nb, (j + 1) * nb) for j in range(rr - 1))  # iterative

    def stop_rule_depth(self, r):
        c = self.comp[shape_key(r)]
        k, _ = self._k_ncols(r)
        i = 0
        while i < 6 and 2 * self._ts(c, max(1, -(-k // 2 ** (i + 1)))) < self._ts(c, max(1, -(-k // 2 ** i))):
            i += 1
        return i

    def choose(self, cand):
        if self.mode == "stop_rule":
            d = self.stop_rule_depth(cand[0])
            want = (1, 64, d) if d >= 1 else (0, 64, 0)
            for r in cand:
                if (r["driver"], r["nb"], r["depth"]) == want:
                    return r
            return cand[0]
        return min(cand, key=self.comp_plan)


def load_components(path):
    out = {}
    if not os.path.exists(path):
        return out
    with open(path) as f:
        for line in f:
            if line.strip():
                r = json.loads(line)
                out[shape_key(r)] = r
    return out


def regret(rows, choose):
    """Per held-out shape: t_chosen / t_best - 1, where choose(candidate
    rows of one shape) returns the chosen row."""
    out = []
    for key, cand in group_by_shape(rows).items():
        best = min(c["ms"] for c in cand)
        out.append(choose(cand)["ms"] / best - 1.0)
    return np.array(out)


def evaluate(train_rows, test_rows, model=None, epochs=400, verbose=False, components=None):
    """Fit the network (unless given) and the fitted-rates policy on the
    training shapes; report the regret of each policy on the held-out shapes,
    including the paper's analytic models with measured task times
    (components: the component database; shapes without components are
    left out of those two)."""
    if model is None:
        model = MLP()
        model.fit(features(train_rows), np.log([r["ms"] for r in train_rows]), epochs=epochs, verbose=verbose)
    Xt = features(test_rows)
    pred = model.predict_log_ms(Xt)
    for r, p in zip(test_rows, pred):
        r["_pred"] = float(p)
    ana = AnalyticPolicy().fit(train_rows)
    reg_mlp = regret(test_rows, lambda c: min(c, key=lambda r: r["_pred"]))
    reg_ana = regret(test_rows, lambda c: min(c, key=ana.predict))

    def fixed128(c):
        same = [r for r in c if r["nb"] == 128 and r["driver"] == 1]
        k = c[0]["m"] if c[0]["side"] == 0 else c[0]["n"]
        want = max(1, min(6, int(np.log2(max(k, 256) / 256))))
        return min(same, key=lambda r: abs(r["depth"] - want)) if same else c[0]
    reg_fix = regret(test_rows, fixed128)
    stats = lambda a: dict(mean=float(np.mean(a)), p90=float(np.percentile(a, 90)), max=float(np.max(a)))  # noqa
    out = dict(mlp=stats(reg_mlp), analytic=stats(reg_ana), fixed_nb128=stats(reg_fix),
               shapes=len(group_by_shape(test_rows)))
    if components:
        covered = [r for r in test_rows if shape_key(r) in components]
        if covered:
            pa = PaperAnalyticPolicy(components, "argmin")
            ps = PaperAnalyticPolicy(components, "stop_rule")
            out["paper_comp_argmin"] = stats(regret(covered, pa.choose))
            out["paper_stop_rule"] = stats(regret(covered, ps.choose))
            out["mlp_on_covered"] = stats(regret(covered, lambda c: min(c, key=lambda r: r["_pred"])))
            out["covered_shapes"] = len(group_by_shape(covered))
    return model, out


# ---- the precision decision ------------------------------------------------------

PREC_DTYPE = {-1: 0, 0: 2, 1: 3}  # plain FP64 / BF16-mixed / FP8-mixed -> feature dtype


def prec_feature_rows(prec_rows):
    """Precision-database rows as rows of the network's feature space."""
    return [dict(r, dtype=PREC_DTYPE[r["prec"]]) for r in prec_rows]


def prec_key(r):
    return (r["side"], r["uplo"], r["trans"], r["m"], r["n"])


def split_prec_shapes(rows, frac=0.8, seed=0):
    keys = sorted({prec_key(r) for r in rows})
    rng = np.random.default_rng(seed)
    rng.shuffle(keys)
    train = set(keys[:int(round(frac * len(keys)))])
    return [r for r in rows if prec_key(r) in train], [r for r in rows if prec_key(r) not in train]


def feasible(r, tol=1e-10):
    """Reached FP64-level accuracy: the plain path always; a mixed run when it
    converged and its distance from the plain FP64 solution is <= tol."""
    return r["prec"] < 0 or (r["status"] == 0 and r["err_vs_fp64"] <= tol)


def precision_regret(test_rows, choose):
    """Per held-out shape: t(chosen) / t(best feasible) - 1; a chosen mixed
    run that did not reach the accuracy is charged its time plus the plain
    FP64 solve that a caller then falls back to."""
    out = []
    groups = {}
    for r in test_rows:
        groups.setdefault(prec_key(r), []).append(r)
    for cand in groups.values():
        plain = [r for r in cand if r["prec"] < 0][0]
        best = min(r["ms"] for r in cand if feasible(r))
        ch = choose(cand)
        t = ch["ms"] if feasible(ch) else ch["ms"] + plain["ms"]
        out.append(t / best - 1.0)
    return np.array(out)


def evaluate_precision(plan_rows, prec_rows, epochs=400, seed=0, prec_weight=8):
    """Train the network on the plan database plus the training shapes of the
    precision database (their rows repeated prec_weight times, they are few)
    and evaluate its precision choice on the held-out precision shapes against
    exhaustive search, always-plain-FP64 and always-BF16 (leaf 1024)."""
    tr, te = split_prec_shapes(prec_rows, 0.8, seed)
    train = list(plan_rows) + prec_feature_rows(tr) * prec_weight
    model = MLP()
    model.fit(features(train), np.log([r["ms"] for r in train]), epochs=epochs)
    ft = prec_feature_rows(te)
    pred = model.predict_log_ms(features(ft))
    for r, p in zip(te, pred):
        r["_pred"] = float(p)
    stats = lambda a: dict(mean=float(np.mean(a)), p90=float(np.percentile(a, 90)), max=float(np.max(a)))  # noqa
    reg_mlp = precision_regret(te, lambda c: min(c, key=lambda r: r["_pred"]))
    reg_plain = precision_regret(te, lambda c: [r for r in c if r["prec"] < 0][0])
    reg_bf16 = precision_regret(te, lambda c: [r for r in c if r["prec"] == 0 and r["leaf"] == 1024][0])
    return model, dict(mlp=stats(reg_mlp), always_plain_fp64=stats(reg_plain), always_bf16_1024=stats(reg_bf16),
                       shapes=len({prec_key(r) for r in te}),
                       mixed_infeasible=int(sum(1 for r in prec_rows if not feasible(r))))


def train_default_model(out=None, epochs=800, prec_weight=8):
    """The committed planner network: trained on every row of the plan and
    precision databases (on the GPU, by the library's kernels) and saved."""
    rows = load_db(DEFAULT_DB)
    if os.path.exists(DEFAULT_PREC_DB):
        rows += prec_feature_rows(load_db(DEFAULT_PREC_DB)) * prec_weight
    model = MLP()
    model.fit(features(rows), np.log([r["ms"] for r in rows]), epochs=epochs)
    model.save(out or DEFAULT_MODEL)
    return model


DEFAULT_DB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "timings_gb300.jsonl")
DEFAULT_MODEL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "costmodel_gb300.bin")
DEFAULT_COMP_DB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "components_gb300.jsonl")
DEFAULT_PREC_DB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "precision_gb300.jsonl")


def main(argv=None):
    import argparse
    p = argparse.ArgumentParser(description="train / evaluate the planner network")
    p.add_argument("--train", action="store_true", help="train on every row and save the model")
    p.add_argument("--out", default=None)
    p.add_argument("--epochs", type=int, default=800)
    p.add_argument("--evaluate", action="store_true", help="held-out regret of every policy")
    a = p.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    api.lib()
    if a.evaluate:
        rows = load_db(DEFAULT_DB)
        tr, te = split_shapes(rows, 0.8, seed=0)
        _, st = evaluate(tr, te, epochs=800, components=load_components(DEFAULT_COMP_DB))
        print(json.dumps({"plans": st}))
        if os.path.exists(DEFAULT_PREC_DB):
            _, sp = evaluate_precision(rows, load_db(DEFAULT_PREC_DB))
            print(json.dumps({"precision": sp}))
    if a.train:
        train_default_model(a.out, a.epochs)
        print("saved", a.out or DEFAULT_MODEL)
    return 0


if __name__ == "__main__":
    import sys
    sys.exit(main())
