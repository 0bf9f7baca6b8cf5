"""Learned cost model: training / inference driver for the library's CUDA MLP
kernels, plus the plan-choice policies it is judged against.

The network maps the 17 plan features of ``gb_plan_features`` to the log of
the measured solve time.  It replaces the paper's analytical performance
models (Section V: ``Comp(i) = r(i) TS(i) + sum r(j) gemm(j)`` for the
recursive model and its iterative / blocked counterparts, with the stop rule
``2 TS(i+1) < TS(i)``).  The analytic policy below keeps that structure --
time = TS work / rate_TS + gemm work / rate_gemm + launches x overhead, with
the three coefficients fitted to the same timings -- as "the method without
the network".

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


def regret(rows, choose):
    """Per held-out shape: t_chosen / t_best - 1, where choose(candidate
    rows of one shape) returns the chosen row."""
    out = []
    for key, cand in group_by_shape(rows).items():
        best = min(c["ms"] for c in cand)
        out.append(choose(cand)["ms"] / best - 1.0)
    return np.array(out)


def evaluate(train_rows, test_rows, model=None, epochs=400, verbose=False):
    """Fit the network (unless given) and the analytic policy on the training
    shapes; report the regret of each policy on the held-out shapes."""
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
    return model, dict(mlp=stats(reg_mlp), analytic=stats(reg_ana), fixed_nb128=stats(reg_fix),
                       shapes=len(group_by_shape(test_rows)))


DEFAULT_DB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "timings_gb300.jsonl")
DEFAULT_MODEL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "costmodel_gb300.bin")
