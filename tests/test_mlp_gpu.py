"""GPU parity of the cost-model network kernels (forward, backward, loss,
Adam) against the FP64 CPU oracle, and a short training run."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
D = 17


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2305_19917_gb300 import build
    build.build()


def _setup(n, seed):
    rng = np.random.default_rng(seed)
    P = (rng.standard_normal(oracle.mlp_param_count(D)) * 0.2).astype(np.float32)
    X = rng.standard_normal((n, D)).astype(np.float32)
    T = rng.standard_normal(n).astype(np.float32)
    return P, X, T


@pytest.mark.parametrize("n", [1, 31, 200])
def test_forward_backward_match_oracle(n):
    import torch
    from paper_2305_19917_gb300 import api
    P, X, T = _setup(n, n)
    loss_o, y_o, g_o = oracle.mlp_loss_grad(P, X, T)
    Pd, Xd, Td = (torch.as_tensor(a, device="cuda") for a in (P, X, T))
    Y = torch.zeros(n, device="cuda")
    Z = torch.zeros(n, 192, device="cuda")
    dY = torch.zeros(n, device="cuda")
    G = torch.zeros(P.size, device="cuda")
    L = torch.zeros(1, device="cuda")
    assert api.gb_mlp_forward(Pd.data_ptr(), D, Xd.data_ptr(), n, Y.data_ptr(), Z.data_ptr()) == 0
    assert api.gb_mlp_loss(Y.data_ptr(), Td.data_ptr(), n, dY.data_ptr(), L.data_ptr()) == 0
    assert api.gb_mlp_backward(Pd.data_ptr(), D, Xd.data_ptr(), Z.data_ptr(), dY.data_ptr(), n, G.data_ptr()) == 0
    torch.cuda.synchronize()
    y = Y.cpu().double().numpy()
    g = G.cpu().double().numpy()
    assert np.linalg.norm(y - y_o) <= 1e-5 * np.linalg.norm(y_o)
    assert abs(L.item() - loss_o) <= 1e-5 * abs(loss_o)
    assert np.linalg.norm(g - g_o) <= 1e-5 * np.linalg.norm(g_o)


def test_adam_matches_oracle():
    import torch
    from paper_2305_19917_gb300 import api
    rng = np.random.default_rng(5)
    npar = 1000
    p = rng.standard_normal(npar).astype(np.float32)
    gs = [rng.standard_normal(npar).astype(np.float32) for _ in range(3)]
    pd, md, vd = torch.as_tensor(p, device="cuda"), torch.zeros(npar, device="cuda"), torch.zeros(npar, device="cuda")
    po, mo, vo = p.astype(np.float64), np.zeros(npar), np.zeros(npar)
    for step, g in enumerate(gs, start=1):
        gd = torch.as_tensor(g, device="cuda")
        assert api.gb_mlp_adam(pd.data_ptr(), gd.data_ptr(), md.data_ptr(), vd.data_ptr(), npar, 1e-2, 0.9, 0.999,
                               1e-8, step) == 0
        oracle.adam_step(po, g.astype(np.float64), mo, vo, 1e-2, 0.9, 0.999, 1e-8, step)
    torch.cuda.synchronize()
    assert np.max(np.abs(pd.cpu().double().numpy() - po)) <= 1e-5


def test_training_reduces_loss():
    from paper_2305_19917_gb300 import costmodel
    rng = np.random.default_rng(0)
    X = rng.uniform(0, 1, (2000, D)).astype(np.float32)
    logt = 3 * X[:, 0] + 2 * X[:, 1] * X[:, 12] - X[:, 13] + 0.5 * np.sin(6 * X[:, 1])
    m = costmodel.MLP()
    before = np.mean((m.predict_log_ms(X) - logt) ** 2)
    m.fit(X, logt, epochs=60, batch=256, lr=3e-3)
    after = np.mean((m.predict_log_ms(X) - logt) ** 2)
    assert after < 0.05 * before, (before, after)
