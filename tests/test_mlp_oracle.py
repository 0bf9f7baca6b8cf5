"""Pins of the FP64 cost-model network oracle (CPU): its gradient against
central finite differences of its own loss (a different computation from the
reverse-mode gradient), and its Adam step against the closed form of the
first step (m_hat = g, v_hat = g^2, so p -= lr g / (|g| + eps))."""
import numpy as np

import oracle

D = 17


def _problem(seed, n=12, scale=0.3):
    rng = np.random.default_rng(seed)
    P = (rng.standard_normal(oracle.mlp_param_count(D)) * scale).astype(np.float32)
    X = rng.standard_normal((n, D)).astype(np.float32)
    T = rng.standard_normal(n).astype(np.float32)
    return P, X, T


def test_param_count():
    assert oracle.mlp_param_count(D) == 64 * D + 64 + 2 * (64 * 64 + 64) + 64 + 1


def test_gradient_matches_finite_differences():
    P, X, T = _problem(0)
    _, _, g = oracle.mlp_loss_grad(P, X, T)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(P.size, 40, replace=False), [P.size - 1, 0, 64 * D]])
    # the oracle promotes float32 parameters to double: perturb in a float64
    # copy by passing float32 values that differ by exactly h
    for i in idx:
        h = 2.0 ** -12
        Pp = P.astype(np.float64).copy()
        Pm = P.astype(np.float64).copy()
        Pp[i] += h
        Pm[i] -= h
        lp = oracle.mlp_loss_grad(Pp.astype(np.float32), X, T, want_grad=False)[0]
        lm = oracle.mlp_loss_grad(Pm.astype(np.float32), X, T, want_grad=False)[0]
        fd = (lp - lm) / (float(np.float32(Pp[i])) - float(np.float32(Pm[i])))
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(g[i])) + 1e-7, (i, fd, g[i])


def test_loss_is_mean_squared_error_of_predictions():
    P, X, T = _problem(2)
    loss, y, _ = oracle.mlp_loss_grad(P, X, T, want_grad=False)
    assert np.isclose(loss, np.mean((y - T.astype(np.float64)) ** 2), rtol=1e-14)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    p = rng.standard_normal(100)
    g = rng.standard_normal(100)
    m = np.zeros(100)
    v = np.zeros(100)
    p0 = p.copy()
    oracle.adam_step(p, g, m, v, 1e-2, 0.9, 0.999, 1e-8, 1)
    assert np.allclose(p, p0 - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
