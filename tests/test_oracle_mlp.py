"""Pin of the reference MLP: analytic gradient vs central finite differences."""
import numpy as np

from oracle import mlp


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_in, n_h, n_out, B = 5, 7, 2, 9
    theta = rng.standard_normal(mlp.n_params(n_in, n_h, n_out)) * 0.5
    X = rng.standard_normal((B, n_in))
    T = rng.standard_normal((B, n_out))
    loss, g = mlp.loss_grad(theta, X, T, n_in, n_h, n_out)
    h = 1e-6
    for i in rng.choice(theta.size, 25, replace=False):
        e = np.zeros_like(theta)
        e[i] = h
        lp, _ = mlp.loss_grad(theta + e, X, T, n_in, n_h, n_out)
        lm, _ = mlp.loss_grad(theta - e, X, T, n_in, n_h, n_out)
        assert abs((lp - lm) / (2 * h) - g[i]) <= 1e-6 * max(1.0, abs(g[i]))


def test_mlp_under_prediction_weight():
    theta = np.zeros(mlp.n_params(1, 2, 1))
    X = np.zeros((1, 1))
    l_under, _ = mlp.loss_grad(theta, X, np.array([[1.0]]), 1, 2, 1, under_weight=4.0)
    l_over, _ = mlp.loss_grad(theta, X, np.array([[-1.0]]), 1, 2, 1, under_weight=4.0)
    assert l_under == 4.0 and l_over == 1.0
