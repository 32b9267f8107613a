"""The predictor's GPU MLP against the numpy reference (oracle.mlp), and the
predictor features against direct evaluation (link spread) and the oracle's
Arnoldi (Ritz values)."""
import numpy as np
import pytest

from helpers import lattice, need_gpu
from oracle import dirac, krylov, mlp
from paper_0710_0341_gb300 import ovl, synth

pytestmark = pytest.mark.gpu


def test_mlp_forward_and_gradient_match_reference():
    need_gpu()
    n_in, n_h, n_out, B = 20, 64, 2, 150
    rng = np.random.default_rng(1)
    net = ovl.ovl_mlp_create(n_in, n_h, n_out)
    try:
        npar = ovl.ovl_mlp_num_params(net)
        assert npar == mlp.n_params(n_in, n_h, n_out)
        theta = (rng.standard_normal(npar) * 0.2).astype(np.float32)
        ovl.ovl_mlp_set_params(net, theta)
        X = rng.standard_normal((B, n_in)).astype(np.float32)
        T = rng.standard_normal((B, n_out)).astype(np.float32)
        Y = np.zeros((B, n_out), np.float32)
        ovl.ovl_mlp_forward(net, X, Y)
        Yr, _ = mlp.forward(theta.astype(np.float64), X.astype(np.float64), n_in, n_h, n_out)
        assert np.abs(Y - Yr).max() <= 1e-4 * np.abs(Yr).max()
        g = np.zeros(npar, np.float32)
        loss = ovl.ovl_mlp_loss_grad(net, X, T, 4.0, g)
        lr, gr = mlp.loss_grad(theta.astype(np.float64), X.astype(np.float64), T.astype(np.float64), n_in, n_h,
                               n_out, 4.0)
        assert abs(loss - lr) <= 1e-4 * abs(lr)
        assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr)
    finally:
        ovl.ovl_mlp_destroy(net)


def test_mlp_training_fits_a_smooth_target():
    need_gpu()
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (256, 4)).astype(np.float32)
    T = np.stack([np.sin(2 * X[:, 0]) + X[:, 1] ** 2, X[:, 2] * X[:, 3]], 1).astype(np.float32)
    net = ovl.ovl_mlp_create(4, 64, 2)
    try:
        npar = ovl.ovl_mlp_num_params(net)
        ovl.ovl_mlp_set_params(net, (rng.standard_normal(npar) * 0.2).astype(np.float32))
        g = np.zeros(npar, np.float32)
        l0 = ovl.ovl_mlp_loss_grad(net, X, T, 1.0, g)
        l1 = ovl.ovl_mlp_train(net, X, T, 2000, 3e-3, 1.0)
        assert l1 < 0.05 * l0, (l0, l1)
    finally:
        ovl.ovl_mlp_destroy(net)


def test_features_link_spread_and_ritz_values():
    need_gpu()
    dims, mu, m_w = (4, 4, 4, 4), 0.3, -1.0
    U = synth.random_su3_field(dims, 0.4, 3)
    b = synth.gaussian_source(dims, 4)
    h = lattice(dims, U)
    try:
        s = ovl.ovl_link_spread(h)
        tr = np.einsum("...aa->...", U).real
        assert abs(s - np.mean(1 - tr / 3)) < 1e-12
        th = np.zeros(64, complex)
        ovl.ovl_ritz_values(h, mu, m_w, 64, b, th)
        A = dirac.hermitian_wilson(U, mu, m_w)
        r = krylov.arnoldi(A, b.ravel(), 64)
        ev = np.linalg.eigvals(r["H"])
        # same Ritz values (up to order)
        d = np.abs(np.sort_complex(th) - np.sort_complex(ev)).max()
        assert d < 1e-8 * np.abs(ev).max(), d
    finally:
        ovl.ovl_destroy_lattice(h)
