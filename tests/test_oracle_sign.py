"""Pins for the oracle's sign function (Sec. 1, Eqs. 4-6).

Checks: the scalar sign of Eq. 5 on hand values; a 2x2 triangular closed form;
sgn(A)^2 = I and [A, sgn A] = 0 (Eq. 6); the Newton iteration as an
independent second route; the free-field closed form; unitarity at mu = 0 and
the adjoint relation that follows from H_w(mu)^dag = H_w(-mu).
"""
import numpy as np
import pytest

from oracle import dirac, freefield, matfunc
from paper_0710_0341_gb300 import synth


def test_scalar_sign_hand_values():
    z = np.array([2.0, -3.0, 1 + 5j, -1e-3 + 7j, 0.5 - 2j, -4 - 1j])
    assert np.allclose(matfunc.sgn_scalar(z), [1, -1, 1, -1, 1, -1])
    s = matfunc.sgn_scalar(z)
    assert np.allclose(s * s, 1.0)


def test_triangular_2x2_closed_form():
    # T = [[a, c], [0, d]], Re a > 0 > Re d: sgn(T) = [[1, y], [0, -1]] with
    # a y - y d = 1*c - c*(-1)  =>  y = 2 c / (a - d)   (Eq. 18 with m = k = 1)
    a, d, c = 0.7 + 0.2j, -0.3 + 1.1j, 0.9 - 0.4j
    T = np.array([[a, c], [0, d]])
    S = matfunc.sign_eig(T)
    assert np.allclose(S, [[1, 2 * c / (a - d)], [0, -1]], atol=1e-14)
    Sn, _ = matfunc.sign_newton(T)
    assert np.allclose(Sn, S, atol=1e-14)


def test_diagonalisable_random_matrix_invariants():
    rng = np.random.default_rng(4)
    n = 60
    lam = rng.standard_normal(n) + 0.5j * rng.standard_normal(n)
    lam += np.sign(lam.real) * 0.05
    X = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = X @ np.diag(lam) @ np.linalg.inv(X)
    S = matfunc.sign_eig(A)
    assert np.linalg.norm(S @ S - np.eye(n)) < 1e-9 * n
    assert np.linalg.norm(A @ S - S @ A) < 1e-9 * np.linalg.norm(A) * n
    # trace counts the eigenvalues right of the imaginary axis minus the left ones
    assert abs(np.trace(S) - np.sum(np.sign(lam.real))) < 1e-8
    Sn, it = matfunc.sign_newton(A)
    assert it < 40
    assert np.linalg.norm(Sn - S) < 1e-8 * np.linalg.norm(S)


@pytest.mark.parametrize("mu", [0.0, 0.3, 0.5])
def test_free_field_dense_sign_matches_closed_form(mu):
    # for mu >= 0.7 the free spectrum touches the imaginary axis (sgn undefined, Eq. 5)
    dims = (2, 2, 2, 4)
    U = synth.unit_gauge_field(dims)
    A = dirac.hermitian_wilson(U, mu, -1.2).toarray()
    b = synth.gaussian_source(dims, 1)
    y = matfunc.sign_eig_apply(A, b.ravel()).reshape(b.shape)
    yf = freefield.sign_hw_free(b, mu, -1.2)
    assert np.linalg.norm(y - yf) <= 1e-11 * np.linalg.norm(yf)
    ev = np.linalg.eigvals(A)
    ef = freefield.spectrum_free(dims, mu, -1.2)
    assert np.abs(ef.real).min() > 0.1
    assert np.allclose(np.sort_complex(np.round(ev, 9)), np.sort_complex(np.round(ef, 9)), atol=1e-8)


def test_sign_of_gauge_field_operator():
    dims = (2, 2, 2, 2)
    U = synth.random_su3_field(dims, 0.5, 0)
    A = dirac.hermitian_wilson(U, 0.3, -1.0).toarray()
    S = matfunc.sign_eig(A)
    n = A.shape[0]
    assert np.linalg.norm(S @ S - np.eye(n)) < 1e-10 * n
    assert np.linalg.norm(A @ S - S @ A) < 1e-10 * n
    Sn, _ = matfunc.sign_newton(A)
    assert np.linalg.norm(Sn - S) < 1e-10 * np.linalg.norm(S)


def test_mu0_sign_is_unitary_and_adjoint_relation():
    dims = (2, 2, 2, 2)
    U = synth.random_su3_field(dims, 0.5, 3)
    b = synth.gaussian_source(dims, 1).ravel()
    a = synth.gaussian_source(dims, 2).ravel()
    A0 = dirac.hermitian_wilson(U, 0.0, -1.0).toarray()
    y0 = matfunc.sign_eig_apply(A0, b)
    assert abs(np.linalg.norm(y0) - np.linalg.norm(b)) < 1e-11 * np.linalg.norm(b)
    Ap = dirac.hermitian_wilson(U, 0.35, -1.0).toarray()
    Am = dirac.hermitian_wilson(U, -0.35, -1.0).toarray()
    lhs = np.vdot(a, matfunc.sign_eig_apply(Ap, b))
    rhs = np.vdot(matfunc.sign_eig_apply(Am, a), b)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
