"""Pins of the oracle's Jordan-form definition of f(A) and sgn(A) for matrices
that cannot be diagonalised (Sec. 1, after Eq. 4), checked against library
routines and the defining properties of the sign function:

* fun_jordan with f = exp against scipy's expm (Pade approximation, no
  eigenvectors): pins the sum over the powers of the shift and its 1/j!;
* sign_jordan against scipy's signm and against the oracle's scaled Newton
  iteration (neither forms eigenvectors);
* sgn(A)^2 = I, sgn(A) commutes with A, and the trace of sgn(A) counts the
  eigenvalues right of the imaginary axis minus those left of it;
* a single Jordan block gives sgn(Re l) I exactly;
* the eigenvector route of Eq. 4 is not a definition here (its error on the
  same defective matrix is many orders larger).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import matfunc as mf

BLOCKS = [(0.3 + 0.1j, 3), (-0.2, 2), (0.5 - 0.4j, 1), (-0.7 + 0.2j, 4), (0.25, 2)]


def _defective(blocks, seed=0, spread=0.3):
    J = mf.jordan_form(blocks)
    n = J.shape[0]
    rng = np.random.default_rng(seed)
    X = np.eye(n) + spread * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    return X, X @ J @ np.linalg.inv(X)


def test_jordan_form_layout():
    J = mf.jordan_form([(2.0, 2), (-1.0 + 1j, 1)])
    ref = np.array([[2, 1, 0], [0, 2, 0], [0, 0, -1 + 1j]], dtype=complex)
    assert np.array_equal(J, ref)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fun_jordan_exp_matches_expm(seed):
    X, A = _defective(BLOCKS, seed)
    E = mf.fun_jordan(X, BLOCKS, lambda lam, j: np.exp(lam))
    ref = sla.expm(A)
    assert np.abs(E - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sign_jordan_matches_signm_and_newton(seed):
    X, A = _defective(BLOCKS, seed)
    S = mf.sign_jordan(X, BLOCKS)
    scale = np.abs(S).max()
    assert np.abs(S - sla.signm(A)).max() < 1e-11 * scale
    assert np.abs(S - mf.sign_newton(A)[0]).max() < 1e-11 * scale


def test_sign_jordan_properties():
    X, A = _defective(BLOCKS, 3)
    S = mf.sign_jordan(X, BLOCKS)
    n = A.shape[0]
    assert np.abs(S @ S - np.eye(n)).max() < 1e-12
    assert np.abs(S @ A - A @ S).max() < 1e-12 * np.abs(A).max()
    right = sum(k for lam, k in BLOCKS if np.real(lam) > 0)
    assert abs(np.trace(S) - (right - (n - right))) < 1e-10


def test_single_block_is_a_multiple_of_the_identity():
    for lam in (0.4 + 2j, -0.05 - 1j):
        J = mf.jordan_form([(lam, 5)])
        S = mf.sign_jordan(np.eye(5), [(lam, 5)])
        assert np.array_equal(S, np.sign(lam.real) * np.eye(5))
        assert np.abs(mf.sign_newton(J)[0] - S).max() < 1e-12


def test_eigenvector_route_is_not_a_definition_for_defective_matrices():
    X, A = _defective(BLOCKS, 0)
    S = mf.sign_jordan(X, BLOCKS)
    assert np.abs(mf.sign_eig(A) - S).max() > 1e3 * np.abs(sla.signm(A) - S).max()


def test_imaginary_axis_eigenvalue_rejected():
    with pytest.raises(ValueError):
        mf.sign_jordan(np.eye(2), [(0.5j, 2)])
