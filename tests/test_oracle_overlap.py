"""Pins of the overlap operator oracle (Sec. 1, Eq. 1).

Dense checks on a 2^4 lattice (N = 192): the Ginsparg-Wilson relation
gamma5 D + D gamma5 = D gamma5 D (it follows from sgn^2 = I, Sec. 1), the
adjoint route (D^dag from sgn(H_w(-mu)) equals the conjugate transpose), at
mu = 0 gamma5-Hermiticity D^dag = gamma5 D gamma5 and the spectrum on the
Ginsparg-Wilson circle |z - 1| = 1, the LR data of the adjoint (Eq. 20 with
left and right swapped), and the matrix-free routes against the dense matrix.
"""
import numpy as np
import pytest

from oracle import dirac, eigen, matfunc, overlap
from paper_0710_0341_gb300 import synth

DIMS = (2, 2, 2, 2)


def _g5(V):
    return dirac.gamma5_matrix(V).toarray()


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_ginsparg_wilson_relation(mu):
    U = synth.random_su3_field(DIMS, 0.5, 0)
    D = overlap.overlap_dense(U, mu, -1.0)
    g5 = _g5(D.shape[0] // 12)
    lhs = g5 @ D + D @ g5
    rhs = D @ g5 @ D
    assert np.linalg.norm(lhs - rhs) <= 1e-11 * np.linalg.norm(lhs)
    # a plausible slip (sgn replaced by a non-involution, e.g. H / |H|_2) breaks it
    A = dirac.hermitian_wilson(U, mu, -1.0).toarray()
    Dbad = np.eye(A.shape[0]) + g5 @ (A / np.linalg.norm(A, 2))
    assert np.linalg.norm(g5 @ Dbad + Dbad @ g5 - Dbad @ g5 @ Dbad) > 1e-3


def test_adjoint_route_equals_conjugate_transpose():
    U = synth.random_su3_field(DIMS, 0.5, 0)
    mu = 0.3
    D = overlap.overlap_dense(U, mu, -1.0)
    Am = dirac.hermitian_wilson(U, -mu, -1.0).toarray()
    x = synth.gaussian_source(DIMS, 7)
    y = overlap.overlap_adjoint_apply(
        lambda v: matfunc.sign_eig_apply(Am, v.ravel()).reshape(v.shape), x)
    ref = (D.conj().T @ x.ravel()).reshape(x.shape)
    assert np.linalg.norm(y - ref) <= 1e-11 * np.linalg.norm(ref)
    # and the forward route against the dense matrix
    A = dirac.hermitian_wilson(U, mu, -1.0).toarray()
    y2 = overlap.overlap_apply(lambda v: matfunc.sign_eig_apply(A, v.ravel()).reshape(v.shape), x)
    assert np.linalg.norm(y2 - (D @ x.ravel()).reshape(x.shape)) <= 1e-11 * np.linalg.norm(y2)


def test_mu0_gamma5_hermitian_and_gw_circle():
    U = synth.random_su3_field(DIMS, 0.5, 0)
    D = overlap.overlap_dense(U, 0.0, -1.0)
    g5 = _g5(D.shape[0] // 12)
    assert np.linalg.norm(D.conj().T - g5 @ D @ g5) <= 1e-11 * np.linalg.norm(D)
    z = np.linalg.eigvals(D)
    assert np.max(np.abs(np.abs(z - 1.0) - 1.0)) < 1e-10
    # at mu != 0 the spectrum leaves the circle (the relation still holds)
    z3 = np.linalg.eigvals(overlap.overlap_dense(U, 0.3, -1.0))
    assert np.max(np.abs(np.abs(z3 - 1.0) - 1.0)) > 1e-6


def test_lr_data_of_the_adjoint():
    U = synth.random_su3_field(DIMS, 0.5, 0)
    A = dirac.hermitian_wilson(U, 0.3, -1.0).toarray()
    lam, R, L = eigen.critical_dense(A, 6)
    lam2, R2, L2 = overlap.lr_adjoint(lam, R, L)
    Ah = A.conj().T
    assert np.linalg.norm(Ah @ R2 - R2 * lam2[None, :]) <= 1e-10 * np.linalg.norm(Ah)
    assert np.linalg.norm(L2.conj().T @ Ah - lam2[:, None] * L2.conj().T) <= 1e-10 * np.linalg.norm(Ah)
    assert np.linalg.norm(L2.conj().T @ R2 - np.eye(6)) <= 1e-10
