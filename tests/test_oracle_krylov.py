"""Pins for the oracle's Arnoldi approximation and the two deflation schemes.

Secs. 2-4: the Arnoldi relation (Eq. 7) and H = V^dag A V (Eq. 9); exactness
once the Krylov space is the whole space; Eq. 19 (Sylvester, Eq. 18) against
Eq. 16 (full block); the eigenpair relations of Eqs. 13 and 20; mu = 0, where
Schur and LR deflation reduce to the Hermitian deflation of Eq. 12; all
eigenvectors deflated (k = 0) giving the exact result; convergence with k and
with m against the dense spectral definition (Eq. 4).
"""
import numpy as np
import pytest

from oracle import dirac, eigen, krylov, matfunc
from paper_0710_0341_gb300 import synth


@pytest.fixture(scope="module")
def small():
    dims = (2, 2, 2, 4)
    U = synth.random_su3_field(dims, 0.5, 0)
    A = dirac.hermitian_wilson(U, 0.3, -1.0)
    Ad = A.toarray()
    b = synth.gaussian_source(dims, 1).ravel()
    ystar = matfunc.sign_eig_apply(Ad, b)
    lam, R, L = eigen.critical_dense(Ad, 24)
    return dict(A=A, Ad=Ad, b=b, ystar=ystar, lam=lam, R=R, L=L, N=Ad.shape[0])


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_arnoldi_relation(small):
    A, b = small["A"], small["b"]
    k = 40
    r = krylov.arnoldi(A, b, k)
    V, H = r["V"], r["H"]
    assert np.abs(V.conj().T @ V - np.eye(k)).max() < 1e-13
    AV = np.column_stack([A @ V[:, i] for i in range(k)])
    E = AV - V @ H
    E[:, -1] -= r["beta_k"] * r["v_next"]
    assert np.linalg.norm(E) < 1e-13 * np.linalg.norm(AV)
    assert np.allclose(H, V.conj().T @ AV, atol=1e-13)
    assert np.abs(np.tril(H, -2)).max() == 0.0
    assert np.allclose(V[:, 0] * r["beta"], b)


def test_full_krylov_is_exact(small):
    A, b, N = small["A"], small["b"], small["N"]
    y = krylov.sign_arnoldi(A, b, N)
    assert rel(y, small["ystar"]) < 1e-10


def test_eigenpair_relations(small):
    Ad, lam, R, L = small["Ad"], small["lam"], small["R"], small["L"]
    assert np.abs(L.conj().T @ R - np.eye(R.shape[1])).max() < 1e-12
    assert np.linalg.norm(Ad @ R - R * lam) < 1e-12 * np.linalg.norm(Ad)
    assert np.linalg.norm(L.conj().T @ Ad - lam[:, None] * L.conj().T) < 1e-10 * np.linalg.norm(L)
    S, T = eigen.schur_from_right(small["A"], R[:, :12])
    assert np.abs(S.conj().T @ S - np.eye(12)).max() < 1e-13
    assert np.abs(np.tril(T, -1)).max() < 1e-12
    assert np.linalg.norm(Ad @ S - S @ T) < 1e-12
    assert np.allclose(np.sort_complex(np.diag(T)), np.sort_complex(lam[:12]))
    # critical = smallest |Re lambda|
    allev = np.linalg.eigvals(Ad)
    assert np.abs(lam.real).max() <= np.sort(np.abs(allev.real))[23] + 1e-12


@pytest.mark.parametrize("m,k", [(6, 20), (12, 30), (24, 12)])
def test_schur_sylvester_equals_block(small, m, k):
    A, b, R = small["A"], small["b"], small["R"]
    S, T = eigen.schur_from_right(A, R[:, :m])
    y19 = krylov.sign_schur(A, b, k, S, T)
    y16 = krylov.sign_schur_block(A, b, k, S, T)
    assert rel(y19, y16) < 1e-12


def test_all_eigenvectors_deflated_is_exact(small):
    Ad, b, N = small["Ad"], small["b"], small["N"]
    lam, R, L = eigen.critical_dense(Ad, N)
    y = krylov.sign_lr(small["A"], b, 0, R, lam, L)
    assert rel(y, small["ystar"]) < 1e-10


def test_convergence_in_k_and_m(small):
    A, b, ystar, lam, R, L = (small[x] for x in ("A", "b", "ystar", "lam", "R", "L"))
    errs = {}
    for m in (0, 12, 24):
        for k in (20, 60, 100):
            if m == 0:
                y = krylov.sign_arnoldi(A, b, k)
            else:
                y = krylov.sign_lr(A, b, k, R[:, :m], lam[:m], L[:, :m])
            errs[m, k] = rel(y, ystar)
    for m in (0, 12, 24):
        assert errs[m, 20] > errs[m, 60] > errs[m, 100]
    for k in (20, 60, 100):
        assert errs[0, k] > errs[12, k] > errs[24, k]
    assert errs[24, 100] < 1e-5


def test_mu0_schur_lr_hermitian_agree():
    dims = (2, 2, 2, 4)
    U = synth.random_su3_field(dims, 0.5, 2)
    A = dirac.hermitian_wilson(U, 0.0, -1.0)
    Ad = A.toarray()
    b = synth.gaussian_source(dims, 1).ravel()
    w, Q = np.linalg.eigh(Ad)
    idx = np.argsort(np.abs(w))[:10]
    y12 = krylov.sign_hermitian_deflated(A, b, 30, Q[:, idx], w[idx])
    lam, R, L = eigen.critical_dense(Ad, 10)
    ylr = krylov.sign_lr(A, b, 30, R, lam, L)
    S, T = eigen.schur_from_right(A, R)
    ysc = krylov.sign_schur(A, b, 30, S, T)
    assert rel(ylr, y12) < 1e-11
    assert rel(ysc, y12) < 1e-11
    # at mu = 0 the left and right eigenvectors coincide and T is diagonal
    assert np.abs(L - R).max() < 1e-10
    assert np.abs(T - np.diag(np.diag(T))).max() < 1e-10


def test_eigenvector_input_basis_invariance(small):
    # the Schur result depends only on span(S) (Eq. 16 is basis-free in Omega_m)
    A, b, R = small["A"], small["b"], small["R"]
    S, T = eigen.schur_from_right(A, R[:, :10])
    rng = np.random.default_rng(0)
    Z, _ = np.linalg.qr(rng.standard_normal((10, 10)) + 1j * rng.standard_normal((10, 10)))
    S2 = S @ Z
    T2 = Z.conj().T @ T @ Z
    y1 = krylov.sign_schur_block(A, b, 25, S, T)
    y2 = krylov.sign_schur_block(A, b, 25, S2, T2)
    assert rel(y1, y2) < 1e-12


def test_sparse_critical_pairs_match_the_dense_route(small):
    """ARPACK on A^2 with Rayleigh-Ritz (the sparse route for lattices too
    large for a dense decomposition) finds the same critical eigenvalues as the
    dense eigendecomposition, eigenvectors spanning the same space, and left
    vectors from H_w(-mu) with L^dag R = I."""
    U = synth.random_su3_field((2, 2, 2, 4), 0.5, 0)
    Am = dirac.hermitian_wilson(U, -0.3, -1.0)
    m = 12
    lam, R, L, res = eigen.critical_sparse(small["A"], Am, m, nev=24)
    assert np.abs(lam - small["lam"][:m]).max() < 1e-10
    assert res.max() < 1e-10 * np.abs(small["Ad"]).max()
    # same span: the dense eigenvectors lie in span(R)
    Qr, _ = np.linalg.qr(R)
    Rd = small["R"][:, :m]
    assert np.linalg.norm(Rd - Qr @ (Qr.conj().T @ Rd)) < 1e-9
    assert np.abs(L.conj().T @ R - np.eye(m)).max() < 1e-9
    # left vectors: L^dag A = Lambda L^dag
    assert np.linalg.norm(L.conj().T @ small["Ad"] - lam[:, None] * L.conj().T) < 1e-9 * np.linalg.norm(L)


def test_lr_result_lies_in_its_search_space(small):
    """Eq. 22 combines R_m and the Krylov vectors of x_minus only: the LR
    approximation lies in span(R_m) + K_k(A, x_minus), and the orthogonal
    projection of the exact result on that space is at least as close."""
    m, k = 8, 25
    R, L, lam = small["R"][:, :m], small["L"][:, :m], small["lam"][:m]
    y = krylov.sign_lr(small["A"], small["b"], k, R, lam, L)
    Q = krylov.lr_search_space(small["A"], small["b"], k, R, L)
    assert Q.shape == (small["N"], m + k)
    assert rel(krylov.best_approximation(Q, y), y) < 1e-12
    yb = krylov.best_approximation(Q, small["ystar"])
    assert rel(yb, small["ystar"]) <= rel(y, small["ystar"]) * (1 + 1e-12)
    # the space is not the whole space: the projection changes the exact result
    assert rel(yb, small["ystar"]) > 1e-8
