"""Pins for the oracle's Wilson-Dirac operator (Sec. 1, Eq. 2).

Each check is independent of the sparse construction it tests: the Clifford
algebra, the momentum-space closed form on the free field, gauge covariance,
gamma5-hermiticity H_w(mu)^dag = H_w(-mu) and hand-derived single values.
"""
import math

import numpy as np
import pytest

from oracle import dirac, freefield
from paper_0710_0341_gb300 import synth


def test_gamma_clifford_and_gamma5():
    G = dirac.GAMMA
    for a in range(4):
        assert np.allclose(G[a], G[a].conj().T)
        for b in range(4):
            ac = G[a] @ G[b] + G[b] @ G[a]
            assert np.allclose(ac, 2.0 * (a == b) * np.eye(4))
    assert np.allclose(dirac.GAMMA5, np.diag([1, 1, -1, -1]))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 3, 2, 4), (3, 2, 5, 2)])
@pytest.mark.parametrize("mu", [0.0, 0.3, 0.8])
@pytest.mark.parametrize("apbc", [False, True])
def test_free_field_matches_momentum_space(dims, mu, apbc):
    U = synth.unit_gauge_field(dims)
    psi = synth.gaussian_source(dims, 3)
    A = dirac.hermitian_wilson(U, mu, -1.3, antiperiodic_t=apbc)
    y = dirac.apply(A, psi)
    yf = freefield.apply_hw_free(psi, mu, -1.3, antiperiodic_t=apbc)
    assert np.linalg.norm(y - yf) <= 1e-13 * np.linalg.norm(yf)


def test_zero_momentum_hand_values():
    # U = 1, constant spinor: hops give a = 1 - 2 kappa (3 + cosh mu) and the
    # time sine sin(-i mu) = -i sinh mu, so D chi = a chi - 2 i kappa gamma_4 (-i sinh mu) chi.
    dims = (2, 2, 2, 2)
    m_w, mu = -1.0, 0.4
    kap = 1.0 / (8 + 2 * m_w)
    chi = np.arange(12, dtype=float).reshape(4, 3) + 1j
    psi = np.broadcast_to(chi, (2, 2, 2, 2, 4, 3)).copy()
    D = dirac.wilson_dirac(synth.unit_gauge_field(dims), mu, m_w)
    out = dirac.apply(D, psi)[0, 0, 0, 0]
    a = 1 - 2 * kap * (3 + math.cosh(mu))
    expect = a * chi - 2 * kap * math.sinh(mu) * (dirac.GAMMA[3] @ chi)
    assert np.allclose(out, expect, atol=1e-14)


def test_diagonal_and_row_counts():
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.5, 0)
    D = dirac.wilson_dirac(U, 0.3, -1.0)
    assert np.allclose(D.diagonal(), 1.0)
    # 1 diagonal + 8 hops x (2 nonzero spin entries per row of 1 +- gamma) x 3 colours
    assert D.nnz == 49 * D.shape[0]


@pytest.mark.parametrize("mu", [0.0, 0.25])
def test_gauge_covariance(mu):
    dims = (3, 4, 2, 4)
    U = synth.random_su3_field(dims, 0.7, 5)
    g = synth.random_gauge_transform(dims, 9)
    lt, lz, ly, lx = U.shape[:4]
    Ug = np.empty_like(U)
    shifts = {0: (3, 1), 1: (2, 1), 2: (1, 1), 3: (0, 1)}
    for nu in range(4):
        ax, s = shifts[nu]
        g_fwd = np.roll(g, -s, axis=ax)  # g_{n + nu}
        Ug[..., nu, :, :] = g @ U[..., nu, :, :] @ np.conj(np.swapaxes(g_fwd, -1, -2))
    psi = synth.gaussian_source(dims, 2)
    A = dirac.hermitian_wilson(U, mu, -1.1)
    Ag = dirac.hermitian_wilson(Ug, mu, -1.1)
    gpsi = np.einsum("...ab,...sb->...sa", g, psi)
    lhs = dirac.apply(Ag, gpsi)
    rhs = np.einsum("...ab,...sb->...sa", g, dirac.apply(A, psi))
    assert np.linalg.norm(lhs - rhs) <= 1e-13 * np.linalg.norm(rhs)


def test_gamma5_hermiticity_and_mu0_hermitian():
    dims = (4, 2, 3, 4)
    U = synth.random_su3_field(dims, 0.6, 11)
    Ap = dirac.hermitian_wilson(U, 0.45, -0.9)
    Am = dirac.hermitian_wilson(U, -0.45, -0.9)
    assert abs(Ap.conj().T - Am).max() < 1e-15
    A0 = dirac.hermitian_wilson(U, 0.0, -0.9)
    assert abs(A0.conj().T - A0).max() < 1e-15
    # and mu != 0 really is non-Hermitian
    assert abs(Ap.conj().T - Ap).max() > 1e-2


def test_links_are_su3():
    U = synth.random_su3_field((2, 2, 2, 2), 0.5, 0)
    I = np.einsum("...ab,...cb->...ac", U, U.conj())
    assert np.allclose(I, np.eye(3), atol=1e-13)
    assert np.allclose(np.linalg.det(U), 1.0, atol=1e-13)


@pytest.mark.parametrize("dims,apbc", [((3, 4, 2, 5), 1), ((4, 4, 4, 4), 0)])
def test_row_evaluation_matches_sparse_operator(dims, apbc):
    """The row-by-row evaluation of H_w(mu) used for sampled checks at full
    lattice sizes equals the sparse matrix of Eq. 2 (boundary sites included)."""
    U = synth.random_su3_field(dims, 0.5, 1)
    x = synth.gaussian_source(dims, 2)
    A = dirac.hermitian_wilson(U, 0.3, -1.2, antiperiodic_t=bool(apbc))
    full = dirac.apply(A, x).reshape(-1, 4, 3)
    V = full.shape[0]
    sites = sorted({0, V - 1, 1, dims[0] - 1, V // 2, V - dims[0]} | set(range(0, V, max(1, V // 17))))
    rows = dirac.hermitian_wilson_rows(U, 0.3, -1.2, x, sites, antiperiodic_t=bool(apbc))
    assert np.abs(rows - full[sites]).max() <= 1e-14 * np.abs(full).max()
