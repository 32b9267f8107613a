"""Closed-form sign of H_w(mu) on the free field U = 1 (derived from Eq. 2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

With U = 1, a plane wave psi_n = e^{i p.n} chi diagonalises the hops of Eq. 2:
psi_{n +- nu} = e^{+- i p_nu} psi_n, and the e^{+-mu} weights of the time hops
combine with e^{+- i p_4} into e^{+- i pt_4}, pt_4 = p_4 - i mu (pt_j = p_j).
Hence

    D_w(p) = a(p) - 2 i kappa sum_nu gamma_nu sin(pt_nu),
    a(p)   = 1 - 2 kappa sum_nu cos(pt_nu),

and, because gamma_5 anticommutes with every gamma_nu,

    H_w(p)^2 = [a(p)^2 + 4 kappa^2 sum_nu sin^2(pt_nu)] * 1   (a scalar),

so sgn(H_w(p)) = H_w(p) / sqrt(omega2(p)) with the principal root (Eq. 5,
applied to the two eigenvalues +-sqrt(omega2)).  The result is assembled with
FFTs: psi_n = (1/V) sum_p e^{+i p.n} chi_p, p_nu = 2 pi k_nu / L_nu (plus
pi / L_t for an antiperiodic time direction).
"""
from __future__ import annotations

import numpy as np

from .dirac import GAMMA, GAMMA5, kappa_of


def _momenta(dims, antiperiodic_t):
    lx, ly, lz, lt = dims
    px = 2 * np.pi * np.arange(lx) / lx
    py = 2 * np.pi * np.arange(ly) / ly
    pz = 2 * np.pi * np.arange(lz) / lz
    pt = 2 * np.pi * np.arange(lt) / lt + (np.pi / lt if antiperiodic_t else 0.0)
    T, Z, Y, X = np.meshgrid(pt, pz, py, px, indexing="ij")
    return X, Y, Z, T


def _hw_momentum(dims, mu, m_w, antiperiodic_t):
    """H_w(p) as (Lt,Lz,Ly,Lx,4,4) spin matrices, and omega2(p)."""
    kap = kappa_of(m_w)
    X, Y, Z, T = _momenta(dims, antiperiodic_t)
    pt = [X, Y, Z, T - 1j * mu]
    a = 1.0 - 2.0 * kap * sum(np.cos(q) for q in pt)
    D = a[..., None, None] * np.eye(4)
    for nu in range(4):
        D = D - 2j * kap * np.sin(pt[nu])[..., None, None] * GAMMA[nu]
    H = np.einsum("st,...tu->...su", GAMMA5, D)
    om2 = a * a + 4.0 * kap * kap * sum(np.sin(q) ** 2 for q in pt)
    return H, om2


def apply_hw_free(psi: np.ndarray, mu: float, m_w: float, antiperiodic_t=False):
    """H_w(mu) psi for U = 1, computed in momentum space."""
    lt, lz, ly, lx = psi.shape[:4]
    dims = (lx, ly, lz, lt)
    H, _ = _hw_momentum(dims, mu, m_w, antiperiodic_t)
    return _apply_spin_in_momentum(psi, H, dims, antiperiodic_t)


def sign_hw_free(psi: np.ndarray, mu: float, m_w: float, antiperiodic_t=False):
    """sgn(H_w(mu)) psi for U = 1, closed form H_w(p)/sqrt(omega2(p))."""
    lt, lz, ly, lx = psi.shape[:4]
    dims = (lx, ly, lz, lt)
    H, om2 = _hw_momentum(dims, mu, m_w, antiperiodic_t)
    S = H / np.sqrt(om2.astype(np.complex128))[..., None, None]
    return _apply_spin_in_momentum(psi, S, dims, antiperiodic_t)


def spectrum_free(dims, mu, m_w, antiperiodic_t=False):
    """All eigenvalues of H_w(mu) at U = 1: +-sqrt(omega2(p)), each 6-fold."""
    _, om2 = _hw_momentum(dims, mu, m_w, antiperiodic_t)
    r = np.sqrt(om2.astype(np.complex128)).ravel()
    return np.concatenate([np.repeat(r, 6), np.repeat(-r, 6)])


def _apply_spin_in_momentum(psi, M, dims, antiperiodic_t):
    lx, ly, lz, lt = dims
    work = psi.astype(np.complex128)
    if antiperiodic_t:
        t = np.arange(lt)
        work = work * np.exp(-1j * np.pi * t / lt)[:, None, None, None, None, None]
    chi = np.fft.fftn(work, axes=(0, 1, 2, 3))
    chi = np.einsum("...st,...tc->...sc", M, chi)
    out = np.fft.ifftn(chi, axes=(0, 1, 2, 3))
    if antiperiodic_t:
        t = np.arange(lt)
        out = out * np.exp(1j * np.pi * t / lt)[:, None, None, None, None, None]
    return out
