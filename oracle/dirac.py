"""Wilson-Dirac operator at chemical potential mu (Sec. 1, Eq. 2), FP64 sparse.

TEST INFRASTRUCTURE ONLY (see the package docstring).

[D_w(mu)]_{nm} = delta_{nm}
    - kappa sum_{j=1..3} [ (1+gamma_j) U_{n,j} delta_{n+j,m}
                          + (1-gamma_j) U^dag_{n-j,j} delta_{n-j,m} ]
    - kappa [ (1+gamma_4) e^{+mu} U_{n,4} delta_{n+4,m}
             + (1-gamma_4) e^{-mu} U^dag_{n-4,4} delta_{n-4,m} ],
kappa = 1/(8 + 2 m_w), and H_w(mu) = gamma_5 D_w(mu) with
gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4.

Readings of the paper (it names only "Euclidean" gamma matrices): the
Hermitian chiral basis below, in which gamma_5 = diag(1, 1, -1, -1); the
directions 1..4 are x, y, z, t and the site index is
n = x + Lx*(y + Ly*(z + Lz*t)); boundaries are periodic, with an optional
antiperiodic time direction (the paper states none).

Vector index: 12*n + 3*spin + colour (the canonical layout of ``synth``).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# Euclidean gamma matrices, Hermitian chiral basis (index 0..3 = x, y, z, t).
GAMMA = np.array(
    [
        [[0, 0, 0, 1j], [0, 0, 1j, 0], [0, -1j, 0, 0], [-1j, 0, 0, 0]],
        [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
        [[0, 0, 1j, 0], [0, 0, 0, -1j], [-1j, 0, 0, 0], [0, 1j, 0, 0]],
        [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
    ],
    dtype=np.complex128,
)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]


def kappa_of(m_w: float) -> float:
    """kappa = 1/(8 + 2 m_w) (Eq. 2)."""
    return 1.0 / (8.0 + 2.0 * m_w)


def _site_coords(dims):
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(
        np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij"
    )
    return [a.ravel() for a in (x, y, z, t)]


def _site_index(coords, dims):
    x, y, z, t = coords
    lx, ly, lz, lt = dims
    return x + lx * (y + ly * (z + lz * t))


def wilson_dirac(U: np.ndarray, mu: float, m_w: float, antiperiodic_t: bool = False):
    """Sparse D_w(mu) of Eq. 2 (CSR, N = 12 V), links U[t,z,y,x,nu,3,3]."""
    lt, lz, ly, lx = U.shape[:4]
    dims = (lx, ly, lz, lt)
    V = lx * ly * lz * lt
    kap = kappa_of(m_w)
    Uf = U.reshape(V, 4, 3, 3)
    coords = _site_coords(dims)
    n = _site_index(coords, dims)
    eye4 = np.eye(4, dtype=np.complex128)

    blocks_r, blocks_c, blocks_d = [n], [n], [np.broadcast_to(np.eye(12), (V, 12, 12))]
    for nu in range(4):
        fwd = [c.copy() for c in coords]
        bwd = [c.copy() for c in coords]
        L = dims[nu]
        fwd[nu] = (coords[nu] + 1) % L
        bwd[nu] = (coords[nu] - 1) % L
        nf = _site_index(fwd, dims)
        nb = _site_index(bwd, dims)
        sf = np.ones(V)
        sb = np.ones(V)
        if nu == 3 and antiperiodic_t:
            sf = np.where(coords[3] == L - 1, -1.0, 1.0)
            sb = np.where(coords[3] == 0, -1.0, 1.0)
        wf = np.exp(mu) if nu == 3 else 1.0
        wb = np.exp(-mu) if nu == 3 else 1.0
        Pp = eye4 + GAMMA[nu]
        Pm = eye4 - GAMMA[nu]
        # forward hop: -kappa (1+gamma_nu) w+ U_{n,nu} psi_{n+nu}
        Ufw = Uf[n, nu]
        blk_f = -kap * wf * sf[:, None, None] * np.einsum("st,nab->nsatb", Pp, Ufw).reshape(V, 12, 12)
        # backward hop: -kappa (1-gamma_nu) w- U^dag_{n-nu,nu} psi_{n-nu}
        Ubw = np.conj(np.swapaxes(Uf[nb, nu], -1, -2))
        blk_b = -kap * wb * sb[:, None, None] * np.einsum("st,nab->nsatb", Pm, Ubw).reshape(V, 12, 12)
        blocks_r += [n, n]
        blocks_c += [nf, nb]
        blocks_d += [blk_f, blk_b]

    rows = np.concatenate(blocks_r)
    cols = np.concatenate(blocks_c)
    data = np.concatenate([np.asarray(d) for d in blocks_d])
    shape3 = (rows.size, 12, 12)
    ri = np.broadcast_to(rows[:, None, None] * 12 + np.arange(12)[None, :, None], shape3)
    ci = np.broadcast_to(cols[:, None, None] * 12 + np.arange(12)[None, None, :], shape3)
    M = sp.coo_matrix((data.ravel(), (ri.ravel(), ci.ravel())), shape=(12 * V, 12 * V))
    M = M.tocsr()
    M.sum_duplicates()
    M.eliminate_zeros()
    return M


def gamma5_matrix(V: int):
    """gamma_5 acting on spin of every site (colour identity), sparse diagonal."""
    d = np.kron(np.ones(V), np.kron(np.diag(GAMMA5).real, np.ones(3)))
    return sp.diags(d.astype(np.complex128)).tocsr()


def hermitian_wilson(U: np.ndarray, mu: float, m_w: float, antiperiodic_t: bool = False):
    """Sparse H_w(mu) = gamma_5 D_w(mu) (Sec. 1)."""
    lt, lz, ly, lx = U.shape[:4]
    V = lx * ly * lz * lt
    return (gamma5_matrix(V) @ wilson_dirac(U, mu, m_w, antiperiodic_t)).tocsr()


def hermitian_wilson_rows(U: np.ndarray, mu: float, m_w: float, psi: np.ndarray, sites,
                          antiperiodic_t: bool = False) -> np.ndarray:
    """(H_w(mu) psi) at the given sites only (Eq. 2, then gamma_5), by plain
    loops over the eight hops: for lattices whose sparse matrix is too large to
    build. psi and U in the canonical shapes; returns (len(sites), 4, 3)."""
    lt, lz, ly, lx = U.shape[:4]
    dims = (lx, ly, lz, lt)
    kap = kappa_of(m_w)
    out = []
    for site in sites:
        x = site % lx
        y = (site // lx) % ly
        z = (site // (lx * ly)) % lz
        t = site // (lx * ly * lz)
        c = [x, y, z, t]
        acc = np.zeros((4, 3), dtype=np.complex128)
        for nu in range(4):
            for fwd in (True, False):
                cn = list(c)
                cn[nu] = (c[nu] + (1 if fwd else -1)) % dims[nu]
                sign = 1.0
                if nu == 3 and antiperiodic_t and ((fwd and c[3] == lt - 1) or (not fwd and c[3] == 0)):
                    sign = -1.0
                w = (np.exp(mu) if fwd else np.exp(-mu)) if nu == 3 else 1.0
                nb = psi[cn[3], cn[2], cn[1], cn[0]]  # (4, 3)
                if fwd:
                    link = U[t, z, y, x, nu]
                    proj = np.eye(4) + GAMMA[nu]
                else:
                    link = np.conj(U[cn[3], cn[2], cn[1], cn[0], nu]).T
                    proj = np.eye(4) - GAMMA[nu]
                acc += sign * w * (proj @ nb @ link.T)
        d = psi[t, z, y, x] - kap * acc
        out.append(GAMMA5 @ d)
    return np.array(out)


def apply(A, psi: np.ndarray) -> np.ndarray:
    """A @ psi for a canonical-shaped spinor (keeps the shape)."""
    return (A @ psi.reshape(-1)).reshape(psi.shape)
