"""Paper-style convergence study on a synthetic field (Sec. 5, Fig. 1 setting).

The paper shows the error of the LR-deflated approximation of sgn(H_w) x
against the Krylov depth k for several numbers m of deflated eigenvectors,
with x = (1, ..., 1) and mu = 0.3, and notes that the result is very close to
the best approximation in Omega_m + K_k. Its gauge configurations and curves
are not available, so this study runs the same setting on a seeded synthetic
4^4 field (eps 0.5, m_w -1) and checks what the paper's statements fix
qualitatively: the error falls with k, deflation lowers the depth needed for
a given accuracy, and the result stays within a small factor of the best
approximation (the orthogonal projection of the exact y* on span(R_m, K_k)).
The exact y* is the oracle's dense spectral sign (Eqs. 4-6). The CUDA path
computes every (m, k) point in one batched call; the table goes to stdout.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from helpers import canon_cols, lattice, need_gpu, rel
from oracle import dirac, eigen, krylov
from paper_0710_0341_gb300 import ovl, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_error_vs_depth_lr_deflation_4x4():
    need_gpu()
    dims, mu, m_w = (4, 4, 4, 4), 0.3, -1.0
    U = synth.random_su3_field(dims, 0.5, 0)
    A = dirac.hermitian_wilson(U, mu, m_w)
    Ad = A.toarray()
    x = synth.ones_source(dims)
    # one dense eigendecomposition: the exact result and the critical eigenpairs
    lam, Lv, Rv = sla.eig(Ad, left=True, right=True)
    ystar = Rv @ (np.sign(lam.real) * sla.lu_solve(sla.lu_factor(Rv), x.ravel()))
    idx = eigen.critical_order(lam)[:24]
    lam_m, R = lam[idx], Rv[:, idx] / np.linalg.norm(Rv[:, idx], axis=0)[None, :]
    L = Lv[:, idx]
    L = L / np.einsum("ni,ni->i", L.conj(), R).conj()[None, :]
    ms = (0, 8, 16, 24)
    ks = tuple(range(20, 321, 20))
    h = lattice(dims, U)
    try:
        defl = {m: ovl.ovl_set_deflation(h, mu, m_w, ovl.OVL_DEFL_LR, m, canon_cols(R[:, :m], dims),
                                         np.ascontiguousarray(lam_m[:m]), canon_cols(L[:, :m], dims))
                for m in ms if m}
        pairs = [(m, k) for m in ms for k in ks]
        params = [dict(mu=mu, m_w=m_w, k=k) for _, k in pairs]
        dl = [defl.get(m) for m, _ in pairs]
        y = np.zeros((len(pairs),) + x.shape, complex)
        infos = ovl.ovl_sign_apply(h, params, dl, np.stack([x] * len(pairs)), y)
        assert all(i["status"] == 0 for i in infos)
        err = {pk: rel(y[i].ravel(), ystar) for i, pk in enumerate(pairs)}
        # best approximation on span(R_m, K_k(A, x_minus)) at a few depths
        best = {}
        for m in (0, 24):
            xm = x.ravel() - R[:, :m] @ (L[:, :m].conj().T @ x.ravel())
            V = krylov.arnoldi(A, xm, max(ks))["V"]
            for k in (40, 120, 200):
                Q = np.hstack([R[:, :m], V[:, :k]]) if m else V[:, :k]
                best[(m, k)] = rel(krylov.best_approximation(Q, ystar), ystar)
        print("\nerror of the LR-deflated approximation, 4^4, x = 1, mu = 0.3 (rows k, columns m)")
        print("   k " + "".join(f"{m:>11d}" for m in ms))
        for k in ks:
            print(f"{k:4d} " + "".join(f"{err[(m, k)]:11.2e}" for m in ms))
        print("best approximation:", {key: f"{v:.2e}" for key, v in best.items()})
        kneed = {m: min([k for k in ks if err[(m, k)] <= 1e-8], default=None) for m in ms}
        print("k for 1e-8:", kneed)
        for m in ms:  # the error falls with the depth
            assert err[(m, ks[-1])] < 1e-3 * err[(m, ks[0])], m
        for k in (80, 160):  # deflation lowers the error at fixed depth
            assert err[(24, k)] < err[(0, k)], k
        reach = [kneed[m] if kneed[m] is not None else 10 ** 9 for m in ms]
        assert all(reach[i + 1] <= reach[i] for i in range(len(ms) - 1)), kneed
        assert kneed[24] is not None
        for (m, k), eb in best.items():  # close to the best approximation
            if eb > 1e-13:
                assert err[(m, k)] <= 10.0 * eb, (m, k, err[(m, k)], eb)
        for d in defl.values():
            ovl.ovl_destroy_deflation(d)
    finally:
        ovl.ovl_destroy_lattice(h)


@pytest.mark.late(2)
def test_error_vs_depth_lr_deflation_6x4_matches_the_oracle_table():
    """The 6^4 leg of the study (m up to 124 = 0.008 N): the CUDA path computes
    every (m, k) point of the oracle's stored table in one batched call, with
    the same critical eigenpairs (oracle.eigen.critical_sparse, recomputed
    here) and the exact y* recomputed by the oracle. Every error of the table
    down to 1e-10 is matched to 5 %, the depths for 1e-8 follow, and deflation
    lowers the depth the accuracy needs."""
    import json
    import os

    need_gpu()
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fig1_6x4_lr_table.json")))
    meta = ref["_meta"]
    dims, mu, m_w = (6, 6, 6, 6), meta["mu"], meta["m_w"]
    U = synth.random_su3_field(dims, meta["eps"], meta["seed"])
    A = dirac.hermitian_wilson(U, mu, m_w)
    Am = dirac.hermitian_wilson(U, -mu, m_w)
    x = synth.ones_source(dims)
    mcrit = ref["eigenpairs"]["m"]
    lam, R, L, _ = eigen.critical_sparse(A, Am, mcrit, nev=ref["eigenpairs"]["nev"])
    ystar = krylov.sign_lr(A, x.ravel(), ref["ystar"]["k_ref"], R, lam, L)
    # the exact result reproduces the stored one (probe sketch)
    P = synth.probe_vectors(ystar.size, len(ref["ystar"]["probe_re"]))
    sk = np.array(ref["ystar"]["probe_re"]) + 1j * np.array(ref["ystar"]["probe_im"])
    assert np.linalg.norm(P.conj() @ ystar - sk) <= 1e-10 * np.linalg.norm(sk)
    ms, ks = ref["ms"], ref["ks"]
    h = lattice(dims, U)
    try:
        defl = {m: ovl.ovl_set_deflation(h, mu, m_w, ovl.OVL_DEFL_LR, m, canon_cols(R[:, :m], dims),
                                         np.ascontiguousarray(lam[:m]), canon_cols(L[:, :m], dims))
                for m in ms if m}
        pairs = [(m, k) for m in ms for k in ks]
        params = [dict(mu=mu, m_w=m_w, k=k) for _, k in pairs]
        y = np.zeros((len(pairs),) + x.shape, complex)
        infos = ovl.ovl_sign_apply(h, params, [defl.get(m) for m, _ in pairs], np.stack([x] * len(pairs)), y)
        assert all(i["status"] == 0 for i in infos)
        err = {pk: rel(y[i].ravel(), ystar) for i, pk in enumerate(pairs)}
        print("\nerror of the LR-deflated approximation, 6^4, x = 1, mu = 0.3 (rows k, columns m): GPU / oracle")
        for j, k in enumerate(ks):
            print(f"{k:4d} " + "".join(f"{err[(m, k)]:10.2e} /{ref['rel_err'][str(m)][j]:9.2e}" for m in ms))
        for m in ms:
            for j, k in enumerate(ks):
                e_ref = ref["rel_err"][str(m)][j]
                if e_ref >= 1e-10:
                    assert abs(err[(m, k)] / e_ref - 1.0) < 0.05, (m, k, err[(m, k)], e_ref)
                else:
                    assert err[(m, k)] < 1e-9, (m, k, err[(m, k)], e_ref)
        kneed = {m: min([k for k in ks if err[(m, k)] <= 1e-8], default=None) for m in ms}
        print("k for 1e-8 (GPU):", kneed, " oracle:", ref["k_for_1e-8"])
        reach = [kneed[m] if kneed[m] is not None else 10 ** 9 for m in ms]
        assert all(reach[i + 1] <= reach[i] for i in range(len(ms) - 1)), kneed
        assert kneed[mcrit] is not None
        for d in defl.values():
            ovl.ovl_destroy_deflation(d)
    finally:
        ovl.ovl_destroy_lattice(h)
