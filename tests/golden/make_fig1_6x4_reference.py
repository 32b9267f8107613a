"""Write the 6^4 leg of the convergence study of Sec. 5 (Fig. 1 setting).

The paper shows the error of the LR-deflated approximation of sgn(H_w) x
against the Krylov depth k for several m, with x = (1, ..., 1) and mu = 0.3,
on a 4^4 and a 6^4 lattice, and observes that at m ~ 0.008 N the depth needed
for 1e-8 grows only slightly with the lattice (their gauge fields are not
available; a seeded synthetic field stands in, eps 0.5, seed 0, m_w -1).

Calls only the oracle and the seeded input generators:
  * the 124 (= 0.008 N) critical eigenpairs with left vectors,
    oracle.eigen.critical_sparse (ARPACK on A^2, Rayleigh-Ritz, Eq. 20);
  * y* = sgn(H_w) x by the oracle's LR approximation (Eq. 22) with all 124
    vectors, the depth grown until two successive depths agree to < 1e-12
    (the approximation converges to the exact result, Sec. 2);
  * the relative error eps(k, m) = |y(k, m) - y*| / |y*| of the oracle's LR
    approximation for m in {0, 41, 83, 124}, k = 20, 40, ..., 400 (m = 0 is
    the undeflated Arnoldi approximation of Eq. 11), the first k on that grid
    with eps <= 1e-8, and the best approximation on span(R_m) + K_k at a few
    points;
  * |y*| and the inner products of y* with 64 seeded Gaussian probe vectors.

Run:  python tests/golden/make_fig1_6x4_reference.py   (about 10 minutes on 8 cores)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dirac, eigen, krylov  # noqa: E402
from paper_0710_0341_gb300 import synth  # noqa: E402

DIMS, EPS, SEED, MW, MU = (6, 6, 6, 6), 0.5, 0, -1.0, 0.3
M_CRIT = 124                       # 0.008 N, N = 15552
MS = (0, 41, 83, 124)
KS = tuple(range(20, 401, 20))
NPROBE = 64
OUT = os.path.join(HERE, "fig1_6x4_lr_table.json")


def main():
    log = lambda s: print(s, flush=True)  # noqa: E731
    U = synth.random_su3_field(DIMS, EPS, SEED)
    A = dirac.hermitian_wilson(U, MU, MW)
    Am = dirac.hermitian_wilson(U, -MU, MW)
    N = A.shape[0]
    x = synth.ones_source(DIMS).ravel()
    t = time.time()
    lam, R, L, res = eigen.critical_sparse(A, Am, M_CRIT, nev=150)
    lr_err = float(np.abs(L.conj().T @ R - np.eye(M_CRIT)).max())
    log(f"eigenpairs {time.time() - t:.0f}s: |Re| {abs(lam[0].real):.4f}..{abs(lam[-1].real):.4f}, "
        f"max residual {res.max():.1e}, |L^dag R - I| {lr_err:.1e}")
    prev, k_ref, gap = None, 300, None
    while True:
        y = krylov.sign_lr(A, x, k_ref, R, lam, L)
        if prev is not None:
            gap = float(np.linalg.norm(y - prev) / np.linalg.norm(y))
            log(f"y*: k={k_ref} gap to k={k_ref - 100}: {gap:.2e}")
            if gap < 1e-12 or k_ref >= 800:
                break
        prev, k_ref = y, k_ref + 100
    ystar = y
    nrm = float(np.linalg.norm(ystar))
    err = {}
    for m in MS:
        for k in KS:
            yk = (krylov.sign_lr(A, x, k, R[:, :m], lam[:m], L[:, :m]) if m else krylov.sign_arnoldi(A, x, k))
            err[(m, k)] = float(np.linalg.norm(yk - ystar) / nrm)
        log(f"m={m}: " + " ".join(f"{err[(m, k)]:.1e}" for k in KS))
    kneed = {m: next((k for k in KS if err[(m, k)] <= 1e-8), None) for m in MS}
    best = {}
    for m, k in ((0, 200), (124, 80), (124, 120)):
        Q = krylov.lr_search_space(A, x, k, R[:, :m], L[:, :m])
        best[f"{m},{k}"] = float(np.linalg.norm(krylov.best_approximation(Q, ystar) - ystar) / nrm)
    log(f"k for 1e-8: {kneed}; best approximation {best}")
    P = synth.probe_vectors(N, NPROBE)
    sk = P.conj() @ ystar
    data = {
        "_meta": {"lattice": "6^4", "N": N, "eps": EPS, "seed": SEED, "m_w": MW, "mu": MU,
                  "source": "x = (1, ..., 1)", "scheme": "LR (Eq. 22)",
                  "method": "oracle LR approximation; y* by self-convergence with the 124 critical pairs",
                  "probes": f"synth.probe_vectors(N, {NPROBE}, seed=12345)"},
        "eigenpairs": {"m": M_CRIT, "nev": 150, "abs_re_min": float(abs(lam[0].real)),
                       "abs_re_max": float(abs(lam[-1].real)), "max_residual": float(res.max()),
                       "lr_biorth_err": lr_err},
        "ystar": {"k_ref": k_ref, "self_convergence_gap": gap, "norm": nrm,
                  "probe_re": [float(v) for v in sk.real], "probe_im": [float(v) for v in sk.imag]},
        "ms": list(MS), "ks": list(KS),
        "rel_err": {str(m): [err[(m, k)] for k in KS] for m in MS},
        "k_for_1e-8": {str(m): kneed[m] for m in MS},
        "best_approximation": best,
    }
    json.dump(data, open(OUT, "w"), indent=1)
    log(f"wrote {OUT}")


if __name__ == "__main__":
    main()
