"""Write the reference sketches of y* = sgn(H_w(mu)) b for the 8^4 workload.

Calls only the oracle and the seeded input generators. For each mu the
critical eigenvectors come from ARPACK (scipy.sparse.linalg.eigs) on A^2
(smallest real part), the Schur deflation of Eq. 19 then runs with growing
Krylov depth until two successive depths agree to < 1e-11 (the method
converges to the exact result as k grows, Sec. 2). Stored per mu: |y*|, the
inner products of y* with 64 seeded Gaussian probe vectors, 16 sampled
entries and the self-convergence gap.

Run:  python tests/golden/make_config2_reference.py  (about an hour on 8 cores)
"""
import json
import os
import sys
import time

import numpy as np
import scipy.sparse.linalg as spla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dirac, eigen, krylov  # noqa: E402
from paper_0710_0341_gb300 import synth  # noqa: E402

DIMS, EPS, SEED, MW = (8, 8, 8, 8), 0.4, 0, -1.0
MUS = [0.0, 0.1, 0.3, 0.6]
NPROBE = 64


def reference(mu, log):
    U = synth.random_su3_field(DIMS, EPS, SEED)
    A = dirac.hermitian_wilson(U, mu, MW)
    N = A.shape[0]
    b = synth.gaussian_source(DIMS, 1).ravel()
    B = spla.LinearOperator((N, N), matvec=lambda v: A @ (A @ v), dtype=np.complex128)
    t = time.time()
    _, W = spla.eigs(B, k=70, which="SR", ncv=240, tol=1e-13, maxiter=200000)
    Q, _ = np.linalg.qr(W)
    AQ = np.column_stack([A @ Q[:, i] for i in range(Q.shape[1])])
    lam, Y = np.linalg.eig(Q.conj().T @ AQ)
    order = eigen.critical_order(lam)
    m = 60
    R = (Q @ Y)[:, order[:m]]
    S, T = eigen.schur_from_right(A, R)
    res = np.linalg.norm(np.column_stack([A @ S[:, i] for i in range(m)]) - S @ T) / np.sqrt(m)
    log(f"mu={mu}: eigs {time.time() - t:.0f}s, |Re lam| {abs(lam[order[0]].real):.4f}..{abs(lam[order[m - 1]].real):.4f}, "
        f"|AS-ST| {res:.1e}")
    prev, k = None, 300
    while True:
        t = time.time()
        y = krylov.sign_schur(A, b, k, S, T)
        gap = None if prev is None else float(np.linalg.norm(y - prev) / np.linalg.norm(y))
        log(f"mu={mu}: k_ref={k} ({time.time() - t:.0f}s) gap to previous {gap}")
        if gap is not None and gap < 1e-11:
            return y, k, gap, float(res)
        prev, k = y, k + 150
        if k > 1200:
            return y, k - 150, gap, float(res)


def main():
    out = os.path.join(HERE, "config2_ystar_sketch.json")
    data = json.load(open(out)) if os.path.exists(out) else {}
    P = synth.probe_vectors(12 * 8 ** 4, NPROBE)
    idx = np.random.default_rng(99).choice(12 * 8 ** 4, 16, replace=False)
    for mu in MUS:
        key = f"{mu}"
        if key in data:
            continue
        y, k, gap, res = reference(mu, lambda s: print(s, flush=True))
        sk = P.conj() @ y
        data[key] = {
            "mu": mu, "norm": float(np.linalg.norm(y)), "k_ref": k, "m_ref": 60, "self_convergence_gap": gap,
            "schur_residual": res,
            "probe_re": [float(v) for v in sk.real], "probe_im": [float(v) for v in sk.imag],
            "sample_index": [int(i) for i in idx],
            "sample_re": [float(y[i].real) for i in idx], "sample_im": [float(y[i].imag) for i in idx],
        }
        meta = {"lattice": "8^4", "eps": EPS, "seed": SEED, "m_w": MW, "source": "gaussian seed 1",
                "probes": f"synth.probe_vectors(N, {NPROBE}, seed=12345)",
                "method": "oracle Schur deflation (Eq. 19), ARPACK critical vectors of A^2, k_ref grown to self-convergence"}
        data["_meta"] = meta
        json.dump(data, open(out, "w"), indent=1)


if __name__ == "__main__":
    main()
