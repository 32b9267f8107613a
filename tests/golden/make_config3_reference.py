"""Write the reference sketches of y* = sgn(H_w(mu)) b for the 16^3x32 workload.

Lattice 16^3x32 (N = 1,572,864), SU(3) links U = exp(i 0.3 X) seed 0,
m_w = -1.2, mu = 0.2; sources: spin-colour point sources at the origin.
Calls only the oracle and the seeded input generators.

y* is the oracle's undeflated Arnoldi approximation of Eq. 11 at a depth
where it has converged: one k_max-step Arnoldi run (Eq. 7, CGS2) gives, by
the nesting of the recurrence, the approximation of every depth k <= k_max
(the first k basis vectors and the leading k x k block of H_k), and the
result is accepted when the approximations at k_max - 100 and k_max agree to
< 1e-11 (the method converges to the exact result as k grows, Sec. 2).
Stored per source: |y*|, the inner products of y* with 64 seeded Gaussian
probe vectors, 16 sampled entries and the self-convergence gap.

Run:  python tests/golden/make_config3_reference.py [spin,colour ...]
      (default sources 0,0 and 2,1; about half an hour per source on 8 cores,
      30 GB of memory)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dirac, krylov, matfunc  # noqa: E402
from paper_0710_0341_gb300 import synth  # noqa: E402

DIMS, EPS, SEED, MW, MU = (16, 16, 16, 32), 0.3, 0, -1.2, 0.2
K_MAX, K_CHECK = 600, 500
NPROBE = 64


def approximation(r, k):
    """beta V_k sgn(H_k) e_1 from the leading part of a longer Arnoldi run."""
    F = matfunc.sign_eig(r["H"][:k, :k])
    return r["beta"] * (r["V"][:, :k] @ F[:, 0])


def main():
    out = os.path.join(HERE, "config3_ystar_sketch.json")
    data = json.load(open(out)) if os.path.exists(out) else {}
    srcs = [tuple(int(v) for v in a.split(",")) for a in sys.argv[1:]] or [(0, 0), (2, 1)]
    U = synth.random_su3_field(DIMS, EPS, SEED)
    A = dirac.hermitian_wilson(U, MU, MW)
    N = A.shape[0]
    idx = np.random.default_rng(99).choice(N, 16, replace=False)
    for s, c in srcs:
        key = f"{s},{c}"
        if key in data:
            continue
        b = synth.point_source(DIMS, s, c).ravel()
        t = time.time()
        r = krylov.arnoldi(A, b, K_MAX)
        y = approximation(r, K_MAX)
        y0 = approximation(r, K_CHECK)
        gap = float(np.linalg.norm(y - y0) / np.linalg.norm(y))
        print(f"source {key}: Arnoldi k={K_MAX} in {time.time() - t:.0f}s, gap k={K_CHECK}..{K_MAX}: {gap:.2e}",
              flush=True)
        del r, y0
        P = synth.probe_vectors(N, NPROBE)
        sk = P.conj() @ y
        del P
        data[key] = {
            "spin": s, "colour": c, "norm": float(np.linalg.norm(y)), "k_ref": K_MAX, "k_check": K_CHECK,
            "self_convergence_gap": gap,
            "probe_re": [float(v) for v in sk.real], "probe_im": [float(v) for v in sk.imag],
            "sample_index": [int(i) for i in idx],
            "sample_re": [float(y[i].real) for i in idx], "sample_im": [float(y[i].imag) for i in idx],
        }
        data["_meta"] = {
            "lattice": "16^3x32", "eps": EPS, "seed": SEED, "m_w": MW, "mu": MU,
            "source": "point source at the origin, spin s, colour c",
            "probes": f"synth.probe_vectors(N, {NPROBE}, seed=12345)",
            "method": "oracle Arnoldi (Eq. 11, no deflation), depth k_ref; self-convergence against depth k_check",
        }
        json.dump(data, open(out, "w"), indent=1)


if __name__ == "__main__":
    main()
