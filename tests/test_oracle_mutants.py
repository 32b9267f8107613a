"""Planted mistakes in the oracle are caught by its pins.

Each case plants one slip of the kind a restatement of the paper could
plausibly contain (a flipped sign, a dropped conjugate, factor or term, a
transposed operand, a wrong index) in a copy of one oracle module, loads the
copy in place of that module inside a child pytest process, and runs the pin
files that guard the step: at least one pin must fail. The oracle's files
are never modified; everything runs on the CPU.
"""
import concurrent.futures as cf
import json
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))

OP, SIGN, KRY, OVL, MLP = ("test_oracle_operator.py", "test_oracle_sign.py", "test_oracle_krylov.py",
                           "test_oracle_overlap.py", "test_oracle_mlp.py")
JOR = "test_oracle_jordan.py"

# (name, module, text in the oracle, planted replacement, pin files)
CASES = [
    # Eq. 2, the operator
    ("mu sign on the forward time hop", "oracle.dirac",
     "wf = np.exp(mu) if nu == 3", "wf = np.exp(-mu) if nu == 3", [OP]),
    ("(1 - gamma) on the forward hop", "oracle.dirac", "Pp = eye4 + GAMMA[nu]", "Pp = eye4 - GAMMA[nu]", [OP]),
    ("U^T instead of U^dag on the backward hop", "oracle.dirac",
     "Ubw = np.conj(np.swapaxes(Uf[nb, nu], -1, -2))", "Ubw = np.swapaxes(Uf[nb, nu], -1, -2)", [OP]),
    ("backward link taken at n instead of n - nu", "oracle.dirac",
     "Ubw = np.conj(np.swapaxes(Uf[nb, nu], -1, -2))", "Ubw = np.conj(np.swapaxes(Uf[n, nu], -1, -2))", [OP]),
    ("forward link transposed", "oracle.dirac",
     'np.einsum("st,nab->nsatb", Pp, Ufw)', 'np.einsum("st,nba->nsatb", Pp, Ufw)', [OP]),
    ("antiperiodic sign dropped on the backward hop", "oracle.dirac",
     "sb = np.where(coords[3] == 0, -1.0, 1.0)", "sb = np.ones(V)", [OP]),
    ("kappa = 1/(8 + m_w)", "oracle.dirac", "return 1.0 / (8.0 + 2.0 * m_w)", "return 1.0 / (8.0 + m_w)", [OP]),
    ("gamma5 as gamma1 gamma2 gamma4 gamma3", "oracle.dirac",
     "GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]", "GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[3] @ GAMMA[2]",
     [OP]),
    ("row evaluation: link not transposed", "oracle.dirac",
     "acc += sign * w * (proj @ nb @ link.T)", "acc += sign * w * (proj @ nb @ link)", [OP]),
    # Eqs. 4-6, the sign function
    ("U^dag instead of U^-1", "oracle.matfunc",
     "return (U * s[None, :]) @ np.linalg.inv(U)", "return (U * s[None, :]) @ U.conj().T", [SIGN]),
    ("sgn(Im) instead of sgn(Re)", "oracle.matfunc",
     "    s = np.sign(lam.real)\n", "    s = np.sign(lam.imag)\n", [SIGN]),
    ("signs scaled on the wrong index", "oracle.matfunc",
     "return (U * s[None, :]) @ np.linalg.inv(U)", "return (U * s[:, None]) @ np.linalg.inv(U)", [SIGN]),
    ("Newton: scaling applied twice", "oracle.matfunc",
     "Xn = 0.5 * (c * X + Xi / c)", "Xn = 0.5 * (c * X + Xi * c)", [SIGN]),
    # the Jordan-form definition (Sec. 1, after Eq. 4)
    ("Jordan: 1/j instead of 1/j!", "oracle.matfunc", "                fact *= j\n", "                fact = j\n",
     [JOR]),
    ("Jordan: ones below instead of above the diagonal", "oracle.matfunc",
     "J[o + i, o + i + 1] = 1.0", "J[o + i + 1, o + i] = 1.0", [JOR]),
    ("Jordan: X^-1 f(J) X", "oracle.matfunc", "return X @ F @ np.linalg.inv(X)",
     "return np.linalg.inv(X) @ F @ X", [JOR]),
    ("Jordan: sgn keeps a first-derivative term", "oracle.matfunc",
     "np.sign(np.real(lam)) if j == 0 else 0.0", "np.sign(np.real(lam)) if j == 0 else (0.5 if j == 1 else 0.0)",
     [JOR]),
    ("free field: mu enters p4 with the wrong sign", "oracle.freefield",
     "pt = [X, Y, Z, T - 1j * mu]", "pt = [X, Y, Z, T + 1j * mu]", [OP, SIGN]),
    ("free field: factor 4 kappa^2 halved", "oracle.freefield",
     "om2 = a * a + 4.0 * kap * kap", "om2 = a * a + 2.0 * kap * kap", [OP, SIGN]),
    # Eqs. 7-22, Arnoldi and deflation
    ("Gram-Schmidt without the conjugate", "oracle.krylov",
     "dh = V[:, : j + 1].conj().T @ w", "dh = V[:, : j + 1].T @ w", [KRY]),
    ("subdiagonal of H negated", "oracle.krylov", "H[j + 1, j] = bk", "H[j + 1, j] = -bk", [KRY]),
    ("first row instead of first column of f(H)", "oracle.krylov",
     'return r["beta"] * (r["V"] @ F[:, 0])', 'return r["beta"] * (r["V"] @ F[0, :])', [KRY]),
    ("Schur projection with + instead of -", "oracle.krylov",
     "x_perp = x - S @ xs  # (1 - S S^dag) x", "x_perp = x + S @ xs  # (1 - S S^dag) x", [KRY]),
    ("Sylvester right-hand side negated", "oracle.krylov",
     "fT @ X - X @ fH", "X @ fH - fT @ X", [KRY]),
    ("beta e_1 placed at the last index", "oracle.krylov", "e1[0] = beta", "e1[-1] = beta", [KRY]),
    ("coupling block X of Eq. 15 dropped", "oracle.krylov", '    H[:m, m:] = r["X"]\n', "", [KRY]),
    ("L^T instead of L^dag", "oracle.krylov", "g = L.conj().T @ x", "g = L.T @ x", [KRY]),
    ("sgn of Im Lambda in Eq. 22", "oracle.krylov",
     "defl = R @ (np.sign(np.asarray(Lam).real) * g)", "defl = R @ (np.sign(np.asarray(Lam).imag) * g)", [KRY]),
    # Eqs. 13 and 20, eigenpairs
    ("left vectors normalised without the conjugate", "oracle.eigen",
     "L = L / d.conj()[None, :]", "L = L / d[None, :]", [KRY]),
    ("critical = smallest Re instead of |Re|", "oracle.eigen",
     "np.abs(lam.imag), np.abs(lam.real)))", "np.abs(lam.imag), lam.real))", [KRY]),
    ("Schur block without the conjugate", "oracle.eigen", "T0 = Q.conj().T @ AQ", "T0 = Q.T @ AQ", [KRY]),
    ("left vectors paired with lambda instead of conj(lambda)", "oracle.eigen",
     "np.abs(lamL - np.conj(z))", "np.abs(lamL - z)", [KRY]),
    ("Rayleigh-Ritz without the conjugate", "oracle.eigen",
     "lam, Y = np.linalg.eig(Q.conj().T @ AQ)", "lam, Y = np.linalg.eig(Q.T @ AQ)", [KRY]),
    # Eq. 1, the overlap operator
    ("gamma5 = diag(-1, -1, 1, 1)", "oracle.overlap", "y[..., 2:, :] *= -1.0", "y[..., :2, :] *= -1.0", [OVL]),
    ("adjoint with gamma5 on the wrong side", "oracle.overlap",
     "return x + sign_apply_minus_mu(gamma5_apply(x))", "return x + gamma5_apply(sign_apply_minus_mu(x))", [OVL]),
    ("adjoint eigenvalues not conjugated", "oracle.overlap",
     "return np.conj(lam), L, R", "return lam, L, R", [OVL]),
    # the predictor's reference network
    ("ReLU derivative dropped", "oracle.mlp", "dz2 = dh2 * (z2 > 0)", "dz2 = dh2", [MLP]),
    ("under-prediction weight on over-prediction", "oracle.mlp",
     "w = np.where(Y < T, under_weight, 1.0)", "w = np.where(Y > T, under_weight, 1.0)", [MLP]),
]


def _run(case):
    name, module, old, new, pins = case
    env = dict(os.environ, ORACLE_MUTANT=json.dumps({"module": module, "old": old, "new": new}),
               OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")  # one BLAS thread per child
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        *[os.path.join(HERE, p) for p in pins]], capture_output=True, text=True, env=env,
                       cwd=os.path.dirname(HERE), timeout=600)
    return r.returncode, (r.stdout + r.stderr)[-600:]


def test_every_planted_mistake_fails_a_pin():
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(_run, CASES))
    missed = [(c[0], rc, out) for c, (rc, out) in zip(CASES, results) if rc != 1]
    # rc 1: a pin failed; 0 would mean the mistake went unnoticed, anything else a broken harness
    assert not missed, missed


def test_unplanted_copies_pass_every_pin():
    """The harness alone changes nothing: each module swapped for an unchanged
    copy of itself passes all the pin files."""
    mods = ["oracle.dirac", "oracle.matfunc", "oracle.freefield", "oracle.krylov", "oracle.eigen",
            "oracle.overlap", "oracle.mlp"]
    same = "TEST INFRASTRUCTURE ONLY"
    cases = [("unchanged " + m, m, same, same, [OP, SIGN, KRY, OVL, MLP, JOR]) for m in mods]
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(_run, cases))
    bad = [(c[0], rc, out) for c, (rc, out) in zip(cases, results) if rc != 0]
    assert not bad, bad
