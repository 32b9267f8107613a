"""The stencil kernels' site arithmetic, run on the host, against the oracle.

tests/hostcheck/stencil_host.cu builds the same templates the kernels of
dslash.cu instantiate (dslash_site.cuh, and the double-float type of dd.cuh)
for the CPU. This checks on the CPU the neighbour indexing, the spin
projections, the link layouts (FP64, FP32 18-real, 12-real with the third row
rebuilt) and the arithmetic of each instantiation against the oracle's sparse
H_w(mu) (Eq. 2), and pins the double-float conversions and operations to
their error bounds. The device layouts are rebuilt here from their
definitions: packed spinor pos(cc, site) = ((cc >> 1) V + site) 2 + (cc & 1),
links per direction and entry pair, site-minor."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import dirac
from paper_0710_0341_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hostcheck", "stencil_host.cu")
CSRC = os.path.join(os.path.dirname(HERE), "paper_0710_0341_gb300", "csrc")
OUT = os.path.join(HERE, "hostcheck", "_build", "libstencil_host.so")


@pytest.fixture(scope="module")
def lib():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    deps = [SRC] + [os.path.join(CSRC, f) for f in ("dslash_site.cuh", "dd.cuh", "df.cuh")]
    if not os.path.exists(OUT) or any(os.path.getmtime(d) > os.path.getmtime(OUT) for d in deps):
        os.makedirs(os.path.dirname(OUT), exist_ok=True)
        subprocess.run([nvcc, "-x", "cu", "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared", SRC, "-o", OUT], check=True)
    L = ctypes.CDLL(OUT)
    P = ctypes.c_void_p
    L.host_apply_hw.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, P, P, P, P]
    L.host_apply_hw.restype = ctypes.c_int
    L.host_dd_ops.argtypes = [P, P, P, P, P, ctypes.c_int]
    L.host_dd_ops.restype = None
    return L


def _ptr(a):
    return a.ctypes.data if a is not None else None


def _pack_spinor(psi, dtype):
    V = psi.size // 12
    return np.ascontiguousarray(psi.reshape(V, 6, 2).transpose(1, 0, 2), dtype=dtype)


def _unpack_spinor(p, shape):
    V = p.size // 12
    return np.ascontiguousarray(p.reshape(6, V, 2).transpose(1, 0, 2)).astype(np.complex128).reshape(shape)


def _links(U, mode):
    V = U.size // 36
    Us = U.reshape(V, 4, 9)  # site, direction, entry 3a + b
    if mode in (0, 1):
        return np.ascontiguousarray(Us.transpose(1, 2, 0)), None  # double2[(nu*9 + e) V + site]
    if mode == 2:  # float4[(nu*4 + p) V + site] = entries (2p, 2p+1); float2[nu V + site] = entry 8
        a = np.ascontiguousarray(Us[:, :, :8].reshape(V, 4, 4, 2).transpose(1, 2, 0, 3), dtype=np.complex64)
        b = np.ascontiguousarray(Us[:, :, 8].T, dtype=np.complex64)
        return a, b
    # 12 reals: float4[(nu*3 + p) V + site] = entries (2p, 2p+1) of rows 0, 1
    return np.ascontiguousarray(Us[:, :, :6].reshape(V, 4, 3, 2).transpose(1, 2, 0, 3), dtype=np.complex64), None


def _apply(lib, U, psi, mu, m_w, apbc, mode):
    dims = np.array(U.shape[:4][::-1], dtype=np.int32)  # Lx, Ly, Lz, Lt
    la, lb = _links(U, mode)
    dt = np.complex128 if mode in (0, 1) else np.complex64
    x = _pack_spinor(psi, dt)
    y = np.zeros_like(x)
    rc = lib.host_apply_hw(_ptr(dims), int(apbc), mu, 1.0 / (8.0 + 2.0 * m_w), mode, _ptr(la), _ptr(lb),
                           _ptr(x), _ptr(y))
    assert rc == 0
    return _unpack_spinor(y, psi.shape)


@pytest.mark.parametrize("dims,apbc,mu", [((4, 4, 4, 4), 0, 0.3), ((3, 4, 2, 5), 1, 0.6), ((2, 2, 2, 2), 0, 0.0)])
def test_site_arithmetic_matches_the_oracle(lib, dims, apbc, mu):
    m_w = -1.1
    U = synth.random_su3_field(dims, 0.5, 2)
    psi = synth.gaussian_source(dims, 4)
    ref = dirac.apply(dirac.hermitian_wilson(U, mu, m_w, antiperiodic_t=bool(apbc)), psi)
    nrm = np.linalg.norm(ref)
    e64 = np.linalg.norm(_apply(lib, U, psi, mu, m_w, apbc, 0) - ref) / nrm
    edd = np.linalg.norm(_apply(lib, U, psi, mu, m_w, apbc, 1) - ref) / nrm
    e32 = np.linalg.norm(_apply(lib, U, psi, mu, m_w, apbc, 2) - ref) / nrm
    e12 = np.linalg.norm(_apply(lib, U, psi, mu, m_w, apbc, 3) - ref) / nrm
    assert e64 < 1e-15, e64
    assert edd < 2e-14, edd  # double-float: about 2^-46 per operation
    assert e32 < 1e-6 and e12 < 1e-6, (e32, e12)


def test_double_float_is_not_fp64_in_disguise(lib):
    """The double-float instantiation differs from FP64 at its own rounding
    level (so it really computes in hi + lo FP32), while agreeing to 2e-14."""
    dims = (4, 4, 4, 4)
    U = synth.random_su3_field(dims, 0.5, 2)
    psi = synth.gaussian_source(dims, 4)
    a = _apply(lib, U, psi, 0.3, -1.1, 0, 0)
    b = _apply(lib, U, psi, 0.3, -1.1, 0, 1)
    d = np.linalg.norm(a - b) / np.linalg.norm(a)
    assert 1e-17 < d < 2e-14, d


def test_double_float_conversion_and_operations(lib):
    rng = np.random.default_rng(7)
    n = 4000
    x = rng.standard_normal(n) * np.exp(rng.uniform(-60, 60, n))
    x[:8] = [0.0, -0.0, 1.0, -1.0, 2.0 ** -100, 2.0 ** -130, 3.0e38, -7.5]
    a = rng.standard_normal(n) * np.exp(rng.uniform(-8, 8, n))
    b = rng.standard_normal(n) * np.exp(rng.uniform(-8, 8, n))
    c = rng.standard_normal(n) * np.exp(rng.uniform(-8, 8, n))
    out = np.zeros(5 * n)
    lib.host_dd_ops(_ptr(x), _ptr(a), _ptr(b), _ptr(c), _ptr(out), n)
    out = out.reshape(n, 5)
    big = np.abs(x) >= 2.0 ** -80
    # conversion: 47 leading bits kept (truncation), below 2^-80 the high part only
    assert np.all(np.abs(out[big, 0] - x[big]) <= 2.0 ** -46 * np.abs(x[big]))
    small = (np.abs(x) < 2.0 ** -80) & (np.abs(x) >= 2.0 ** -126)
    assert np.all(np.abs(out[small, 0] - x[small]) <= 2.0 ** -23 * np.abs(x[small]))
    assert out[5, 0] == 0.0  # below 2^-126
    # operations: error within a few 2^-46 of the operands' size
    u = 2.0 ** -44
    assert np.all(np.abs(out[:, 1] - (a + b)) <= u * (np.abs(a) + np.abs(b)))
    assert np.all(np.abs(out[:, 2] - (a - b)) <= u * (np.abs(a) + np.abs(b)))
    assert np.all(np.abs(out[:, 3] - a * b) <= u * np.abs(a * b))
    assert np.all(np.abs(out[:, 4] - (a * b + c)) <= u * (np.abs(a * b) + np.abs(c)))
    # and it is more than FP32: most products carry bits below 2^-24
    assert np.mean(np.abs(out[:, 3] - a * b) <= 2.0 ** -30 * np.abs(a * b)) > 0.99
    # NaN and overflow
    nan_inf = np.array([np.nan, np.inf, -1e300])
    o2 = np.zeros(15)
    lib.host_dd_ops(_ptr(nan_inf), _ptr(np.ones(3)), _ptr(np.ones(3)), _ptr(np.ones(3)), _ptr(o2), 3)
    assert np.isnan(o2[0]) and o2[5] == np.inf and o2[10] == -np.inf


class _HostOperator:
    """H_w(mu) applied by a host build of one stencil instantiation (for the
    oracle's Arnoldi, which takes anything with A @ v)."""

    def __init__(self, lib, U, mu, m_w, mode):
        self.lib, self.U, self.mu, self.m_w, self.mode = lib, U, mu, m_w, mode
        self.shape = U.shape[:4] + (4, 3)

    def __matmul__(self, v):
        return _apply(self.lib, self.U, np.asarray(v).reshape(self.shape), self.mu, self.m_w, 0, self.mode).ravel()


def test_sign_function_with_double_float_matvecs(lib):
    """What the FP64 mode's result would lose with the double-float stencil: the
    oracle's deflated and undeflated approximations of sgn(H_w) b driven by the
    host build of that stencil differ from those with the exact operator by far
    less than the 1e-10 parity bar."""
    from oracle import eigen, krylov

    dims, mu, m_w = (2, 2, 2, 4), 0.3, -1.0
    U = synth.random_su3_field(dims, 0.5, 0)
    A = dirac.hermitian_wilson(U, mu, m_w)
    Add = _HostOperator(lib, U, mu, m_w, 1)
    b = synth.gaussian_source(dims, 1).ravel()
    lam, R, L = eigen.critical_dense(A.toarray(), 16)
    S, T = eigen.schur_from_right(A, R[:, :12])
    for f in (lambda Op: krylov.sign_arnoldi(Op, b, 80),
              lambda Op: krylov.sign_lr(Op, b, 60, R, lam, L),
              lambda Op: krylov.sign_schur_block(Op, b, 60, S, T)):
        y, ydd = f(A), f(Add)
        d = np.linalg.norm(ydd - y) / np.linalg.norm(y)
        assert d < 1e-12, d
