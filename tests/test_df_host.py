"""The double-float accumulation of df.cuh, built for the host, against exact
rational arithmetic.

Pass B of the Gram-Schmidt step, the deflation projections, the
recombination y = Q g and the Newton-Schulz products all accumulate complex
sums sum_k q_k g_k with q and g stored as FP32 hi + lo pairs (dfacc_mac), and
the Newton-Schulz update forms c - a b in the same arithmetic (dfc_fms); the
Gauss-Jordan Newton kernels divide by their pivots with dfc_inv. This holds
them to their error bounds on the CPU: the split of an FP64 value within
2^-48, a length-n accumulation within n 2^-47 of sum |q| |g| (observed about
sqrt(n) 2^-48), c - a b within 2^-45 of |a| |b| + |c|, and 1 / z within
2^-44 of |1 / z|."""
import ctypes
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hostcheck", "df_host.cu")
DEP = os.path.join(os.path.dirname(HERE), "paper_0710_0341_gb300", "csrc", "df.cuh")
OUT = os.path.join(HERE, "hostcheck", "_build", "libdf_host.so")


@pytest.fixture(scope="module")
def lib():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    if not os.path.exists(OUT) or max(os.path.getmtime(SRC), os.path.getmtime(DEP)) > os.path.getmtime(OUT):
        os.makedirs(os.path.dirname(OUT), exist_ok=True)
        subprocess.run([nvcc, "-x", "cu", "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared", SRC, "-o", OUT], check=True)
    L = ctypes.CDLL(OUT)
    P = ctypes.c_void_p
    L.host_dfacc_dot.argtypes = [P, P, P, P, ctypes.c_int, P]
    L.host_dfc_fms.argtypes = [P, P, P, P]
    L.host_split_d.argtypes = [P, P, ctypes.c_int]
    L.host_dfc_inv.argtypes = [P, P]
    for f in (L.host_dfacc_dot, L.host_dfc_fms, L.host_split_d, L.host_dfc_inv):
        f.restype = None
    return L


def _split(lib, x):
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    out = np.zeros(2 * x.size, np.float32)
    lib.host_split_d(x.ctypes.data, out.ctypes.data, x.size)
    return np.ascontiguousarray(out[0::2]), np.ascontiguousarray(out[1::2])


def _F(v):
    return Fraction(float(v))


def test_split_of_fp64_values(lib):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(5000) * np.exp(rng.uniform(-30, 30, 5000))
    hi, lo = _split(lib, x)
    err = np.array([abs(_F(h) + _F(l) - _F(v)) for h, l, v in zip(hi, lo, x)], dtype=float)
    assert np.all(err <= 2.0 ** -48 * np.abs(x))
    assert np.all(np.abs(lo) <= 2.0 ** -24 * np.abs(hi))


@pytest.mark.parametrize("n", [1, 37, 400])
def test_complex_accumulation_against_exact_sums(lib, n):
    rng = np.random.default_rng(n)
    worst = 0.0
    for trial in range(10):
        q = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * np.exp(rng.uniform(-3, 3, n))
        g = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * np.exp(rng.uniform(-3, 3, n))
        qh, ql = _split(lib, np.column_stack([q.real, q.imag]))
        gh, gl = _split(lib, np.column_stack([g.real, g.imag]))
        out = np.zeros(2)
        lib.host_dfacc_dot(qh.ctypes.data, ql.ctypes.data, gh.ctypes.data, gl.ctypes.data, n, out.ctypes.data)
        # exact value of the sum of the stored (hi + lo) operands
        re = im = Fraction(0)
        scale = 0.0
        for k in range(n):
            qr, qi = _F(qh[2 * k]) + _F(ql[2 * k]), _F(qh[2 * k + 1]) + _F(ql[2 * k + 1])
            gr, gi = _F(gh[2 * k]) + _F(gl[2 * k]), _F(gh[2 * k + 1]) + _F(gl[2 * k + 1])
            re += qr * gr - qi * gi
            im += qr * gi + qi * gr
            scale += abs(q[k]) * abs(g[k])
        e = max(abs(_F(out[0]) - re), abs(_F(out[1]) - im))
        assert float(e) <= n * 2.0 ** -47 * scale, (n, trial, float(e) / scale)
        worst = max(worst, float(e) / scale)
    # observed: about sqrt(n) 2^-48 (1.1 to 2.2 sqrt(n) 2^-48 for these seeds), far inside the bound
    assert worst <= 8.0 * np.sqrt(n) * 2.0 ** -48


def test_fused_multiply_subtract_against_exact(lib):
    rng = np.random.default_rng(3)
    for _ in range(500):
        vals = rng.standard_normal(6) * np.exp(rng.uniform(-4, 4, 6))
        h, lo = _split(lib, vals)
        c = np.array([h[0], h[1], lo[0], lo[1]], np.float32)
        a = np.array([h[2], h[3], lo[2], lo[3]], np.float32)
        b = np.array([h[4], h[5], lo[4], lo[5]], np.float32)
        out = np.zeros(4, np.float32)
        lib.host_dfc_fms(c.ctypes.data, a.ctypes.data, b.ctypes.data, out.ctypes.data)
        cr, ci = _F(c[0]) + _F(c[2]), _F(c[1]) + _F(c[3])
        ar, ai = _F(a[0]) + _F(a[2]), _F(a[1]) + _F(a[3])
        br, bi = _F(b[0]) + _F(b[2]), _F(b[1]) + _F(b[3])
        xr, xi = cr - (ar * br - ai * bi), ci - (ar * bi + ai * br)
        scale = abs(complex(vals[2], vals[3])) * abs(complex(vals[4], vals[5])) + abs(complex(vals[0], vals[1]))
        er = abs(_F(out[0]) + _F(out[2]) - xr)
        ei = abs(_F(out[1]) + _F(out[3]) - xi)
        assert float(max(er, ei)) <= 2.0 ** -45 * scale
        # the result is renormalised: the low part is below one unit of the high part
        assert abs(out[2]) <= 2.0 ** -23 * abs(out[0]) + 1e-45 and abs(out[3]) <= 2.0 ** -23 * abs(out[1]) + 1e-45


def test_pivot_reciprocal_against_exact(lib):
    rng = np.random.default_rng(11)
    worst = 0.0
    for _ in range(2000):
        v = rng.standard_normal(2) * np.exp(rng.uniform(-20, 20))
        if rng.random() < 0.1:  # nearly real or nearly imaginary pivots
            v[rng.integers(2)] *= 1e-9
        h, lo = _split(lib, v)
        z = np.array([h[0], h[1], lo[0], lo[1]], np.float32)
        out = np.zeros(4, np.float32)
        lib.host_dfc_inv(z.ctypes.data, out.ctypes.data)
        zr, zi = _F(z[0]) + _F(z[2]), _F(z[1]) + _F(z[3])
        n2 = zr * zr + zi * zi
        xr, xi = zr / n2, -zi / n2  # exact 1 / z
        mag = float(abs(complex(float(xr), float(xi))))
        e = float(max(abs(_F(out[0]) + _F(out[2]) - xr), abs(_F(out[1]) + _F(out[3]) - xi)))
        assert e <= 2.0 ** -44 * mag, (v, e / mag)
        worst = max(worst, e / mag)
    assert worst > 0.0  # a double-float result, not an exact one by accident
