"""Planted mistakes in the stencil's site arithmetic are caught by the host check.

Each case copies the kernel headers (dslash_site.cuh, dd.cuh, df.cuh, ovl.h) and the
host harness into a scratch tree, plants one slip in the copy, builds the
harness against it and runs the comparison of tests/test_stencil_host.py for
the instantiation it touches: the planted copy must miss the oracle by far
more than that instantiation's bound. The repository's files are never
modified; everything runs on the CPU.
"""
import concurrent.futures as cf
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import test_stencil_host as hc
from oracle import dirac
from paper_0710_0341_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0710_0341_gb300", "csrc")

# (name, header, text, planted replacement, mode, bound the plant must exceed)
CASES = [
    ("(1 - gamma_x) on the forward x hop", "dslash_site.cuh",
     "h[c] = FWD ? p0 + ti(p3) : p0 - ti(p3);", "h[c] = FWD ? p0 - ti(p3) : p0 - ti(p3);", 0, 1e-15),
    ("e^{+mu} and e^{-mu} swapped", "dslash_site.cuh", "T wtp = wp, wtm = wm;", "T wtp = wm, wtm = wp;", 0, 1e-15),
    ("U instead of U^dag on the backward hop", "dslash_site.cuh",
     "z = cjfma(u[3 * b + ai], h[3 * s + b], z);  // U^dag h", "z = cfma(u[3 * ai + b], h[3 * s + b], z);", 0, 1e-15),
    ("backward link taken at the site", "dslash_site.cuh",
     "load_link<T, LINKS>(a, NU, FWD ? site : nb, u);", "load_link<T, LINKS>(a, NU, site, u);", 0, 1e-15),
    ("gamma_5 on the upper spins", "dslash_site.cuh", "o[i] = i < 6 ? d : mk<T>(-d.r, -d.i);",
     "o[i] = i >= 6 ? d : mk<T>(-d.r, -d.i);", 0, 1e-15),
    ("12-real links: third row not conjugated", "dslash_site.cuh",
     "u[8] = conj(u[0] * u[4] - u[1] * u[3]);", "u[8] = u[0] * u[4] - u[1] * u[3];", 3, 1e-6),
    ("double-float product without the cross terms", "dd.cuh",
     "    e = f_fma(a.lo, b.hi, e);\n    float s, t;\n    dd_fast_two_sum(p, e, s, t);",
     "    float s, t;\n    dd_fast_two_sum(p, e, s, t);", 1, 2e-14),
    ("double-float conversion without the low part", "dd.cuh", "                lo = sgn ? -l : l;",
     "                lo = 0.f;", 1, 2e-14),
    ("double-float U^dag without the conjugate", "dd.cuh",
     "const float wih = FWD ? w.i.hi : -w.i.hi, wil = FWD ? w.i.lo : -w.i.lo;",
     "const float wih = w.i.hi, wil = w.i.lo;", 1, 2e-14),
]


def _build(case, tmp):
    name, header, old, new, mode, bound = case
    d = os.path.join(tmp, str(CASES.index(case)))
    os.makedirs(os.path.join(d, "paper_0710_0341_gb300", "csrc"))
    os.makedirs(os.path.join(d, "include"))
    os.makedirs(os.path.join(d, "tests", "hostcheck"))
    for h in ("dslash_site.cuh", "dd.cuh", "df.cuh"):
        src = open(os.path.join(CSRC, h)).read()
        if h == header:
            assert src.count(old) == 1, (name, src.count(old))
            src = src.replace(old, new)
        open(os.path.join(d, "paper_0710_0341_gb300", "csrc", h), "w").write(src)
    shutil.copy(os.path.join(ROOT, "include", "ovl.h"), os.path.join(d, "include", "ovl.h"))
    shutil.copy(hc.SRC, os.path.join(d, "tests", "hostcheck", "stencil_host.cu"))
    out = os.path.join(d, "libmutant.so")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    subprocess.run([nvcc, "-x", "cu", "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared",
                    os.path.join(d, "tests", "hostcheck", "stencil_host.cu"), "-o", out], check=True,
                   capture_output=True)
    return out


def test_every_planted_mistake_misses_the_oracle():
    if not os.path.exists(shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    dims, mu, m_w = (3, 4, 2, 5), 0.4, -1.1
    U = synth.random_su3_field(dims, 0.5, 2)
    psi = synth.gaussian_source(dims, 4)
    ref = dirac.apply(dirac.hermitian_wilson(U, mu, m_w), psi)
    with tempfile.TemporaryDirectory() as tmp:
        with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
            libs = list(ex.map(lambda c: _build(c, tmp), CASES))
        missed = []
        for case, path in zip(CASES, libs):
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            L.host_apply_hw.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, P, P, P, P]
            L.host_apply_hw.restype = ctypes.c_int
            err = np.linalg.norm(hc._apply(L, U, psi, mu, m_w, 0, case[4]) - ref) / np.linalg.norm(ref)
            if not err > 10 * case[5]:
                missed.append((case[0], err))
        assert not missed, missed
