"""Small cases of the sign-function workloads, for kernel profiling under ncu
(not a test module: pytest collects only test_*.py).

Default: one batch of the 8^4 workload.

Runs ovl_sign_apply once for 8 solves (mu in {0, 0.1, 0.3, 0.6} x Schur/LR,
k = 400, m = 30, FP64 mode) with deflation data imported from a seeded
orthonormal block (the kernels' work does not depend on the eigenvectors,
so the expensive eigensolver setup is skipped), inside an NVTX range
"sign_batch". Used as the command under ncu, e.g.

    ncu --set full --clock-control none -k regex:k_gs_update -s 200 -c 1 \\
        python tests/profile_case.py

``python tests/profile_case.py stencil r12 [tuned]`` instead applies the
stencil alone (24^3x48, one right-hand side, 12-real links) five times, with
the built-in launch shape or the autotuner's;
``python tests/profile_case.py c3 [prec [bulk]]`` runs one solve of the 16^3x32
workload's shape at reduced depth (one point source, k = 120, m = 40 Schur
vectors from a seeded orthonormal block; prec 0 = the 48-bit mode,
4 = plain FP64, 2 = mixed with 12-real links).
"""
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_0710_0341_gb300 import build, ovl, synth  # noqa: E402


def main():
    build.build()
    dims, m = (8, 8, 8, 8), 30
    N = 12 * 8 ** 4
    U = synth.random_su3_field(dims, 0.4, 0)
    h = ovl.ovl_create_lattice(dims)
    ovl.ovl_set_links(h, torch.from_numpy(U).cuda())
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((N, m)) + 1j * rng.standard_normal((N, m)))
    cols = np.ascontiguousarray(Q.T.reshape((m,) + synth.lattice_shape(dims) + (4, 3)))
    lam = np.linspace(0.17, 0.2, m).astype(complex)
    T = np.diag(lam)
    mus = [0.0, 0.1, 0.3, 0.6]
    defl = [ovl.ovl_set_deflation(h, mu, -1.0, ovl.OVL_DEFL_SCHUR, m, cols, T.ravel(order="F").copy(), None)
            for mu in mus]
    defl += [ovl.ovl_set_deflation(h, mu, -1.0, ovl.OVL_DEFL_LR, m, cols, lam, cols) for mu in mus]
    b = torch.from_numpy(np.stack([synth.gaussian_source(dims, 1)] * 8)).cuda()
    y = torch.zeros_like(b)
    params = [dict(mu=mu, m_w=-1.0, k=400) for mu in mus] * 2
    torch.cuda.nvtx.range_push("sign_batch")
    infos = ovl.ovl_sign_apply(h, params, defl, b, y)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print("profile case done; newton iterations", [i["newton_iters"] for i in infos])


def stencil(fmt_name="r12", tuned="", dims=(24, 24, 24, 48), reps=5):
    """Repeated single-RHS stencil applications on packed spinors (24^3x48),
    inside an NVTX range "stencil"; with "tuned" the launch shapes are first
    chosen by the autotuner (the shape the benchmark's stencil line uses)."""
    build.build()
    V = int(np.prod(dims))
    h = ovl.ovl_create_lattice(dims)
    ovl.ovl_set_links(h, torch.from_numpy(synth.random_su3_field(dims, 0.3, 0)).cuda())
    fmt, links = {"r12": (1, 2), "f32": (1, 1), "f64": (0, 0)}[fmt_name]
    if tuned == "tuned":
        ovl.ovl_autotune(h, 1)
        print("autotuned shape", ovl.ovl_autotune_shape(h, fmt, links))
    x = torch.randn(12 * V, dtype=torch.complex64 if fmt == 1 else torch.complex128, device="cuda")
    o = torch.zeros_like(x)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("stencil")
    for _ in range(reps):
        ovl.ovl_apply_Hw_packed(h, [0.3], -1.0, x, o, 1, fmt, links)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    ovl.ovl_destroy_lattice(h)
    print("stencil case done", fmt_name, tuned or "built-in shape", dims)


def config3(prec=0, load="", k=120, m=40):
    """One solve of the 16^3x32 workload's shape (point source at the origin,
    mu = 0.2, m_w = -1.2) at depth k with m seeded orthonormal Schur vectors;
    load "bulk" streams pass B's columns by bulk copies (ovl_set_pass_b)."""
    build.build()
    dims = (16, 16, 16, 32)
    N = 12 * int(np.prod(dims))
    h = ovl.ovl_create_lattice(dims)
    if load == "bulk":
        ovl.ovl_set_pass_b(h, 1)
    ovl.ovl_set_links(h, torch.from_numpy(synth.random_su3_field(dims, 0.3, 0)).cuda())
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((N, m)) + 1j * rng.standard_normal((N, m)))
    cols = np.ascontiguousarray(Q.T.reshape((m,) + synth.lattice_shape(dims) + (4, 3)))
    T = np.diag(np.linspace(0.3, 0.4, m).astype(complex))
    d = ovl.ovl_set_deflation(h, 0.2, -1.2, ovl.OVL_DEFL_SCHUR, m, cols, T.ravel(order="F").copy(), None)
    b = torch.from_numpy(synth.point_source(dims, 0, 0)).cuda()
    y = torch.zeros_like(b)
    infos = ovl.ovl_sign_apply(h, [dict(mu=0.2, m_w=-1.2, k=k, prec=int(prec))], [d], b, y)
    torch.cuda.synchronize()
    ovl.ovl_destroy_deflation(d)
    ovl.ovl_destroy_lattice(h)
    print("config3 case done; newton iterations", [i["newton_iters"] for i in infos])


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "stencil":
        stencil(*(sys.argv[2:4] or ["r12"]))
    elif len(sys.argv) > 1 and sys.argv[1] == "c3":
        config3(*(sys.argv[2:4] or [0]))
    else:
        main()
