"""Shared helpers for the GPU tests: load the library, move arrays, and build
deflation inputs with the oracle (tests only)."""
import numpy as np
import pytest

from paper_0710_0341_gb300 import ovl


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0710_0341_gb300 import build

    build.build()
    ovl.lib()
    return torch


def to_dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def lattice(dims, U, apbc=0):
    h = ovl.ovl_create_lattice(dims, apbc, None)
    ovl.ovl_set_links(h, np.ascontiguousarray(U))
    return h


def canon_cols(M, dims):
    """N x m column matrix -> m canonical spinors stacked (m, Lt, Lz, Ly, Lx, 4, 3)."""
    lx, ly, lz, lt = dims
    return np.ascontiguousarray(M.T.reshape(M.shape[1], lt, lz, ly, lx, 4, 3))
