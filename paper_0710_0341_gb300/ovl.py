"""ctypes binding of the C ABI in include/ovl.h (argument marshalling only).

Every ``ovl_*`` function here has the name and arguments of its C
counterpart; arrays may be numpy arrays (host) or torch tensors (host or
CUDA) of complex128 in the canonical layouts the header describes. Nothing
here computes: every step runs in libovl.so, and a missing library raises
``OvlError`` instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "libovl.so")

OVL_OK, OVL_EINVAL, OVL_ENOMEM, OVL_ECUDA, OVL_ENOCONV, OVL_ETIMEOUT, OVL_ENOTSUP = range(7)
OVL_PREC_FP64, OVL_PREC_MIXED, OVL_PREC_MIXED_R12, OVL_PREC_FP64_DFSTENCIL, OVL_PREC_FP64_PLAIN = 0, 1, 2, 3, 4
OVL_PREC_DF40 = 5
OVL_DEFL_NONE, OVL_DEFL_SCHUR, OVL_DEFL_LR = 0, 1, 2
OVL_VEC_F64, OVL_VEC_F32 = 0, 1
OVL_LINKS_F64, OVL_LINKS_F32, OVL_LINKS_R12, OVL_LINKS_F64DF = 0, 1, 2, 3


class OvlError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ovl error {code}: {msg}")
        self.code = code


class ovl_sign_params(C.Structure):
    _fields_ = [("mu", C.c_double), ("m_w", C.c_double), ("k", C.c_int), ("prec", C.c_int),
                ("newton_max_iter", C.c_int), ("newton_tol", C.c_double), ("newton_fp64", C.c_int),
                ("adapt_every", C.c_int), ("k_max", C.c_int), ("tol", C.c_double), ("schur_route", C.c_int)]


class ovl_sign_info(C.Structure):
    _fields_ = [("status", C.c_int), ("k_used", C.c_int), ("m_used", C.c_int), ("newton_iters", C.c_int),
                ("beta", C.c_double), ("beta_k", C.c_double), ("err_est", C.c_double)]


_lib = None
_P = C.c_void_p
_SIGS = {
    "ovl_create_lattice": (C.c_int, [C.POINTER(C.c_int), C.c_int, _P, C.POINTER(_P)]),
    "ovl_destroy_lattice": (C.c_int, [_P]),
    "ovl_set_links": (C.c_int, [_P, _P]),
    "ovl_apply_Hw": (C.c_int, [_P, C.c_double, C.c_double, _P, _P, C.c_int, C.c_int]),
    "ovl_apply_Hw_noalloc": (C.c_int, [_P, C.c_double, C.c_double, _P, _P, C.c_int, C.c_int]),
    "ovl_apply_Hw_packed": (C.c_int, [_P, _P, C.c_double, _P, _P, C.c_int, C.c_int, C.c_int]),
    "ovl_pack_spinor": (C.c_int, [_P, _P, _P, C.c_int, C.c_int]),
    "ovl_unpack_spinor": (C.c_int, [_P, _P, _P, C.c_int, C.c_int]),
    "ovl_set_deflation": (C.c_int, [_P, C.c_double, C.c_double, C.c_int, C.c_int, _P, _P, _P, C.POINTER(_P)]),
    "ovl_deflation_setup": (C.c_int, [_P, C.c_double, C.c_double, C.c_int, C.c_int, C.c_double, C.c_int,
                                      C.POINTER(_P)]),
    "ovl_deflation_setup_ex": (C.c_int, [_P, C.c_double, C.c_double, C.c_int, C.c_int, C.c_double, C.c_int,
                                         C.c_int, C.POINTER(_P)]),
    "ovl_get_deflation": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), _P, _P, _P]),
    "ovl_destroy_deflation": (C.c_int, [_P]),
    "ovl_deflation_save": (C.c_int, [_P, C.c_char_p]),
    "ovl_deflation_load": (C.c_int, [_P, C.c_char_p, C.POINTER(_P)]),
    "ovl_deflation_stats": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "ovl_sign_apply": (C.c_int, [_P, C.c_int, C.POINTER(ovl_sign_params), C.POINTER(_P), _P, _P,
                                 C.POINTER(ovl_sign_info)]),
    "ovl_sign_workspace_bytes": (C.c_int, [_P, C.c_int, C.POINTER(ovl_sign_params), C.POINTER(_P),
                                           C.POINTER(C.c_double)]),
    "ovl_overlap_apply": (C.c_int, [_P, C.c_int, C.POINTER(ovl_sign_params), C.POINTER(_P), _P, _P, C.c_int,
                                    C.POINTER(ovl_sign_info)]),
    "ovl_deflation_adjoint": (C.c_int, [_P, C.POINTER(_P)]),
    "ovl_launch_count": (C.c_int, [_P, C.POINTER(C.c_longlong)]),
    "ovl_mlp_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(_P)]),
    "ovl_mlp_destroy": (C.c_int, [_P]),
    "ovl_mlp_num_params": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "ovl_mlp_set_params": (C.c_int, [_P, _P]),
    "ovl_mlp_get_params": (C.c_int, [_P, _P]),
    "ovl_mlp_forward": (C.c_int, [_P, _P, C.c_int, _P]),
    "ovl_mlp_loss_grad": (C.c_int, [_P, _P, _P, C.c_int, C.c_float, _P, _P]),
    "ovl_mlp_train": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.c_float, C.c_float, _P]),
    "ovl_mlp_last_error": (C.c_char_p, [_P]),
    "ovl_link_spread": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "ovl_set_graphs": (C.c_int, [_P, C.c_int, C.POINTER(C.c_longlong)]),
    "ovl_set_pass_b": (C.c_int, [_P, C.c_int]),
    "ovl_autotune": (C.c_int, [_P, C.c_int, _P, C.c_int, C.POINTER(C.c_int)]),
    "ovl_autotune_shape": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "ovl_autotune_set_shape": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "ovl_wait_selftest": (C.c_int, [_P, C.c_longlong, C.POINTER(C.c_int)]),
    "ovl_ritz_values": (C.c_int, [_P, C.c_double, C.c_double, C.c_int, _P, _P]),
    "ovl_profile": (C.c_int, [_P, C.c_int, _P]),
    "ovl_last_error": (C.c_char_p, [_P]),
    "ovl_version": (C.c_char_p, []),
}


def lib():
    """Load libovl.so (raises OvlError if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIBPATH):
            raise OvlError(OVL_ENOTSUP, f"{LIBPATH} is not built; run paper_0710_0341_gb300.build.build()")
        L = C.CDLL(LIBPATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc, h=None):
    if rc != OVL_OK:
        msg = lib().ovl_last_error(h)
        raise OvlError(rc, msg.decode() if msg else "")


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (must be contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    import numpy as np

    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def ovl_version():
    return lib().ovl_version().decode()


def ovl_create_lattice(dims, antiperiodic_t=0, stream=None):
    h = _P()
    d = (C.c_int * 4)(*[int(x) for x in dims])
    _check(lib().ovl_create_lattice(d, int(antiperiodic_t), _stream_ptr(stream), C.byref(h)))
    return h


def ovl_destroy_lattice(h):
    _check(lib().ovl_destroy_lattice(h), h)


def ovl_set_links(h, U):
    _check(lib().ovl_set_links(h, _ptr(U)), h)


def ovl_apply_Hw(h, mu, m_w, x, out, nrhs=1, links=OVL_LINKS_F64):
    _check(lib().ovl_apply_Hw(h, float(mu), float(m_w), _ptr(x), _ptr(out), int(nrhs), int(links)), h)
    return out


def ovl_apply_Hw_noalloc(h, mu, m_w, x, out, nrhs=1, links=OVL_LINKS_F64):
    """ovl_apply_Hw without device allocation (device tensors only)."""
    _check(lib().ovl_apply_Hw_noalloc(h, float(mu), float(m_w), _ptr(x), _ptr(out), int(nrhs), int(links)), h)
    return out


def ovl_apply_Hw_packed(h, mus, m_w, x, out, nrhs, fmt, links):
    arr = (C.c_double * nrhs)(*[float(m) for m in mus])
    _check(lib().ovl_apply_Hw_packed(h, C.cast(arr, _P), float(m_w), _ptr(x), _ptr(out), int(nrhs), int(fmt),
                                     int(links)), h)
    return out


def ovl_pack_spinor(h, canon, packed, nrhs, fmt):
    _check(lib().ovl_pack_spinor(h, _ptr(canon), _ptr(packed), int(nrhs), int(fmt)), h)


def ovl_unpack_spinor(h, packed, canon, nrhs, fmt):
    _check(lib().ovl_unpack_spinor(h, _ptr(packed), _ptr(canon), int(nrhs), int(fmt)), h)


def ovl_set_deflation(h, mu, m_w, scheme, m, S_or_R, T, L=None):
    d = _P()
    _check(lib().ovl_set_deflation(h, float(mu), float(m_w), int(scheme), int(m), _ptr(S_or_R), _ptr(T), _ptr(L),
                                   C.byref(d)), h)
    return d


def ovl_deflation_setup(h, mu, m_w, scheme, m, tol=1e-12, max_restarts=500):
    d = _P()
    _check(lib().ovl_deflation_setup(h, float(mu), float(m_w), int(scheme), int(m), float(tol), int(max_restarts),
                                     C.byref(d)), h)
    return d


def ovl_deflation_setup_ex(h, mu, m_w, scheme, m, tol=1e-12, max_restarts=500, poly_degree=-1):
    d = _P()
    _check(lib().ovl_deflation_setup_ex(h, float(mu), float(m_w), int(scheme), int(m), float(tol),
                                        int(max_restarts), int(poly_degree), C.byref(d)), h)
    return d


def ovl_get_deflation(d, S_or_R=None, T=None, L=None, h=None):
    sch, m = C.c_int(), C.c_int()
    _check(lib().ovl_get_deflation(d, C.byref(sch), C.byref(m), _ptr(S_or_R), _ptr(T), _ptr(L)), h)
    return sch.value, m.value


def ovl_deflation_stats(d):
    r, m = C.c_int(), C.c_int()
    _check(lib().ovl_deflation_stats(d, C.byref(r), C.byref(m)))
    return r.value, m.value


def ovl_deflation_save(d, path):
    _check(lib().ovl_deflation_save(d, os.fsencode(path)))


def ovl_deflation_load(h, path):
    d = _P()
    _check(lib().ovl_deflation_load(h, os.fsencode(path), C.byref(d)), h)
    return d


def ovl_destroy_deflation(d):
    _check(lib().ovl_destroy_deflation(d))


def ovl_sign_apply(h, params, defl, b, y, info=True):
    """params: list of dicts (mu, m_w, k, prec[, newton_max_iter, newton_tol]);
    defl: list of deflation handles or None (same length)."""
    n = len(params)
    P = (ovl_sign_params * n)()
    for i, p in enumerate(params):
        P[i].mu = p["mu"]
        P[i].m_w = p["m_w"]
        P[i].k = int(p["k"])
        P[i].prec = int(p.get("prec", OVL_PREC_FP64))
        P[i].newton_max_iter = int(p.get("newton_max_iter", 0))
        P[i].newton_tol = float(p.get("newton_tol", 0.0))
        P[i].newton_fp64 = int(p.get("newton_fp64", 0))
        P[i].adapt_every = int(p.get("adapt_every", 0))
        P[i].k_max = int(p.get("k_max", 0))
        P[i].tol = float(p.get("tol", 0.0))
        P[i].schur_route = int(p.get("schur_route", 0))
    D = (_P * n)(*[(d.value if isinstance(d, _P) else d) if d is not None else None for d in (defl or [None] * n)])
    I = (ovl_sign_info * n)()
    rc = lib().ovl_sign_apply(h, n, P, D, _ptr(b), _ptr(y), I)
    infos = [dict(status=I[i].status, k_used=I[i].k_used, m_used=I[i].m_used, newton_iters=I[i].newton_iters,
                  beta=I[i].beta, beta_k=I[i].beta_k, err_est=I[i].err_est) for i in range(n)]
    if rc != OVL_OK:
        msg = lib().ovl_last_error(h)
        err = OvlError(rc, (msg.decode() if msg else "") + f" infos={infos}")
        err.infos = infos
        raise err
    return infos


def _params(params):
    n = len(params)
    P = (ovl_sign_params * n)()
    for i, p in enumerate(params):
        P[i].mu = p["mu"]
        P[i].m_w = p["m_w"]
        P[i].k = int(p["k"])
        P[i].prec = int(p.get("prec", OVL_PREC_FP64))
        P[i].newton_max_iter = int(p.get("newton_max_iter", 0))
        P[i].newton_tol = float(p.get("newton_tol", 0.0))
        P[i].newton_fp64 = int(p.get("newton_fp64", 0))
        P[i].adapt_every = int(p.get("adapt_every", 0))
        P[i].k_max = int(p.get("k_max", 0))
        P[i].tol = float(p.get("tol", 0.0))
        P[i].schur_route = int(p.get("schur_route", 0))
    return P


def ovl_sign_workspace_bytes(h, params, defl=None):
    """Device bytes ovl_sign_apply needs for this batch (nothing runs)."""
    n = len(params)
    D = (_P * n)(*[(d.value if isinstance(d, _P) else d) if d is not None else None for d in (defl or [None] * n)])
    out = C.c_double()
    _check(lib().ovl_sign_workspace_bytes(h, n, _params(params), D, C.byref(out)), h)
    return int(out.value)


def ovl_overlap_apply(h, params, defl, x, y, adjoint=False):
    """D_ov(mu) x (adjoint=False) or D_ov(mu)^dag x (True) per solve; params and
    defl as in ovl_sign_apply (for the adjoint: deflation data of H_w(-mu))."""
    n = len(params)
    P = (ovl_sign_params * n)()
    for i, p in enumerate(params):
        P[i].mu = p["mu"]
        P[i].m_w = p["m_w"]
        P[i].k = int(p["k"])
        P[i].prec = int(p.get("prec", OVL_PREC_FP64))
        P[i].newton_max_iter = int(p.get("newton_max_iter", 0))
        P[i].newton_tol = float(p.get("newton_tol", 0.0))
        P[i].newton_fp64 = int(p.get("newton_fp64", 0))
        P[i].adapt_every = int(p.get("adapt_every", 0))
        P[i].k_max = int(p.get("k_max", 0))
        P[i].tol = float(p.get("tol", 0.0))
        P[i].schur_route = int(p.get("schur_route", 0))
    D = (_P * n)(*[(d.value if isinstance(d, _P) else d) if d is not None else None for d in (defl or [None] * n)])
    I = (ovl_sign_info * n)()
    rc = lib().ovl_overlap_apply(h, n, P, D, _ptr(x), _ptr(y), int(bool(adjoint)), I)
    infos = [dict(status=I[i].status, k_used=I[i].k_used, m_used=I[i].m_used, newton_iters=I[i].newton_iters,
                  beta=I[i].beta, beta_k=I[i].beta_k, err_est=I[i].err_est) for i in range(n)]
    if rc != OVL_OK:
        msg = lib().ovl_last_error(h)
        err = OvlError(rc, (msg.decode() if msg else "") + f" infos={infos}")
        err.infos = infos
        raise err
    return infos


def ovl_deflation_adjoint(d):
    """LR deflation data of H_w(-mu) from those of H_w(mu) (new handle)."""
    out = _P()
    _check(lib().ovl_deflation_adjoint(d, C.byref(out)))
    return out


def ovl_launch_count(h):
    n = C.c_longlong()
    _check(lib().ovl_launch_count(h, C.byref(n)), h)
    return n.value


PROF_CLASSES = ["stencil", "gs_pass_a", "gs_reduce", "gs_small", "gs_pass_b", "newton", "projection",
                "recombination"]


def ovl_set_graphs(h, enable):
    """enable 1/0 CUDA-graph replay of the Arnoldi loop, -1 query; returns the replay count."""
    n = C.c_longlong()
    _check(lib().ovl_set_graphs(h, int(enable), C.byref(n)), h)
    return n.value


def ovl_set_pass_b(h, bulk):
    """1: pass B streams the basis by bulk copies into shared memory; 0: register loads (default)."""
    _check(lib().ovl_set_pass_b(h, int(bulk)), h)


def ovl_autotune(h, nrhs=1, max_report=256):
    """Time the stencil's launch shapes and keep the fastest per (format,
    links); returns the timed candidates as dicts."""
    buf = (C.c_double * (8 * max_report))()
    n = C.c_int()
    _check(lib().ovl_autotune(h, int(nrhs), C.cast(buf, _P), int(max_report), C.byref(n)), h)
    keys = ("fmt", "links", "tpb", "tx", "ty", "tz", "variant", "us")
    return [dict(zip(keys, [int(buf[8 * i + j]) for j in range(7)] + [buf[8 * i + 7]])) for i in range(n.value)]


def ovl_autotune_shape(h, fmt, links):
    s = (C.c_int * 5)()
    _check(lib().ovl_autotune_shape(h, int(fmt), int(links), s), h)
    return tuple(s)


def ovl_autotune_set_shape(h, fmt, links, shape):
    s = (C.c_int * 5)(*[int(v) for v in shape])
    _check(lib().ovl_autotune_set_shape(h, int(fmt), int(links), s), h)


def ovl_profile(h, enable):
    """Start (enable=1, clears) or stop (0) per-class timing; returns the
    per-class {launches, ms, bytes} collected so far."""
    buf = (C.c_double * (3 * len(PROF_CLASSES)))()
    _check(lib().ovl_profile(h, int(enable), C.cast(buf, _P)), h)
    return {n: dict(launches=int(buf[3 * i]), ms=buf[3 * i + 1], bytes=buf[3 * i + 2])
            for i, n in enumerate(PROF_CLASSES)}


def _mcheck(rc, net=None):
    if rc != OVL_OK:
        m = lib().ovl_last_error(None)
        raise OvlError(rc, m.decode() if m else "")


def ovl_mlp_create(n_in, n_hidden, n_out):
    net = _P()
    _mcheck(lib().ovl_mlp_create(int(n_in), int(n_hidden), int(n_out), C.byref(net)))
    return net


def ovl_mlp_destroy(net):
    _mcheck(lib().ovl_mlp_destroy(net))


def ovl_mlp_num_params(net):
    n = C.c_int()
    _mcheck(lib().ovl_mlp_num_params(net, C.byref(n)))
    return n.value


def ovl_mlp_set_params(net, theta):
    _mcheck(lib().ovl_mlp_set_params(net, _ptr(theta)))


def ovl_mlp_get_params(net, theta):
    _mcheck(lib().ovl_mlp_get_params(net, _ptr(theta)))
    return theta


def ovl_mlp_forward(net, X, Y):
    _mcheck(lib().ovl_mlp_forward(net, _ptr(X), int(X.shape[0]), _ptr(Y)))
    return Y


def ovl_mlp_loss_grad(net, X, T, under_weight, grad):
    loss = (C.c_float * 1)()
    _mcheck(lib().ovl_mlp_loss_grad(net, _ptr(X), _ptr(T), int(X.shape[0]), float(under_weight),
                                    C.cast(loss, _P), _ptr(grad)))
    return float(loss[0])


def ovl_mlp_train(net, X, T, steps, lr, under_weight):
    loss = (C.c_float * 1)()
    _mcheck(lib().ovl_mlp_train(net, _ptr(X), _ptr(T), int(X.shape[0]), int(steps), float(lr), float(under_weight),
                                C.cast(loss, _P)))
    return float(loss[0])


def ovl_wait_selftest(h, max_polls=10000):
    st = C.c_int()
    _check(lib().ovl_wait_selftest(h, int(max_polls), C.byref(st)), h)
    return st.value


def ovl_link_spread(h):
    v = C.c_double()
    _check(lib().ovl_link_spread(h, C.byref(v)), h)
    return v.value


def ovl_ritz_values(h, mu, m_w, k, b, out):
    _check(lib().ovl_ritz_values(h, float(mu), float(m_w), int(k), _ptr(b), _ptr(out)), h)
    return out


def ovl_last_error(h=None):
    m = lib().ovl_last_error(h)
    return m.decode() if m else ""


def header_functions():
    """Names of the functions include/ovl.h declares (parsed from the header)."""
    import re

    hdr = os.path.join(_HERE, "..", "include", "ovl.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(ovl_\w+)\s*\(", txt, flags=re.M)))
