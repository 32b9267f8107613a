"""Host logic of bench.py, on the CPU with stand-ins for the library and for
torch's device calls (the GPU measurement itself runs only on a GPU)."""
import numpy as np
import pytest

import bench


def test_clock_summary_reads_median_max_and_reasons():
    row = lambda mhz, hw="Not Active", cap="Not Active": [  # noqa: E731
        "0", str(mhz), "2070", "900.5", "0x0", hw, "Not Active", "Not Active", cap]
    s = bench.clock_summary([row(2070), row(1980, cap="Active"), row(2055), ["0", "[N/A]"]])
    assert s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    s = bench.clock_summary([row(1500, hw="Active")])
    assert s["reasons"] == ["hw_slowdown"]
    assert bench.clock_summary([]) == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}


class _Event:
    t = 0.0

    def __init__(self, enable_timing=True):
        self.at = None

    def record(self):
        _Event.t += 50.0  # 50 ms between consecutive records
        self.at = _Event.t

    def elapsed_time(self, other):
        return other.at - self.at


class _Cuda:
    Event = _Event

    @staticmethod
    def synchronize():
        pass


class _Tensor:
    def __init__(self, a):
        self.a = a

    def cpu(self):
        return self

    def numpy(self):
        return self.a


class _Torch:
    cuda = _Cuda

    @staticmethod
    def zeros_like(t):
        return _Tensor(np.zeros_like(t.a))


class _Lib:
    OVL_PREC_FP64, OVL_PREC_MIXED, OVL_PREC_MIXED_R12, OVL_PREC_FP64_DFSTENCIL, OVL_PREC_FP64_PLAIN = 0, 1, 2, 3, 4
    OVL_PREC_DF40 = 5

    def __init__(self):
        self.calls = []

    def ovl_sign_apply(self, h, params, defl, b, y):
        assert len(params) == len(defl) == len(b.a)
        self.calls.append([p["prec"] for p in params])
        y.a[:] = b.a


class _Tensor2(_Tensor):
    def __getitem__(self, s):
        return _Tensor2(self.a[s])

    def contiguous(self):
        return self


@pytest.mark.parametrize("headline,other,other_prec", [("df48", "df40_bf16_low_planes", 5),
                                                       ("df40", "df48_fp32_hi_lo_basis", 0)])
def test_precision_arms_time_each_form_once_on_its_sources(monkeypatch, headline, other, other_prec):
    lib = _Lib()
    errs = {4: [1e-12, 2e-12], 0: [3e-13] * 12, 5: [6e-11] * 12, 2: [6e-8] * 12, 1: [5e-8, None] + [7e-8] * 10}
    monkeypatch.setattr(bench, "accuracy", lambda ys, sk, keys: errs[lib.calls[-1][0]][:len(keys)])
    bd = _Tensor2(np.ones((12, 4), complex))
    out = bench.precision_arms(_Torch, lib, None, None, bd, {}, [f"{i}" for i in range(12)], headline=headline)
    # one call per form: the plain FP64 form on 2 sources, the other basis and the mixed forms on all 12
    assert [(c[0], len(c)) for c in lib.calls] == [(4, 2), (other_prec, 12), (2, 12), (1, 12)]
    assert out[other]["meets_1e-8"] is True
    p = out["plain_fp64"]
    assert p["solves"] == 2 and abs(p["ms_per_step"] - 50.0) < 1e-9 and abs(p["solves_per_s"] - 40.0) < 1e-9
    assert p["meets_1e-8"] is True
    assert out["mixed_fp32_basis_r12_links"]["meets_1e-8"] is False
    assert out["mixed_fp32_basis_fp32_links"]["rel_err_per_solve"][1] is None


def test_depth_cost_fit_recovers_the_model():
    a, c, m = 0.3, 2e-3, 40
    T = lambda k: a * k + c * (m * k + k * (k + 1) / 2)  # noqa: E731
    assert abs(bench.fit_depth_cost({6: T(6), 18: T(18)}, m, 600) - T(600)) < 1e-9 * T(600)
    # negative fitted parts (timing noise) are clamped at zero
    assert bench.fit_depth_cost({6: 1.0, 18: 1.0}, m, 600) >= 0.0


def test_sketch_error_is_the_relative_error_in_expectation():
    from paper_0710_0341_gb300 import synth

    rng = np.random.default_rng(0)
    n = 4000
    y = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    e = 1e-3 * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    P = synth.probe_vectors(n, 256)
    sk = P.conj() @ y
    ref = {"probe_re": list(sk.real), "probe_im": list(sk.imag), "norm": float(np.linalg.norm(y))}
    est = bench.sketch_error(y + e, ref, P)
    true = np.linalg.norm(e) / np.linalg.norm(y)
    assert 0.8 * true < est < 1.2 * true
    assert bench.accuracy([y, y], {"a": ref, "_meta": {}}, ["a", "b"])[1] is None


def test_roofline_uses_the_dominant_class_and_the_committed_traffic_ratio():
    prof = {"stencil": {"launches": 10, "ms": 1.0, "bytes": 1e9}, "gs_pass_a": {"launches": 10, "ms": 3.0, "bytes": 1e10},
            "gs_pass_b": {"launches": 10, "ms": 5.0, "bytes": 2e10}}
    r = bench.roofline(prof, {"hbm_gbs": 8000.0}, {"gs_pass_b": 1.01})
    assert r["kernel"] == "gs_pass_b"
    assert abs(r["achieved"] - 2e9 / 0.5e-3 / 1e9) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 8000.0) < 1e-12
    assert abs(r["traffic"] - 1.01 * 2e9) < 1e-3
    assert bench.roofline(prof, None, {})["traffic"] is None


def test_committed_profiles_give_the_pass_b_traffic_ratio():
    r = bench.traffic_ratios()
    assert 0.9 < r.get("gs_pass_b", 1.0) < 1.3


class _Buf:
    def __init__(self, n, dtype):
        self.n, self.dtype = n, dtype

    def cuda(self):
        return self


class _Torch2(_Torch):
    complex64, complex128 = "c64", "c128"

    @staticmethod
    def from_numpy(a):
        return _Buf(a.size, a.dtype)

    @staticmethod
    def randn(n, dtype=None, device=None):
        return _Buf(n, dtype)

    @staticmethod
    def zeros_like(t):
        return _Buf(t.n, t.dtype)


class _StencilLib:
    """Stand-in whose stencil takes 10 us per launch and records each call."""

    def __init__(self):
        self.calls, self.lat = [], {}
        self.on = False
        self.launches = 0

    def ovl_create_lattice(self, dims, apbc, stream):
        h = len(self.lat) + 1
        self.lat[h] = dims
        return h

    def ovl_set_links(self, h, U):
        pass

    def ovl_destroy_lattice(self, h):
        del self.lat[h]

    def ovl_apply_Hw_packed(self, h, mus, m_w, x, o, nrhs, fmt, links):
        V = int(np.prod(self.lat[h]))
        assert x.n == o.n == 12 * V * nrhs and len(mus) == nrhs
        assert x.dtype == ("c64" if fmt == 1 else "c128")
        self.calls.append((self.lat[h], nrhs, fmt, links))
        self.launches += self.on

    def ovl_autotune(self, h, nrhs):
        self.tuned = getattr(self, "tuned", 0) + 1
        return []

    def ovl_autotune_shape(self, h, fmt, links):
        return (128, 8, 4, 4)

    def ovl_profile(self, h, enable):
        self.on = bool(enable)
        if enable:
            self.launches = 0
            return None
        return {"stencil": {"ms": 0.01 * self.launches, "launches": self.launches}}


class _Synth:
    @staticmethod
    def random_su3_field(dims, eps, seed):
        return np.zeros(1)


def test_stencil_cases_count_spinors_per_rhs_and_links_once():
    lib = _StencilLib()
    res = bench.stencil_gbs(_Torch2, lib, _Synth)
    assert not lib.lat  # every lattice destroyed
    V24, V16 = 24 ** 3 * 48, 16 ** 3 * 32
    expect = {"fp32_r12": (V24, 1, 2 * 12 * 8 + 4 * 48), "fp32_18": (V24, 1, 2 * 12 * 8 + 4 * 72),
              "fp64": (V24, 1, 2 * 12 * 16 + 4 * 144), "fp64_double_float": (V24, 1, 2 * 12 * 16 + 4 * 144),
              "fp32_r12_16x3x32_12rhs": (V16, 12, 12 * 2 * 12 * 8 + 4 * 48)}
    for name, (V, nrhs, bps) in expect.items():
        r = res[name]
        assert r["rhs"] == nrhs and r["bytes_per_site"] == bps
        assert abs(r["us_per_launch"] - 10.0) < 1e-9
        assert abs(r["GB_per_s"] - V * bps / 10e-6 / 1e9) < 1e-6 * r["GB_per_s"]
    # per case 3 warm-up and 20 timed launches with the built-in shape, then the
    # same after the autotuner (once per lattice); the 12-rhs case in one launch each
    assert len(lib.calls) == 2 * 5 * 23 and lib.calls[-1] == ((16, 16, 16, 32), 12, 1, 2)
    assert lib.tuned == 3
    assert all(res[k]["shape_tpb_tx_ty_tz"] == (128, 8, 4, 4) and "builtin_shape" in res[k] for k in expect)
    assert ((24, 24, 24, 48), 1, 0, 3) in lib.calls  # FP64 data, double-float links format


def test_amortised_throughput_includes_the_setup():
    a = bench.amortised(100.0, 250.0, 8)
    assert abs(a["1_batches_per_setup"] - 8 / 100.25) < 1e-12
    assert abs(a["12_batches_per_setup"] - 96 / 103.0) < 1e-12


class _UnevenLib:
    """ovl stand-in for the uneven 12^4 batch: adaptive depths by mu, the mu = 0.8
    solves capped at k_max with a large estimate."""
    OVL_DEFL_SCHUR = 1

    def __init__(self):
        self.graphs = 0
        self.replays = 0
        self.calls = []
        self.live = set()

    def ovl_create_lattice(self, dims, apbc, stream):
        self.live.add("lat")
        return "lat"

    def ovl_set_links(self, h, U):
        pass

    def ovl_autotune(self, h, nrhs):
        return []

    def ovl_deflation_setup(self, h, mu, m_w, scheme, m, tol, maxit):
        self.live.add(("d", mu))
        return ("d", mu)

    def ovl_sign_apply(self, h, params, defl, b, y):
        self.calls.append([dict(p) for p in params])
        if self.graphs:
            self.replays += 1
        out = []
        for p in params:
            if "adapt_every" in p:
                k, e = {0.05: (250, 5e-10), 0.2: (275, 6e-10), 0.4: (350, 8e-10), 0.8: (700, 4e-5)}[p["mu"]]
            else:
                k, e = p["k"], 0.0
            out.append(dict(status=0, k_used=k, err_est=e))
        return out

    def ovl_set_graphs(self, h, g):
        if g >= 0:
            self.graphs = g
        return self.replays

    def ovl_destroy_deflation(self, d):
        self.live.discard(d)

    def ovl_destroy_lattice(self, h):
        self.live.discard(h)


class _Torch3(_Torch):
    @staticmethod
    def from_numpy(a):
        t = _Tensor(a)
        t.cuda = lambda: t
        return t


class _Synth3(_Synth):
    @staticmethod
    def point_source(dims, s, c):
        return np.zeros(2, complex)


def test_uneven_batch_reports_depths_and_estimates_per_mu():
    lib = _UnevenLib()
    out = bench.extra_12x4(_Torch3, lib, _Synth3)
    assert not lib.live  # lattice and the four deflation objects released
    assert out["solves"] == 48
    assert out["k_per_mu"] == {"0.05": [250], "0.2": [275], "0.4": [350], "0.8": [700]}
    assert out["adaptive_err_est_max_per_mu"]["0.8"] == 4e-5 and out["adaptive_err_est_max_per_mu"]["0.2"] == 6e-10
    assert out["err_est_below_1e-8_per_mu"] == {"0.05": True, "0.2": True, "0.4": True, "0.8": False}
    # the timed calls run the adaptive depths as fixed depths, eager and as graph replays
    timed = lib.calls[1:]
    assert len(timed) == 8 and all(len(c) == 48 and "adapt_every" not in c[0] for c in timed)
    assert sorted({p["k"] for p in timed[0]}) == [250, 275, 350, 700]
    assert out["graph_replays"] == 4 and "eager" in out and "graph" in out
