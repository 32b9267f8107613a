"""Host logic of bench.py, on the CPU with stand-ins for the library and for
torch's device calls (the GPU measurement itself runs only on a GPU)."""
import numpy as np

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
    OVL_PREC_FP64, OVL_PREC_MIXED, OVL_PREC_MIXED_R12, OVL_PREC_FP64_DFSTENCIL = 0, 1, 2, 3

    def __init__(self):
        self.calls = []

    def ovl_sign_apply(self, h, params, defl, b, y):
        self.calls.append([p["prec"] for p in params])
        y.a[:] = b.a


def test_mixed_modes_times_both_modes_on_the_batch(monkeypatch):
    errs = {1: [5e-8] * 8, 2: [7e-8] * 7 + [2e-7], 3: [2e-9] * 8}
    lib = _Lib()
    monkeypatch.setattr(bench, "reference_sketch", lambda: {"0.0": {}})
    monkeypatch.setattr(bench, "accuracy", lambda y, sk: errs[lib.calls[-1][0]])
    bd = _Tensor(np.ones((8, 4), complex))
    out = bench.mixed_modes(_Torch, lib, None, [None] * 8, bd, 3)
    # one warm-up and three timed calls per mode, each over the 8-solve batch in one precision
    assert [c[0] for c in lib.calls] == [1] * 4 + [2] * 4 + [3] * 4
    assert all(len(set(c)) == 1 and len(c) == 8 for c in lib.calls)
    a, b = out["fp32_basis_fp32_links"], out["fp32_basis_r12_links"]
    assert abs(a["ms_per_step"] - 50.0 / 3) < 1e-9
    assert abs(a["solves_per_s"] - 8 / (50.0 / 3 / 1e3)) < 1e-6
    assert a["meets_1e-8"] is False and b["rel_err_est_per_solve"][-1] == 2e-7
    assert out["fp64_basis_double_float_stencil"]["meets_1e-8"] is True


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
    # 3 warm-up and 20 timed launches per case, the 12-rhs case in one launch each
    assert len(lib.calls) == 5 * 23 and lib.calls[-1] == ((16, 16, 16, 32), 12, 1, 2)
    assert ((24, 24, 24, 48), 1, 0, 3) in lib.calls  # FP64 data, double-float links format


def test_amortised_throughput_includes_the_setup():
    a = bench.amortised(100.0, 250.0, 8)
    assert abs(a["1_sources_per_operator"] - 8 / 100.25) < 1e-12
    assert abs(a["12_sources_per_operator"] - 96 / 103.0) < 1e-12
