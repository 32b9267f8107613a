"""The C-ABI library builds for sm_103a, loads, and exports every function
include/ovl.h declares (no compute calls: this runs without a GPU)."""
import ctypes

from paper_0710_0341_gb300 import build, ovl


def test_library_exports_header_functions():
    path = build.build()
    L = ctypes.CDLL(path)
    names = ovl.header_functions()
    assert "ovl_sign_apply" in names and "ovl_apply_Hw" in names
    for n in names:
        assert hasattr(L, n), n
    assert ovl.ovl_version().endswith("sm_103a")


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(ovl, "_lib", None)
    monkeypatch.setattr(ovl, "LIBPATH", str(tmp_path / "nope.so"))
    try:
        ovl.lib()
    except ovl.OvlError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("expected OvlError")
