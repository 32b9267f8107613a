"""The ctypes binding marshals exactly what include/ovl.h declares: the kind
of every parameter of every prototype, the two parameter structs field by
field (names, types, order, size), and the status, precision, scheme and
format constants. CPU only: nothing is called."""
import ctypes as C
import os
import re

from paper_0710_0341_gb300 import ovl

HDR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "include", "ovl.h")


def _header():
    return re.sub(r"/\*.*?\*/", " ", open(HDR).read(), flags=re.S)


def _c_kind(decl):
    """Kind of one C parameter declaration: 'ptr' for pointers, arrays and
    the library's opaque handles, else the scalar type."""
    d = " ".join(decl.split())
    if d in ("", "void"):
        return None
    if "*" in d or "[" in d:
        return "ptr"
    base = " ".join(d.replace("const ", "").split()[:-1])
    if base.startswith("ovl_"):  # typedef'd handle pointers
        return "ptr"
    return {"int": "int", "double": "double", "float": "float", "long long": "longlong"}[base]


def _ctypes_kind(t):
    if t is C.c_int:
        return "int"
    if t is C.c_double:
        return "double"
    if t is C.c_float:
        return "float"
    if t is C.c_longlong:
        return "longlong"
    if t in (C.c_void_p, C.c_char_p) or issubclass(t, C._Pointer):
        return "ptr"
    raise AssertionError(f"unexpected ctypes type {t}")


def _prototypes():
    out = {}
    for ret, name, args in re.findall(r"^\s*(int|const\s+char\s*\*)\s+(ovl_\w+)\s*\(([^)]*)\)\s*;", _header(),
                                      flags=re.M):
        kinds = [k for k in (_c_kind(a) for a in args.split(",")) if k is not None]
        out[name] = ("int" if ret == "int" else "str", kinds)
    return out


def test_every_prototype_has_a_matching_binding():
    protos = _prototypes()
    assert sorted(protos) == ovl.header_functions()
    assert set(protos) == set(ovl._SIGS), set(protos) ^ set(ovl._SIGS)
    for name, (ret, kinds) in protos.items():
        res, args = ovl._SIGS[name]
        assert (res is C.c_int) == (ret == "int") and (res is C.c_char_p) == (ret == "str"), name
        assert [_ctypes_kind(a) for a in args] == kinds, (name, kinds)


def _struct_fields(tag):
    m = re.search(r"typedef\s+struct\s*\{([^}]*)\}\s*" + tag + r"\s*;", _header(), flags=re.S)
    assert m, tag
    fields = []
    for line in m.group(1).split(";"):
        toks = line.split()
        if toks:
            fields.append((toks[-1], toks[0]))
    return fields


def test_parameter_structs_match_the_header():
    for tag, cls in (("ovl_sign_params", ovl.ovl_sign_params), ("ovl_sign_info", ovl.ovl_sign_info)):
        hdr = _struct_fields(tag)
        py = [(n, {C.c_int: "int", C.c_double: "double"}[t]) for n, t in cls._fields_]
        assert hdr == py, (tag, hdr, py)
    # natural alignment of the C layout: the sizes a C compiler gives these structs
    assert C.sizeof(ovl.ovl_sign_params) == 72 and C.sizeof(ovl.ovl_sign_info) == 40


def test_constants_match_the_header():
    defs = dict((n, int(v)) for n, v in re.findall(r"#define\s+(OVL_[A-Z0-9_]+)\s+(-?\d+)", _header()))
    for prefix in ("OVL_E", "OVL_OK", "OVL_PREC_", "OVL_DEFL_", "OVL_VEC_", "OVL_LINKS_"):
        names = [n for n in defs if n.startswith(prefix)]
        assert names, prefix
        for n in names:
            assert getattr(ovl, n) == defs[n], n
