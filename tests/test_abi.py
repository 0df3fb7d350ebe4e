"""The C ABI: the shared library loads without a GPU and exports every
function include/lsw.h declares; the binding's structs match the header's."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lsw.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lsw_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2005_01372_gb300 import build
    if not os.path.exists(build.LIB):
        try:
            build.build()
        except (RuntimeError, OSError) as e:
            pytest.skip(f"cannot build the library here: {e}")
    return build.LIB


def test_header_declares_the_method_calls():
    names = _declared()
    for n in ("lsw_build_green", "lsw_apply_operator", "lsw_sketch_range", "lsw_build_hmatrix",
              "lsw_apply_precond", "lsw_solve_series"):
        assert n in names


def test_every_declared_symbol_is_exported(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.lsw_status_string.restype = ctypes.c_char_p
    assert lib.lsw_status_string(0) == b"ok"
    assert b"unsupported" in lib.lsw_status_string(2)


def test_binding_struct_sizes_match_header():
    from paper_2005_01372_gb300 import lsw
    # lsw_grid: 2 int32 + 3 double; lsw_hparams: 8 int32 + uint64;
    # lsw_solve_params: 2 int32 + 2 double + 4 int32; lsw_solve_info: 4 int32 + double
    assert ctypes.sizeof(lsw._Grid) == 32
    assert ctypes.sizeof(lsw._HParams) == 40
    assert ctypes.sizeof(lsw._SolveParams) == 40
    assert ctypes.sizeof(lsw.SolveInfo) == 24
    # lsw_fno_params: 6 int32 + uint64
    assert ctypes.sizeof(lsw._FnoParams) == 32
    # lsw_sweep_policy: 4 int32; lsw_sweep_info: double + 4 int32 + double + 2 int32
    assert ctypes.sizeof(lsw._SweepPolicy) == 16
    assert ctypes.sizeof(lsw.SweepInfo) == 40


def test_invalid_arguments_fail_without_touching_the_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.lsw_build_green.restype = ctypes.c_int
    assert lib.lsw_build_green(None, None, None) == 1          # LSW_ERR_INVALID_ARG
    lib.lsw_apply_operator.restype = ctypes.c_int
    assert lib.lsw_apply_operator(None, 0, None, None, None, None, 1, 0, None) == 1


def _header_struct_fields(name):
    """Field names, in order, of `typedef struct { ... } name;` in lsw.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct\s*\{([^}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "int32_t nz, nx" / "double h" / "const double* velocity" / "lsw_grid grid"
        head, *rest = decl.split(",")
        names = [head.split()[-1]] + [r.strip() for r in rest]
        fields += [n.lstrip("*") for n in names]
    return fields


@pytest.mark.parametrize("cname,pyname", [("lsw_grid", "_Grid"), ("lsw_box", "_Box"), ("lsw_hparams", "_HParams"),
                                          ("lsw_solve_params", "_SolveParams"), ("lsw_solve_info", "SolveInfo"),
                                          ("lsw_problem", "_Problem"), ("lsw_fno_params", "_FnoParams"),
                                          ("lsw_sweep_policy", "_SweepPolicy"), ("lsw_sweep_info", "SweepInfo")])
def test_binding_struct_fields_follow_the_header(cname, pyname):
    from paper_2005_01372_gb300 import lsw
    want = _header_struct_fields(cname)
    got = [f[0] for f in getattr(lsw, pyname)._fields_]
    assert got == want, (cname, got, want)


def _header_enum(name):
    """{enumerator: value} of `typedef enum { ... } name;` in lsw.h."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    m = re.search(r"typedef enum\s*\{([^}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    out = {}
    for item in m.group(1).split(","):
        k, v = (t.strip() for t in item.split("="))
        out[k] = int(v)
    return out


@pytest.mark.parametrize("cname,names", [
    ("lsw_prec", {"LSW_C128": "C128", "LSW_C64": "C64", "LSW_MIXED": "MIXED", "LSW_BF16": "BF16"}),
    ("lsw_h_kind", {"LSW_H_LOWRANK_SMW": "H_LOWRANK_SMW", "LSW_H_HODLR": "H_HODLR"}),
])
def test_binding_constants_follow_the_header(cname, names):
    from paper_2005_01372_gb300 import lsw
    enum = _header_enum(cname)
    assert set(enum) == set(names), (cname, sorted(enum))
    for cn, pyn in names.items():
        assert getattr(lsw, pyn) == enum[cn], (cn, pyn)

