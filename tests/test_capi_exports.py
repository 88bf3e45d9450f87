"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/ckks_mf.h."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ckks_mf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fhe_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2509_03024_gb300 import build, capi
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(capi.EXPORTS) == names


def test_binding_refuses_without_library(tmp_path, monkeypatch):
    from paper_2509_03024_gb300 import capi
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        capi.lib()


_CTYPE = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
          "size_t": ctypes.c_size_t, "double": ctypes.c_double, "int": ctypes.c_int}


def _header():
    src = open(os.path.join(ROOT, "include", "ckks_mf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return re.sub(r"\s+", " ", src)


def _prototypes():
    """{name: (return type, [parameter types])} of every entry point, parameter names stripped."""
    out = {}
    for ret, name, params in re.findall(r"(int|void|const char\*) (fhe_[a-z0-9_]+)\(([^)]*)\);", _header()):
        types = []
        for p in params.split(","):
            p = p.strip()
            stars = p.count("*")
            base = re.sub(r"\bconst\b|\*", " ", p).split()[0]
            types.append((base, stars))
        out[name] = (ret, types)
    return out


def _matches(ct, base, stars):
    if stars == 0:
        return ct is _CTYPE[base]
    if base == "char":      # strings in, and an out-parameter receiving a static string
        return ct is (ctypes.c_char_p if stars == 1 else ctypes.POINTER(ctypes.c_char_p))
    if stars == 2:          # an out-parameter receiving a handle
        return ct is ctypes.POINTER(ctypes.c_void_p)
    # one level of pointer: plain buffers and handles are void*, struct pointers may be typed
    if ct is ctypes.c_void_p:
        return True
    return hasattr(ct, "_type_") and issubclass(ct._type_, ctypes.Structure)


def test_binding_signatures_match_the_header():
    """Every ctypes prototype of the binding has the header's arity, scalar types and pointer
    levels, so a drifting argument list fails here instead of corrupting memory on a GPU."""
    from paper_2509_03024_gb300 import build, capi
    build.build()
    L = capi.lib()
    protos = _prototypes()
    assert sorted(protos) == sorted(capi.EXPORTS)
    for name, (ret, types) in protos.items():
        f = getattr(L, name)
        assert len(f.argtypes) == len(types), (name, f.argtypes, types)
        for i, (ct, (base, stars)) in enumerate(zip(f.argtypes, types)):
            assert _matches(ct, base, stars), (name, i, ct, base, stars)
        want = {"int": ctypes.c_int, "void": None, "const char*": ctypes.c_char_p}[ret]
        assert f.restype is want, (name, f.restype, ret)


def _struct_fields(name):
    body = re.search(r"typedef struct \{([^}]*)\} " + name + ";", _header()).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"(const )?([a-z0-9_]+)(\*?) (.*)", decl)
        for var in m.group(4).split(","):
            var = var.strip()
            fields.append((var.lstrip("*"), m.group(2), bool(m.group(3)) or var.startswith("*")))
    return fields


@pytest.mark.parametrize("cname,pyname", [("fhe_params", "Params"), ("fhe_ctx_info", "CtxInfo"),
                                          ("fhe_kernel_stat", "KernelStat"), ("fhe_mf_plan_info", "PlanInfo"),
                                          ("fhe_int_pipe_rates", "IntPipeRates"),
                                          ("fhe_tune_result", "TuneResult")])
def test_binding_structs_match_the_header(cname, pyname):
    from paper_2509_03024_gb300 import capi
    fields = _struct_fields(cname)
    py = getattr(capi, pyname)._fields_
    assert [f[0] for f in fields] == [p[0] for p in py], (cname, fields, py)
    for (name, base, ptr), (_, ct) in zip(fields, py):
        if ptr:
            assert ct is ctypes.c_char_p or hasattr(ct, "_type_"), (cname, name, ct)
        else:
            assert ct is _CTYPE[base], (cname, name, ct, base)


def test_buffer_marshalling_refuses_strided_views():
    import numpy as np
    import torch
    from paper_2509_03024_gb300 import capi
    a = np.zeros((4, 4))
    assert capi._ptr(a) == a.ctypes.data and capi._ptr(None) is None
    with pytest.raises(ValueError):
        capi._ptr(a[:, ::2])
    t = torch.zeros(4, 4, dtype=torch.int64)
    assert capi._ptr(t) == t.data_ptr()
    with pytest.raises(ValueError):
        capi._ptr(t.t())
