"""The C ABI library builds for sm_103a, loads without a GPU, exports every
entry point include/upr.h declares, and the binding's struct layouts match
the header's (checked against the C compiler)."""
from __future__ import annotations

import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "upr.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2308_15494_gb300 import build
    build.build()
    import paper_2308_15494_gb300 as upr
    return upr.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(upr_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound(lib):
    import paper_2308_15494_gb300 as upr
    names = declared_functions()
    assert "upr_create" in names and "upr_refine" in names and "upr_poll" in names
    for name in names:
        assert hasattr(lib, name), name
        assert name in upr.SIGNATURES, name
    out = subprocess.run(["nm", "-D", "--defined-only", upr.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (upr_\w+)", out))
    assert set(names) <= exported


def test_struct_layouts_match_header(lib):
    import ctypes
    import paper_2308_15494_gb300 as upr
    structs = {"upr_graph": upr.Graph, "upr_params": upr.Params, "upr_stats": upr.Stats,
               "upr_trace": upr.Trace, "upr_server_params": upr.ServerParams}
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"upr.h\"\nint main(void){\n"
    for cname in structs:
        src += f'printf("{cname} %zu\\n", sizeof({cname}));\n'
    for cname, cls in structs.items():
        for f, _ in cls._fields_:
            src += f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));\n'
    src += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        lines = subprocess.check_output([exe], text=True).split("\n")
    got = dict(l.split() for l in lines if l)
    for cname, cls in structs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, f"{cname}.{f}"


def test_host_only_entry_points(lib):
    import paper_2308_15494_gb300 as upr
    p = upr.upr_params_default()
    assert (p.t_num, p.t_den, p.tau1_num, p.tau1_den, p.max_subrounds, p.validate) == (7, 10, 1, 4, 64, 1)
    assert upr.status_name(upr.UPR_ERR_INFEASIBLE) == "UPR_ERR_INFEASIBLE"
    assert upr.status_name(0) == "UPR_OK"


def test_binding_fails_loudly_without_library(tmp_path, lib):
    import paper_2308_15494_gb300 as upr
    saved = upr._lib
    upr._lib = None
    try:
        with pytest.raises(ImportError):
            upr.load(str(tmp_path / "missing.so"))
    finally:
        upr._lib = saved
