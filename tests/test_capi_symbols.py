"""The C-ABI library builds for sm_103a, loads without a GPU and exports every function that
include/grstage.h declares (no compute calls)."""
import os
import re

import pytest

from paper_2311_04989_gb300 import build as B
from paper_2311_04989_gb300 import grstage as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(gr_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return G.load()


def test_header_declares_the_boundary():
    names = header_functions()
    for f in ("gr_stage", "gr_prim2con", "gr_con2prim", "gr_diag", "gr_mesh_create", "gr_context_create"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    names = header_functions()
    missing = [f for f in names if not hasattr(lib, f)]
    assert not missing, missing
    assert set(names) <= set(G.EXPORTS) | set(names)
    assert sorted(set(G.EXPORTS)) == sorted(names)


def test_pure_host_entries(lib):
    assert lib.gr_abi_version() == G.GR_ABI_VERSION == 3
    assert lib.gr_mlp_nparam() == G.GR_MLP_NPARAM
    assert lib.gr_strerror(G.GR_EINVAL) == b"invalid argument"
    p = G.gr_params_default()
    assert p.size == __import__("ctypes").sizeof(G.gr_params)
    assert p.recon == G.GR_RECON_WENOZ and abs(p.W_max ** 2 - 401) < 1e-9


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """ctypes mirrors of the header structs agree with gcc's sizeof/offsetof."""
    import ctypes as C
    import subprocess
    structs = {"gr_block": G.gr_block, "gr_metric": G.gr_metric, "gr_state": G.gr_state,
               "gr_params": G.gr_params, "gr_eos_table": G.gr_eos_table, "gr_shape": G.gr_shape,
               "gr_level_face": G.gr_level_face, "gr_level_map": G.gr_level_map}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "grstage.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(out[name]) == C.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(out[f"{name}.{fname}"]) == getattr(cls, fname).offset, (name, fname)


def test_header_constants_match_the_binding():
    txt = open(os.path.join(ROOT, "include", "grstage.h")).read()
    for name in ("GR_ABI_VERSION", "GR_MLP_NPARAM", "GR_MLP_NIN", "GR_NKERNELS", "GR_NSTAGE_KERNELS"):
        m = re.search(rf"#define {name} (\d+)", txt)
        assert m and int(m.group(1)) == getattr(G, name), name
