"""The C-ABI library builds, loads and exports every entry point include/gp2s.h declares (no GPU
compute here: only host-side calls that need no device)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gp2s.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gp2s_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2512_06143_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    fns = declared_functions()
    for f in ["gp2s_assemble", "gp2s_solve", "gp2s_logdet", "gp2s_lml", "gp2s_lml_grad", "gp2s_lml_batched",
              "gp2s_create", "gp2s_destroy", "gp2s_last_error", "gp2s_opts_default", "gp2s_csr"]:
        assert f in fns


def test_library_exports_every_declared_symbol(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_2512_06143_gb300 as gp
    assert set(gp.EXPORTED) == set(declared_functions())


def test_host_only_calls(lib):
    import paper_2512_06143_gb300 as gp
    gp.load()
    o = gp.default_opts()
    assert o.precision == gp.PREC_MIXED and o.probes == 64 and o.lanczos_steps == 100
    assert o.tol_refine == 1e-8 and o.n_exact == 20000
    assert gp.load().gp2s_num_params(3, 8) == 42


def test_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2512_06143_gb300 as gp
    with pytest.raises(gp.GP2SError):
        gp.Context(0)


def test_struct_layouts_match_header(tmp_path):
    # sizes and field offsets of the public structs as a C compiler sees the header, against the
    # ctypes mirrors of the Python binding
    import subprocess
    import paper_2512_06143_gb300 as gp
    structs = {"gp2s_hyper": gp._Hyper, "gp2s_opts": gp.Opts, "gp2s_assemble_info": gp.AssembleInfo,
               "gp2s_solve_info": gp.SolveInfo, "gp2s_logdet_info": gp.LogdetInfo, "gp2s_lml_info": gp.LmlInfo,
               "gp2s_csr_view": gp.CsrView}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gp2s.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {}
    for l in out:
        if l.strip():
            a, b, v = l.split()
            got[(a, b)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
