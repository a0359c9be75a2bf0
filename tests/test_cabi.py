"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports every
function include/acac.h declares, and its structs have the layout the binding
assumes.  No compute call is made (there may be no GPU)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "acac.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2007_04560_gb300 import build
    build.build()
    import paper_2007_04560_gb300.acac as A
    return A.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(acac_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("acac_create", "acac_step", "acac_energy", "acac_destroy", "acac_status_string",
                     "acac_residual", "acac_jacobian", "acac_jvp", "acac_spmv", "acac_ras_factor",
                     "acac_ras_apply", "acac_gmres", "acac_nks_solve", "acac_step_host"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    import paper_2007_04560_gb300.acac as A
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in A.SIGNATURES, "binding lacks " + name


def test_struct_layout_matches_binding():
    import paper_2007_04560_gb300.acac as A
    fields_p = [f for f, _ in A.acac_params._fields_]
    fields_i = [f for f, _ in A.acac_step_info._fields_]
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "acac.h"', "int main(void){",
           'printf("%zu %zu\\n", sizeof(acac_params), sizeof(acac_step_info));']
    for f in fields_p:
        src.append('printf("p %s %%zu\\n", offsetof(acac_params, %s));' % (f, f))
    for f in fields_i:
        src.append('printf("i %s %%zu\\n", offsetof(acac_step_info, %s));' % (f, f))
    src.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write("\n".join(src))
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe])
        out = subprocess.check_output([exe], text=True).split("\n")
    sp, si = map(int, out[0].split())
    assert sp == ctypes.sizeof(A.acac_params)
    assert si == ctypes.sizeof(A.acac_step_info)
    for line in out[1:]:
        if not line:
            continue
        kind, name, off = line.split()
        cls = A.acac_params if kind == "p" else A.acac_step_info
        assert getattr(cls, name).offset == int(off), name


def test_defaults_and_validation_without_gpu(lib):
    import paper_2007_04560_gb300.acac as A
    p = A.acac_params()
    lib.acac_default_params(ctypes.byref(p))
    assert (p.n[0], p.n[1], p.taylor_S, p.gmres_restart, p.cgs_refine) == (64, 64, 10, 30, 1)
    assert p.newton_rtol == 1e-8 and p.gmres_rtol == 1e-6
    assert lib.acac_status_string(-5).decode() == "time step fell below dt_min"
    h = ctypes.c_void_p()
    # argument errors are detected before any CUDA call
    for field, bad in (("dim", 4), ("taylor_S", 0), ("gamma", -1.0), ("batch", 0), ("batch", 1025),
                       ("gmres_restart", 99), ("subdomain_solver", 4), ("subdomain_solver", -1)):
        q = A.acac_params()
        lib.acac_default_params(ctypes.byref(q))
        setattr(q, field, bad)
        assert lib.acac_create(ctypes.byref(q), None, ctypes.byref(h)) == A.E_ARG, field
    q = A.acac_params()
    lib.acac_default_params(ctypes.byref(q))
    q.ras_parts[0] = 1                          # periodic needs >= 2 boxes per direction
    assert lib.acac_create(ctypes.byref(q), None, ctypes.byref(h)) == A.E_ARG
    q = A.acac_params()
    lib.acac_default_params(ctypes.byref(q))
    q.n[0] = q.n[1] = 1024
    q.ras_parts[0] = q.ras_parts[1] = 2          # 514 x 514-cell boxes: too large for a fill solver
    q.subdomain_solver = 3
    assert lib.acac_create(ctypes.byref(q), None, ctypes.byref(h)) == A.E_ARG
    assert lib.acac_kernel_name(8).decode() == "ras_apply"


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import importlib

    import paper_2007_04560_gb300.acac as A
    monkeypatch.setattr(A, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(A, "_LIB", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        A.load()
    importlib.reload(A)


def test_python_parameters_match_the_c_struct():
    """Every field of acac_params has a Params field of the same name and vice versa, so no
    setting is silently dropped or defaulted on its way to the library; and the binding
    refuses host tensors before it reaches the library."""
    import dataclasses
    import paper_2007_04560_gb300.acac as A
    from workloads import Params
    py = {f.name for f in dataclasses.fields(Params)}
    c = {n for n, _ in A.acac_params._fields_}
    assert py == c
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        A._dev(torch.zeros(4), torch.float64, 4, "u")
    with pytest.raises(TypeError):
        A._dev([0.0] * 4, torch.float64, 4, "u")
