"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports every
entry point that include/npfem.h declares (no compute call without a GPU)."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(npfem_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("npfem_create", "npfem_step", "npfem_destroy", "npfem_last_error", "npfem_step_host", "npfem_eval"):
        assert required in names


def test_library_builds_loads_and_exports_every_declared_symbol():
    from paper_1903_06479_gb300 import npfem
    L = npfem.lib()
    path = npfem.lib_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for name in declared_functions():
        assert name in exported, name
        assert getattr(L, name) is not None
    # the product binding has no CPU fallback: it never imports the oracle
    src = open(os.path.join(ROOT, "paper_1903_06479_gb300", "npfem.py")).read()
    assert "oracle" not in src


def test_default_opts_and_error_path_without_gpu():
    from paper_1903_06479_gb300 import npfem
    o = npfem.default_opts()
    assert o.precision == 1 and o.lbfgs_m == 5 and o.max_iter == 50 and abs(o.tol - 1e-6) < 1e-18
    # a null argument is rejected before any CUDA call
    import ctypes as C
    rc = npfem.lib().npfem_create(None, None, None, 0.1, 0, C.byref(C.c_void_p()))
    assert rc == -1 and b"null" in npfem.lib().npfem_last_error()
