"""The C-ABI library builds, loads and exports every symbol include/*.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            text = "\n".join(l for l in text.splitlines() if not l.lstrip().startswith("#"))
            for m in re.finditer(r"RTE_API\s+[^;]*?\b(\w+)\s*\(", text):
                names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2604_23265_gb300 import _build
    return _build.build()


def test_header_declares_core_calls():
    names = _declared()
    for core in ("rte_setup", "rte_apply", "rte_solve", "rte_block_apply", "rte_reconstruct"):
        assert core in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header(libpath):
    from paper_2604_23265_gb300 import rte
    lib = rte.load(libpath)
    assert set(rte.SIGNATURES) <= _declared()
    assert _declared() <= set(rte.SIGNATURES) | _optional_bindings()
    assert lib is rte.load()


def _optional_bindings():
    from paper_2604_23265_gb300 import rte
    return set(getattr(rte, "EXTRA_SIGNATURES", {}))


def test_setup_rejects_bad_arguments_without_gpu(libpath):
    """Argument checks happen before any device work."""
    from paper_2604_23265_gb300 import rte
    lib = rte.load(libpath)
    out = ctypes.c_void_p()
    one = (ctypes.c_double * 4)(1.0, 1.0, 1.0, 1.0)
    p = ctypes.cast(one, ctypes.c_void_p)
    st = lib.rte_setup(ctypes.byref(rte.Grid(2)), ctypes.byref(rte.Quadrature(6)), p, p, p, p, 1,
                       0.0, None, None, ctypes.byref(out))
    assert st == rte.RTE_EINVAL and not out.value
    assert b"multiple of 4" in lib.rte_last_error(None)
    st = lib.rte_setup(ctypes.byref(rte.Grid(2)), ctypes.byref(rte.Quadrature(8)), p, p, p, p, 1,
                       1.0, None, None, ctypes.byref(out))
    assert st == rte.RTE_EINVAL
    opts = rte.SolveOpts()
    lib.rte_solve_opts_default(ctypes.byref(opts))
    assert opts.tol == 1e-8 and opts.restart == 50 and opts.inner_precision == rte.RTE_F32
