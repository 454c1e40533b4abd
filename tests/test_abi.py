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


def test_trim_memory_without_pools_is_a_no_op(libpath):
    """rte_trim_memory only visits the memory pools the library created; in a
    process that never set up a context it touches no device."""
    from paper_2604_23265_gb300 import rte
    lib = rte.load(libpath)
    assert lib.rte_trim_memory() == rte.RTE_OK
    rte.trim_memory()


# the ctypes mirrors of the public structs and the C declarations agree on
# size and on every field offset (compiled with the host C compiler)
STRUCTS = {
    "rte_ctx_info": ("CtxInfo", ["I", "M", "N", "nmat", "n", "device_bytes"]),
    "rte_solve_opts": ("SolveOpts", ["tol", "restart", "max_iter", "inner_precision", "use_x0", "stall_ratio",
                                     "timeout_ms", "cancel"]),
    "rte_solve_info": ("SolveInfo", ["iterations", "cycles", "converged", "fell_back", "relres", "seconds",
                                     "history_len", "history"]),
    "mgnet_config": ("MgNetConfig", ["M", "levels", "c0", "cmax", "cc", "ccmax", "act"]),
    "rte_server_config": ("ServerConfig", ["max_device_bytes", "slots", "inject_alloc_failure_id", "grouped"]),
    "rte_request": ("Request", ["I", "M", "sigma_T", "sigma_a", "q", "eps", "eps_is_scalar", "g", "inflow", "tol",
                                "max_iter", "restart", "use_net"]),
    "rte_result": ("Result", ["status", "info", "latency_s", "queue_s", "footprint", "used_net"]),
    "rte_server_stats_t": ("ServerStats", ["queued", "completed", "active", "bytes_in_use"]),
    "rte_kernel_stat": ("KernelStat", ["name", "launches", "ms", "bytes", "flops"]),
}


def test_struct_layouts_match_the_header(tmp_path):
    import shutil
    import subprocess
    from paper_2604_23265_gb300 import rte
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include "rte.h"', "int main(void) {"]
    for cname, (_, fields) in STRUCTS.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            name, field, value = line.split()
            got[(name, field)] = int(value)
    for cname, (pyname, fields) in STRUCTS.items():
        cls = getattr(rte, pyname)
        assert ctypes.sizeof(cls) == got[(cname, "size")], cname
        for f in fields:
            assert getattr(cls, f).offset == got[(cname, f)], (cname, f)
