"""The C ABI library builds, loads and exports every symbol include/eda.h declares (no GPU needed).

Calls made here never reach the device: argument validation rejects them first, and
eda_strerror / eda_config_default are host-only.
"""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "eda.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eda_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1512_06500_gb300 import build_lib, eda
    path = build_lib.build()
    return eda.load(path), path


def test_header_matches_binding_list(lib):
    from paper_1512_06500_gb300 import eda
    assert _declared() == sorted(eda.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    _, path = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [s for s in _declared() if s not in syms]
    assert not missing, missing


def test_host_only_calls(lib):
    from paper_1512_06500_gb300 import eda
    L, _ = lib
    assert L.eda_strerror(0) == b"success"
    assert L.eda_strerror(-8).startswith(b"not converged")
    c = eda.config()
    assert (c.prec, c.block_b, c.m_max, c.check_every, c.tau, c.c2) == (0, 8, 0, 1, 10.0, 0.0)


def test_invalid_arguments_rejected_before_device_work(lib):
    from paper_1512_06500_gb300 import eda
    L, _ = lib
    h = ctypes.c_void_p()
    c = eda.config()
    # null sample pointer, zero dimension, k > n
    assert L.eda_build(None, 0, 10, 5, 10, None, 2, ctypes.byref(c), None, ctypes.byref(h)) == -1
    assert L.eda_build(ctypes.c_void_p(16), 0, 0, 5, 10, ctypes.c_void_p(16), 2, ctypes.byref(c), None,
                       ctypes.byref(h)) == -1
    assert L.eda_build(ctypes.c_void_p(16), 0, 10, 5, 10, ctypes.c_void_p(16), 6, ctypes.byref(c), None,
                       ctypes.byref(h)) == -1
    bad = eda.config(block_b=0)
    assert L.eda_build(ctypes.c_void_p(16), 0, 10, 5, 10, ctypes.c_void_p(16), 2, ctypes.byref(bad), None,
                       ctypes.byref(h)) == -1
    assert L.eda_solve(None, 3, 1e-6, None, 0, None, None, None, None, None) == -1
    assert L.eda_apply_exp(None, 0, 1.0, None, None, 10, 1, 0, None) == -1
    L.eda_destroy(None)


def test_product_path_has_no_oracle_or_cpu_fallback():
    # the package and the library sources never reference the oracle
    pkg = os.path.join(ROOT, "paper_1512_06500_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_batched_invalid_arguments_rejected_before_device_work(lib):
    from paper_1512_06500_gb300 import eda
    L, _ = lib
    c = eda.config()
    assert L.eda_solve_batched(None, -1, ctypes.byref(c), 0, None) == -1
    assert L.eda_solve_batched(None, 2, ctypes.byref(c), 0, None) == -1
    assert L.eda_solve_batched(None, 0, ctypes.byref(c), 0, None) == 0
    arr = (eda.Problem * 1)()
    # k > n, and (separately) a missing output pointer: rejected by validation alone
    arr[0] = eda.Problem(X=1, x_dtype=0, k=5, d=10, n=3, ldx=10, labels=1, t=2, block_b=0, tol=1e-6, V=1, lam=1)
    assert L.eda_solve_batched(arr, 1, ctypes.byref(c), 0, None) == -1
    arr[0] = eda.Problem(X=1, x_dtype=0, k=2, d=10, n=3, ldx=10, labels=1, t=2, block_b=0, tol=1e-6, V=0, lam=1)
    assert L.eda_solve_batched(arr, 1, ctypes.byref(c), 0, None) == -1


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not available")
def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of the C structs have the header's sizes and field offsets."""
    from paper_1512_06500_gb300 import eda
    checks = [("eda_config", eda.Config), ("eda_solve_info", eda.SolveInfo), ("eda_problem", eda.Problem)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for cname, py in checks:
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            cf = "lambda" if fname == "lam" else fname
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {cf}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-o", str(exe), str(src)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                              check=True).stdout.splitlines())
    for cname, py in checks:
        assert int(out[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(out[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


def test_library_has_no_undefined_internal_symbols(lib):
    """Every function of the library's own namespace that is referenced is defined in it."""
    _, path = lib
    out = subprocess.run(["nm", "-D", "--undefined-only", path], capture_output=True, text=True, check=True).stdout
    undefined = [line.split()[-1] for line in out.splitlines() if "_ZN3eda" in line or " eda_" in line]
    assert not undefined, undefined


def test_noalloc_rejects_overlaps_and_oversize_before_device_work(lib):
    """The no-allocation product checks its arguments on the host, before any CUDA call: Y may overlap
    none of X, H, K (it is written while they are still read), and m * b is bounded by the fixed
    scratch. The pointers here are never dereferenced."""
    L, _ = lib
    fn = L.eda_lowrank_exp_apply_noalloc
    d, m, b = 1000, 10, 4
    H, K, X, Y = 1 << 20, 1 << 24, 1 << 28, 1 << 32          # disjoint address ranges
    P = ctypes.c_void_p
    # Y inside H, inside K, inside X
    assert fn(P(H), d, m, P(K), P(X), P(H + 8 * 64), d, b, None) == -1
    assert fn(P(H), d, m, P(K), P(X), P(K), d, b, None) == -1
    assert fn(P(H), d, m, P(K), P(X), P(X + 8), d, b, None) == -1
    # m * b above the scratch (2^19 / 3 doubles), and ld < d
    assert fn(P(H), d, 2000, P(K), P(X), P(Y), d, 100, None) == -1
    assert fn(P(H), d, m, P(K), P(X), P(Y), d - 1, b, None) == -1
