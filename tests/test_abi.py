"""The C ABI builds, loads and exports every entry point that include/la.h
declares, and the Python binding's structs match the C layout (no GPU)."""

import ctypes
import os
import re
import subprocess

import pytest

from paper_1110_6231_gb300 import build as labuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
                 if f.endswith(".h"))


def declared_functions():
    names = []
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(la_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libla():
    path = labuild.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("la_solve", "la_solve_ex", "la_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(libla):
    out = subprocess.run(["nm", "-D", "--defined-only", labuild.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (la_\w+)$", out, flags=re.M))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        getattr(libla, f)


def test_status_strings_without_gpu(libla):
    libla.la_status_string.restype = ctypes.c_char_p
    libla.la_status_string.argtypes = [ctypes.c_int]
    for s in range(9):
        assert libla.la_status_string(s).startswith(b"LA_")
    assert libla.la_version() >= 100


def test_struct_layout_matches_header(tmp_path):
    import paper_1110_6231_gb300 as la
    src = tmp_path / "layout.c"
    fields = {name: [f for f, _ in getattr(la, name)._fields_]
              for name in ("la_options", "la_stats", "la_batch_options", "la_batch_stats",
                           "la_maxflow_options", "la_maxflow_stats")}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "la.h"', "int main(void){"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for st, fs in fields.items():
        cls = getattr(la, st)
        assert int(got[st]) == ctypes.sizeof(cls), st
        for f in fs:
            assert int(got[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_1110_6231_gb300 as la
    monkeypatch.setattr(la, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(la, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        la.lib()


def test_invalid_arguments_rejected_on_host(libla):
    """Argument errors return before anything touches a device."""
    libla.la_solve.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p]
    libla.la_solve.restype = ctypes.c_int
    assert libla.la_solve(None, -1, None, None, None) == 1
    assert libla.la_solve(None, 4, None, None, ctypes.c_void_p(8)) == 1      # NULL cost
    assert libla.la_solve(ctypes.c_void_p(8), 4, None, None, None) == 1      # NULL cost_out
    assert libla.la_solve(ctypes.c_void_p(8), (1 << 20), None, None, ctypes.c_void_p(8)) == 1


def test_probe_rejects_bad_arguments_on_host(libla):
    f = libla.la_probe_read
    f.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.POINTER(ctypes.c_float)]
    f.restype = ctypes.c_int
    ms = ctypes.c_float()
    assert f(None, 16, 1, None, ctypes.byref(ms)) == 1                     # NULL buffer
    assert f(ctypes.c_void_p(256), 24, 1, None, ctypes.byref(ms)) == 1     # not a multiple of 16
    assert f(ctypes.c_void_p(256), 16, 0, None, ctypes.byref(ms)) == 1     # no pass
    assert f(ctypes.c_void_p(264), 16, 1, None, ctypes.byref(ms)) == 1     # misaligned
    assert f(ctypes.c_void_p(256), 16, 1, None, None) == 1                 # NULL ms_out
