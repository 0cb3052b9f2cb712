"""The C-ABI library builds, loads and exports every symbol include/rr.h
declares (CPU only: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rr.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(rr_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def librr():
    from paper_2506_11273_gb300 import build
    path = build.build()
    return path


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rr_compute_keys", "rr_sort", "rr_permute", "rr_trace", "rr_build_bvh"):
        assert required in names


def test_library_exports_every_declared_symbol(librr):
    lib = ctypes.CDLL(librr)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", librr], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (rr_[a-z_0-9]+)", out))
    assert set(declared_functions()) <= exported


def test_binding_lists_every_declared_symbol(librr):
    from paper_2506_11273_gb300 import rr
    assert sorted(rr.EXPORTS) == declared_functions()
    rr.lib()  # argtypes resolve against the library


def test_status_strings_without_a_gpu(librr):
    from paper_2506_11273_gb300 import rr
    assert rr.rr_status_string(0) == "ok"
    assert rr.rr_status_string(1) == "invalid argument"
    assert rr.rr_status_string(4) == "device wait timed out"


def test_build_targets_sm_103a_only():
    from paper_2506_11273_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2506_11273_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                text = open(os.path.join(dirpath, f), errors="replace").read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "liboracle" not in text and "oracle.c" not in text, f


def test_host_argument_checks_without_a_gpu(librr):
    """Entry points that need no device answer on the host: workspace sizes
    follow the documented layout and bad arguments are refused before any
    device work; calls that need a device fail with a status, not a crash."""
    lib = ctypes.CDLL(librr)
    lib.rr_sort_workspace_size.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.POINTER(ctypes.c_size_t)]
    size = ctypes.c_size_t()
    prev = 0
    for n in (1, 1000, 4096, 4097, 1 << 20, 8294400):
        for bits, radix in ((32, 8), (64, 8), (64, 4), (16, 4)):
            assert lib.rr_sort_workspace_size(n, bits, radix, ctypes.byref(size)) == 0
            kb = 8 if bits > 32 else 4
            passes = -(-bits // radix)
            # two key buffers and one value buffer, plus counts and look-back words
            assert size.value >= 2 * kb * n + 4 * n + passes * (1 << radix) * 4
        assert lib.rr_sort_workspace_size(n, 64, 8, ctypes.byref(size)) == 0
        assert size.value >= prev
        prev = size.value
    for bits, radix, n in ((0, 8, 10), (65, 8, 10), (32, 5, 10), (32, 8, 1 << 30)):
        assert lib.rr_sort_workspace_size(n, bits, radix, ctypes.byref(size)) == 1  # RR_ERR_INVALID_ARG
    lib.rr_compute_keys.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_uint32] + [ctypes.c_void_p] * 3
    assert lib.rr_compute_keys(None, None, 10, None, None, None) == 1  # NULL params: refused first
    import torch
    if not torch.cuda.is_available():
        lib.rr_build_bvh.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p)]
        tri = (ctypes.c_float * 9)(0, 0, 0, 1, 0, 0, 0, 1, 0)
        h = ctypes.c_void_p()
        assert lib.rr_build_bvh(tri, 1, ctypes.byref(h)) == 2  # RR_ERR_CUDA: no device, no crash
        assert not h.value


def test_header_is_plain_c_and_links(librr, tmp_path):
    """include/rr.h compiles as C11 and as C++17, and a C program built
    against it links with librr.so and calls a host-only entry point."""
    import shutil
    if shutil.which("gcc") is None or shutil.which("g++") is None:
        pytest.skip("gcc/g++ missing")
    inc = os.path.dirname(HEADER)
    for cc, std, lang in (("gcc", "-std=c11", "c"), ("g++", "-std=c++17", "c++")):
        r = subprocess.run([cc, "-fsyntax-only", std, "-Wall", "-Wextra", "-Werror", "-x", lang, HEADER],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
    src = tmp_path / "use_rr.c"
    src.write_text('#include <stdio.h>\n#include <string.h>\n#include "rr.h"\n'
                   'int main(void) {\n'
                   '    const char *s = rr_status_string(RR_ERR_INVALID_ARG);\n'
                   '    if (!s || strcmp(s, "invalid argument") != 0) return 1;\n'
                   '    size_t b = 0;\n'
                   '    if (rr_sort_workspace_size(1000, 64, 8, &b) != RR_OK || b == 0) return 2;\n'
                   '    if (rr_sort_workspace_size(1000, 65, 8, &b) != RR_ERR_INVALID_ARG) return 3;\n'
                   '    puts("ok");\n'
                   '    return 0;\n'
                   '}\n')
    exe = tmp_path / "use_rr"
    r = subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), librr, "-Wl,-rpath," + os.path.dirname(librr),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
