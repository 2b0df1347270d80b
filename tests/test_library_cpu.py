"""CPU-side checks of the CUDA library: it builds for sm_103a, loads, and
exports every entry point that include/swe.h declares.  No GPU work."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(swe_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1309_1230_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("swe_create", "swe_set_bed", "swe_set_state", "swe_step", "swe_get_state", "swe_destroy"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_pure_host_calls(lib):
    from paper_1309_1230_gb300 import swe
    p = swe.swe_params()
    L = swe.load()
    L.swe_params_default(ctypes.byref(p))
    assert p.g == 9.81 and p.cfl == 0.5 and p.h_dry == 1e-3 and p.dir_cycle == 1
    assert p.kernel == swe.SWE_KERNEL_FUSED and p.precision == swe.SWE_FP64
    assert L.swe_status_string(3).decode() == "non-finite state"
    # NULL out-pointer is rejected before any CUDA call
    assert L.swe_create(ctypes.byref(p), None) == swe.SWE_ERR_ARG
    bad = swe.swe_params()
    L.swe_params_default(ctypes.byref(bad))
    bad.nx = 0
    out = ctypes.c_void_p()
    assert L.swe_create(ctypes.byref(bad), ctypes.byref(out)) == swe.SWE_ERR_ARG
    assert out.value is None


def test_product_path_does_not_import_the_oracle():
    """The package never reaches into oracle/ (the oracle is test-only)."""
    pkg = os.path.join(ROOT, "paper_1309_1230_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower().replace("oracle", "", 0) or "import oracle" not in text
                assert "from oracle" not in text and "import oracle" not in text and "swe_oracle" not in text


def test_ctypes_layout_matches_the_header(tmp_path):
    """The binding's structs have the C layout of include/swe.h (gcc decides)."""
    import subprocess
    from paper_1309_1230_gb300 import swe
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "swe.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(swe_params), sizeof(swe_step_info),'
                   ' offsetof(swe_params, stream), offsetof(swe_params, reserved), offsetof(swe_step_info, flags));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    want = [ctypes.sizeof(swe.swe_params), ctypes.sizeof(swe.swe_step_info),
            swe.swe_params.stream.offset, swe.swe_params.reserved.offset, swe.swe_step_info.flags.offset]
    assert got == want


def test_kernel_hash_ignores_comments_only():
    """bench.py reports the recorded DRAM traffic only while the kernel code
    hashes to the captured value; comments and layout must not count, code
    and string literals (inline PTX) must."""
    import bench
    a = 'int f(){ asm("mov.b64 %0, 1; // not a comment"); return 1; } // note\n/* block\ncomment */'
    b = 'int f(){   asm("mov.b64 %0, 1; // not a comment");\n return 1; }'
    c = 'int f(){ asm("mov.b64 %0, 2; // not a comment"); return 1; }'
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)
    assert "not a comment" in bench._code_only(a)


def test_checked_build_compiles_and_exports_the_abi():
    """The checked build (-DSWE_CHECKED: device-side index and alignment
    checks, NaN-poisoned planes) cross-compiles for sm_103a and exports the
    same entry points; the GPU test of what it checks is test_gpu_checked.py."""
    from paper_1309_1230_gb300 import _build, swe
    path = _build.build(checked=True)
    assert path == _build.LIB_CHECKED and os.path.exists(path)
    chk = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(chk, n)]
    assert not missing, f"declared but not exported by the checked build: {missing}"
    chk.swe_status_string.restype = ctypes.c_char_p
    assert chk.swe_status_string(swe.SWE_ERR_CHECK).decode() == "device-side check failed"
