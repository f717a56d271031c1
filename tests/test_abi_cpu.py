"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every entry point include/*.h declares; host-side argument checks work
without touching the device."""
import ctypes
import glob
import os
import re

import pytest

from paper_2302_05662_gb300 import binding
from paper_2302_05662_gb300 import build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_mod.build()
    return binding.load_library()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:SPMV_API\s+)?(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(spmv_[A-Za-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    decl = declared_functions()
    assert "spmv_create" in decl and "spmv_run" in decl
    for name in decl:
        assert hasattr(lib, name), name
    assert decl == set(binding.EXPORTED)


def test_only_the_abi_is_exported(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True,
                         text=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert declared_functions() <= syms
    assert not [s for s in syms if s.startswith("_Z")], "C++ symbols leak out of the library"


def test_config_default_host_only(lib):
    cfg = binding.spmv_config()
    lib.spmv_config_default(ctypes.byref(cfg), binding.FMT_BSR)
    assert cfg.as_dict() == {"format": 4, "threads_per_block": 256, "threads_per_row": 0, "unroll": 0,
                             "regcap": 0, "carveout": -1, "bsr_block": 4, "hyb_ell_width": 0}
    lib.spmv_config_default(ctypes.byref(cfg), binding.FMT_ELL)
    assert cfg.format == binding.FMT_ELL and cfg.unroll == 0 and cfg.regcap == 0


def test_host_argument_errors(lib):
    h = ctypes.c_void_p()
    assert lib.spmv_create(ctypes.byref(h), -1, 3, 0, None, None, None, 0, None, None) == -1
    assert b"negative" in lib.spmv_last_error()
    assert lib.spmv_create(ctypes.byref(h), 3, 3, 5, None, None, None, 0, None, None) == -1
    assert lib.spmv_create(ctypes.byref(h), 3, 3, 0, None, None, None, 7, None, None) == -1
    assert lib.spmv_create(ctypes.byref(h), 1 << 31, 3, 0, None, None, None, 0, None, None) == -4
    assert lib.spmv_run(None, 1.0, None, 0.0, None, None) == -1
    assert lib.spmv_destroy(None) == 0
    assert lib.spmv_get_info(None, None) == -1


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "spmv.h"

int main(void) {
    spmv_config cfg;
    spmv_handle h = NULL;
    spmv_config_default(&cfg, SPMV_FMT_SELL);
    if (cfg.format != SPMV_FMT_SELL || cfg.threads_per_block != 256) return 1;
    if (spmv_create(&h, -1, 3, 0, NULL, NULL, NULL, SPMV_F64, NULL, NULL) != SPMV_ERR_INVALID) return 2;
    if (h != NULL || strstr(spmv_last_error(), "negative") == NULL) return 3;
    if (spmv_get_panel_limit() != SPMV_PANEL_LIMIT_MAX) return 4;
    if (spmv_set_panel_limit(0) != SPMV_ERR_INVALID) return 5;
    if (spmv_destroy(NULL) != SPMV_OK) return 6;
    printf("ok\n");
    return 0;
}
"""


def test_header_is_plain_c_and_a_c_program_links(lib, tmp_path):
    """include/spmv.h compiles as strict C99 and as C++; a C program links
    against the library and runs its host-only paths (no GPU touched)."""
    import shutil
    import subprocess
    inc = os.path.join(ROOT, "include")
    for compiler, std in (("gcc", "-std=c99"), ("g++", "-std=c++17")):
        if shutil.which(compiler) is None:
            pytest.skip(f"{compiler} not installed")
        lang = "c" if compiler == "gcc" else "c++"
        r = subprocess.run([compiler, std, "-x", lang, "-pedantic", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                            "-I", inc, os.path.join(inc, "spmv.h")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    libdir = os.path.dirname(binding.LIB_PATH)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", inc, str(src), "-o", str(exe), "-L", libdir,
                        "-l:" + os.path.basename(binding.LIB_PATH), "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)


class _FakeDeviceTensor:
    """Stands in for a CUDA tensor in the binding's host-side checks."""
    is_cuda = True

    def __init__(self, n, dtype, contiguous=True):
        self.n, self.dtype, self.contiguous = n, dtype, contiguous

    def numel(self):
        return self.n

    def is_contiguous(self):
        return self.contiguous

    def data_ptr(self):
        return 1 << 20


def test_binding_refuses_host_strided_short_and_mistyped_buffers():
    """Buffers that would send kernels to host memory or past an end are
    refused in the binding, with SPMV_ERR_INVALID, before any call."""
    import torch
    E = binding.SpmvError
    F = _FakeDeviceTensor
    with pytest.raises(E) as ei:
        binding._ptr(torch.zeros(3))
    assert ei.value.status == -1 and "CUDA" in str(ei.value)
    with pytest.raises(E):
        binding._ptr(F(8, torch.float64, contiguous=False))
    assert binding._ptr(None) is None and binding._ptr(F(8, torch.float64)) == 1 << 20
    assert binding._vec(F(8, torch.float64), 8, binding.SPMV_F64, "x") == 1 << 20
    assert binding._vec(F(8, torch.float32), 5, binding.SPMV_BF16, "x") == 1 << 20
    assert binding._vec(None, 0, binding.SPMV_F64, "y") is None
    for t, need, vt in ((F(7, torch.float64), 8, binding.SPMV_F64),      # too short
                        (F(8, torch.float32), 8, binding.SPMV_F64),      # fp32 vector, fp64 matrix
                        (F(8, torch.float64), 8, binding.SPMV_F32),      # fp64 vector, fp32 matrix
                        (F(8, torch.bfloat16), 8, binding.SPMV_BF16),    # bf16 matrices take fp32 vectors
                        (None, 1, binding.SPMV_F64)):
        with pytest.raises(E) as ei:
            binding._vec(t, need, vt, "x")
        assert ei.value.status == -1
    i32, i64 = torch.int32, torch.int64
    for r, c, v in ((F(4, i64), F(4, i32), F(4, torch.float64)),
                    (F(4, i32), F(3, i32), F(4, torch.float64)),
                    (F(4, i32), F(4, i32), F(4, torch.float16)),
                    (F(4, i32), None, F(4, torch.float64))):
        with pytest.raises(E):
            binding._triplets(r, c, v)
    assert binding._triplets(F(4, i32), F(4, i32), F(4, torch.bfloat16))[:2] == (4, binding.SPMV_BF16)
    assert binding._triplets(None, None, None)[0] == 0
    with pytest.raises(E) as ei:            # host vectors never reach the library
        binding.spmv_run(None, 1.0, torch.zeros(3), 0.0, torch.zeros(3))
    assert ei.value.status == -1
