"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol that include/apf.h declares, and refuses to run without a device."""
import ctypes
import os
import re
import shutil
import subprocess
import tempfile

import pytest

from paper_2306_09257_gb300 import apf, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build_lib()
    return apf.load_library()


def declared_symbols():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    return sorted(set(re.findall(r"\b(apf_[A-Za-z_]+)\s*\(", src)))


def test_header_matches_binding_list():
    assert declared_symbols() == sorted(apf.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_version(lib):
    assert lib.apf_version() >> 16 == 2


def test_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = lib.apf_create(ctypes.byref(h), 0, apf.APF_FP64)
    assert rc == apf.APF_ECUDA
    assert h.value is None
    assert b"device" in lib.apf_last_error(None)


def test_create_rejects_bad_precision(lib):
    h = ctypes.c_void_p()
    assert lib.apf_create(ctypes.byref(h), 0, 77) == apf.APF_EINVAL
    # the precision enum: 0 float64, 1 TF32 (reserved, not built), 2 bf16x3
    assert (apf.APF_FP64, apf.APF_MIXED_TF32, apf.APF_MIXED_BF16X3) == (0, 1, 2)
    assert lib.apf_create(ctypes.byref(h), 0, apf.APF_MIXED_TF32) == apf.APF_EINVAL
    assert b"TF32" in lib.apf_last_error(None)


def test_null_context_calls(lib):
    assert lib.apf_set_grid(None, 64, 100, 20, 20, 16.0, None) == apf.APF_EINVAL
    assert lib.apf_solve_S(None, None, None) == apf.APF_EINVAL
    lib.apf_destroy(None)


def test_new_entry_points_reject_null_context(lib):
    assert lib.apf_set_ridges(None, None, 0, 1, 4.0, 1.0, -1, 1, 2.25, 1.0, None, None) == apf.APF_EINVAL
    assert lib.apf_ridge_grad(None, None, None, None) == apf.APF_EINVAL
    assert lib.apf_reflection(None, None, 0, None, None) == apf.APF_EINVAL
    assert lib.apf_reverse_S(None, None, None) == apf.APF_EINVAL
    assert lib.apf_substrate_orders(None, None, None) == apf.APF_EINVAL
    assert lib.apf_set_krylov(None, 2) == apf.APF_EINVAL


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_headers_compile_as_plain_c():
    """The public headers are plain C (no C++ or torch types): a C99 file that
    includes both compiles."""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "use.c")
        with open(src, "w") as f:
            f.write('#include "apf.h"\n#include "apf_surrogate.h"\n'
                    "int main(void) { apf_stats st; apf_profile pr; (void)st; (void)pr; return apf_version() < 0; }\n")
        r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I", os.path.join(ROOT, "include"),
                            src], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_every_kernel_waits_for_its_predecessor():
    """Library kernels are launched with programmatic dependent launch, so
    each must wait for the preceding grid (griddepcontrol.wait) before it
    touches global memory: every __global__ function in csrc/ (the surrogate
    kernels are launched without the attribute) starts with
    APF_KERNEL_PROLOGUE, or calls pdl_wait in its body (the GEMM kernels,
    after their barrier and tensor-memory set-up)."""
    csrc = os.path.join(ROOT, "paper_2306_09257_gb300", "csrc")
    missing = []
    for f in sorted(os.listdir(csrc)):
        if not f.endswith(".cu") or f == "surrogate.cu":
            continue
        src = open(os.path.join(csrc, f)).read()
        for m in re.finditer(r"__global__\s+void[^;{]*?\)\s*\{", src, re.S):
            # the kernel body: up to the matching closing brace
            depth, i = 1, m.end()
            while depth and i < len(src):
                depth += {"{": 1, "}": -1}.get(src[i], 0)
                i += 1
            body = src[m.end():i]
            name = re.search(r"(k_\w+)\s*\(", m.group(0))
            if "APF_KERNEL_PROLOGUE" not in body[:200] and "pdl_wait()" not in body:
                missing.append(f"{f}:{name.group(1) if name else '?'}")
    assert not missing, missing
