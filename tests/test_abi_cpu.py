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

