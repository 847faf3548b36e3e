"""The allocation-free entry point (apf_solve_S_noalloc) against the regular
context-based float64 solve, through the C ABI.

It serves callers that cannot allocate device memory; its scratch is one
fixed device array shared by all calls, so the test makes two calls in a row
with different inputs and checks that the second does not see the first's
leftovers.  Collected last on purpose (file name), so a failure here comes
after every other test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_2306_09257_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_09257_gb300 import apf, build
    build.build_lib()
    return apf, apf.load_library()


def noalloc_S(apf, L, w, eps, S_out):
    rc = L.apf_solve_S_noalloc(w.nx, w.ny, w.npml, w.npml, w.lambda_px, None,
                               eps.ctypes.data if isinstance(eps, np.ndarray) else eps.data_ptr(),
                               w.j0, w.h, w.eps_sub, w.eps_clad, None, 0, None, 0,
                               S_out.ctypes.data if isinstance(S_out, np.ndarray) else S_out.data_ptr(), None)
    assert rc == 0, L.apf_last_error(None)
    return S_out


def test_noalloc_matches_solve_S_on_two_calls(lib):
    apf, L = lib
    w = W.TINY
    for seed in (0, 1):
        eps = np.ascontiguousarray(w.eps_slab(seed))
        s = apf.solver_for_workload(w, eps, precision="fp64")
        ref = s.solve_S()
        s.close()
        out = np.full(ref.shape, np.nan + 1j * np.nan)
        noalloc_S(apf, L, w, eps, out)
        err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
        assert err <= TOL_FP64, (seed, err)


def test_noalloc_device_buffers(lib):
    apf, L = lib
    import torch
    w = W.TINY
    eps = np.ascontiguousarray(w.eps_slab(2))
    s = apf.solver_for_workload(w, eps, precision="fp64")
    ref = s.solve_S()
    s.close()
    eps_d = torch.tensor(eps, device="cuda")
    S_d = torch.empty(ref.shape, dtype=torch.complex128, device="cuda")
    noalloc_S(apf, L, w, eps_d, S_d)
    assert np.linalg.norm(S_d.cpu().numpy() - ref) / np.linalg.norm(ref) <= TOL_FP64


def test_noalloc_rejects_sizes_beyond_the_limit(lib):
    apf, L = lib
    w = W.MID  # nx = 1024 > 64
    eps = np.ascontiguousarray(np.ones((w.h, w.nx)))
    out = np.empty((103, 103), np.complex128)
    rc = L.apf_solve_S_noalloc(w.nx, w.ny, w.npml, w.npml, w.lambda_px, None, eps.ctypes.data, w.j0, w.h,
                               w.eps_sub, w.eps_clad, None, 0, None, 0, out.ctypes.data, None)
    assert rc == apf.APF_EINVAL
    assert b"nx" in L.apf_last_error(None)
