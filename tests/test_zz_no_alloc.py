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


def test_noalloc_at_its_size_limit_on_a_side_stream(lib):
    """The tightest fit of the scratch array: nx = 64, h = 16 and 63 + 63
    explicit channel orders (the most that nx = 64 admits: order -32 never
    propagates when order 0 does), with device buffers on a non-default
    stream, twice in a row, against the context-based solve."""
    apf, L = lib
    import torch
    nx, ny, npml, h = 64, 80, 20, 16
    lam = 2.0 * np.pi / (2.0 * np.sqrt(0.9999))  # k^2/4 just below 1: orders -31..31 propagate
    orders = list(range(-31, 32))
    side = torch.cuda.Stream()
    for seed in (5, 6):
        eps = np.ascontiguousarray(W.iid_eps(h, nx, seed, 1.0, 2.0))
        s = apf.Solver(0, "fp64")
        s.set_grid(nx, ny, npml, npml, lam)
        s.set_eps(eps, 1.0, 1.0)
        s.set_channels(orders, orders)
        ref = s.solve_S()
        s.close()
        oi = (ctypes.c_int * len(orders))(*orders)
        with torch.cuda.stream(side):
            eps_d = torch.tensor(eps, device="cuda")
            S_d = torch.full((len(orders), len(orders)), complex("nan+nanj"), dtype=torch.complex128, device="cuda")
            rc = L.apf_solve_S_noalloc(nx, ny, npml, npml, lam, None, eps_d.data_ptr(), -1, h, 1.0, 1.0,
                                       oi, len(orders), oi, len(orders), S_d.data_ptr(),
                                       ctypes.c_void_p(side.cuda_stream))
        assert rc == 0, L.apf_last_error(None)
        got = S_d.cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL_FP64, seed


@pytest.mark.parametrize("what", ["h", "channels"])
def test_noalloc_rejects_just_over_the_limit(lib, what):
    apf, L = lib
    nx, ny, npml = 64, 100, 20
    h = 17 if what == "h" else 16
    eps = np.ascontiguousarray(np.full((h, nx), 1.5))
    n = 65 if what == "channels" else 4
    orders = (ctypes.c_int * n)(*range(n))
    out = np.empty((n, n), np.complex128)
    rc = L.apf_solve_S_noalloc(nx, ny, npml, npml, 16.0, None, eps.ctypes.data, -1, h, 2.25, 1.0,
                               orders, n, orders, n, out.ctypes.data, None)
    assert rc == apf.APF_EINVAL
    assert (b"h must be" if what == "h" else b"channels") in L.apf_last_error(None)


def test_noalloc_threads_take_turns(lib):
    """Four host threads call the allocation-free solve at once, each with its
    own design and stream: calls on one device take turns, so none sees
    another's data in the shared scratch array (each S equals its own
    context-based solve)."""
    import threading

    import torch
    apf, L = lib
    w = W.TINY
    seeds = [3, 4, 5, 6]
    eps = [np.ascontiguousarray(w.eps_slab(sd)) for sd in seeds]
    refs = []
    for e in eps:
        s = apf.solver_for_workload(w, e, precision="fp64")
        refs.append(s.solve_S())
        s.close()
    outs = [np.full(r.shape, np.nan + 1j * np.nan) for r in refs]
    errs = []

    def worker(b):
        try:
            st = torch.cuda.Stream()
            for _ in range(3):
                rc = L.apf_solve_S_noalloc(w.nx, w.ny, w.npml, w.npml, w.lambda_px, None, eps[b].ctypes.data,
                                           w.j0, w.h, w.eps_sub, w.eps_clad, None, 0, None, 0,
                                           outs[b].ctypes.data, ctypes.c_void_p(st.cuda_stream))
                assert rc == 0, L.apf_last_error(None)
        except BaseException as e:  # noqa: BLE001
            errs.append(e)
    ths = [threading.Thread(target=worker, args=(b,)) for b in range(len(seeds))]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert not errs, errs
    for b in range(len(seeds)):
        err = np.linalg.norm(outs[b] - refs[b]) / np.linalg.norm(refs[b])
        assert err <= TOL_FP64, (seeds[b], err)
