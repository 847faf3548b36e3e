"""Kernel micro-benchmarks (CUDA-event timings of single library kernels):

    python -m paper_2306_09257_gb300.kernelbench gemm M N K [nsplit]   # complex M x K @ K x N on tcgen05
    python -m paper_2306_09257_gb300.kernelbench inv N [leaf]          # mixed inversion of a slab-like block
    python -m paper_2306_09257_gb300.kernelbench step large [K] [B]    # K steps of S + grad for B designs

They drive the library's test hooks (apf_debug_cgemm, apf_debug_inv32) on
seeded random inputs; used for the ncu captures summarised under profiles/.
"""
from __future__ import annotations

import ctypes
import sys

import numpy as np
import torch

from . import apf


def _hooks():
    L = apf.load_library()
    f = ctypes.c_void_p
    L.apf_debug_cgemm.argtypes = [f, ctypes.c_int, ctypes.c_int, ctypes.c_int] + [f] * 6 + [ctypes.c_int]
    L.apf_debug_inv32.argtypes = [f, ctypes.c_int, f, f, ctypes.c_int]
    return L


def gemm(m, n, k, nsplit=2, reps=3):
    L = _hooks()
    s = apf.Solver(0, "mixed")
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn(m, k, dtype=torch.complex64, device="cuda", generator=g)
    B = torch.randn(k, n, dtype=torch.complex64, device="cuda", generator=g)
    Ar, Ai, Br, Bi = A.real.contiguous(), A.imag.contiguous(), B.real.contiguous(), B.imag.contiguous()
    Cr = torch.empty(m, n, device="cuda")
    Ci = torch.empty(m, n, device="cuda")
    ts, tg = [], []
    for _ in range(reps):
        s.set_profiling(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rc = L.apf_debug_cgemm(s._h, m, n, k, Ar.data_ptr(), Ai.data_ptr(), Br.data_ptr(), Bi.data_ptr(),
                               Cr.data_ptr(), Ci.data_ptr(), nsplit)
        e1.record()
        torch.cuda.synchronize()
        if rc:
            raise apf.APFError(rc, L.apf_last_error(s._h).decode())
        ts.append(e0.elapsed_time(e1))
        tg.append(s.profile()["gemm_ms"])
    s.set_profiling(False)
    planes = {1: 1, 2: 3, 3: 6}[nsplit]
    g_ms = min(tg)
    print(f"gemm {m}x{n}x{k} nsplit {nsplit}: {min(ts):.3f} ms incl. operand packing "
          f"({8.0 * m * n * k / (min(ts) * 1e-3) / 1e12:.1f} complex TFLOP/s); GEMM launch alone {1000 * g_ms:.1f} us "
          f"({8.0 * m * n * k * planes / (g_ms * 1e-3) / 1e12:.1f} bf16 TFLOP/s on the tensor pipe)")


def inv(n, leaf=128, reps=3):
    L = _hooks()
    s = apf.Solver(0, "mixed")
    s.set_grid(n, 16, 4, 4, 8.0)
    s.set_eps(np.full((1, n), 1.5), 2.25, 1.0)
    s.set_channels([0], [0])
    g = torch.Generator(device="cuda").manual_seed(n)
    P = torch.randn(n, n, dtype=torch.complex64, device="cuda", generator=g) * (0.3 / n ** 0.5)
    X = P + P.T
    idx = torch.arange(n, device="cuda")
    X[idx, idx] += 3.6 + 0.2j
    X[idx, (idx + 1) % n] -= 1
    X[idx, (idx - 1) % n] -= 1
    ts = []
    for _ in range(reps):
        re, im = X.real.contiguous(), X.imag.contiguous()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rc = L.apf_debug_inv32(s._h, n, re.data_ptr(), im.data_ptr(), leaf)
        e1.record()
        torch.cuda.synchronize()
        if rc:
            raise apf.APFError(rc, L.apf_last_error(s._h).decode())
        ts.append(e0.elapsed_time(e1))
    Xi = torch.complex(re, im)
    res = (torch.linalg.norm(Xi @ X - torch.eye(n, device="cuda", dtype=X.dtype)) / n ** 0.5).item()
    print(f"inv {n} leaf {leaf}: {min(ts):.3f} ms, rms residual {res:.2e}")


def step(workload="large", k=1, nb=1):
    """One warm-up and k timed S + grad f evaluations of nb designs of a
    workload (mixed, refinement to 1e-7 as in bench.py; nb > 1 in one
    apf_solve_S_grad_batch call per step): the smallest command that runs the
    whole hot path, for launch lists under a profiler."""
    from . import workloads as W
    w = {"tiny": W.TINY, "mid": W.MID, "large": W.LARGE, "xlarge": W.XLARGE}[workload]
    sv = [apf.solver_for_workload(w, w.eps_slab(b), precision="mixed") for b in range(nb)]
    for s in sv:
        s.set_refinement(1e-7, 40)
    orders = [-2, -1, 0, 1, 2]

    def run():
        if nb == 1:
            sv[0].solve_S_grad("splitter", orders, 0.18)
        else:
            apf.solve_S_grad_batch(sv, "splitter", orders, 0.18)

    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(k):
        for b, s in enumerate(sv):
            s.set_eps(w.eps_slab(nb * (i + 1) + b), w.eps_sub, w.eps_clad, j0=w.j0)
        run()
    e1.record()
    torch.cuda.synchronize()
    st = [s.stats() for s in sv]
    print(f"step {w.name} x {nb}: {e0.elapsed_time(e1) / k:.1f} ms per step "
          f"({1000.0 * k * nb / e0.elapsed_time(e1):.2f} evaluations/s), "
          f"{st[0]['kernel_launches']} launches, refinement sweeps {[x['refine_iters'] for x in st]}")


if __name__ == "__main__":
    a = sys.argv[1:]
    if a and a[0] == "gemm":
        gemm(*[int(x) for x in a[1:4]], *([int(a[4])] if len(a) > 4 else []))
    elif a and a[0] == "inv":
        inv(*[int(x) for x in a[1:]])
    elif a and a[0] == "step":
        step(a[1] if len(a) > 1 else "large", *[int(x) for x in a[2:4]])
    else:
        print(__doc__)
