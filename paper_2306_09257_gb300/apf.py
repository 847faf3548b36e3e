"""Python binding of libapf (ctypes): argument marshalling only.

Every numerical step runs inside ``_lib/libapf.so``.  There is no CPU
fallback: if the library is missing or fails to load, construction raises.
Arrays may be NumPy arrays (host) or torch tensors (host or CUDA); results
are written where the caller's buffers live.
"""
from __future__ import annotations

import ctypes
import os
import sys
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libapf.so")

APF_OK, APF_EINVAL, APF_ENOMEM, APF_ESINGULAR = 0, -1, -2, -3
APF_ENOCONV, APF_ETIMEOUT, APF_ECUDA, APF_ESTATE = -4, -5, -6, -7
APF_FP64, APF_MIXED_TF32, APF_MIXED_BF16X3 = 0, 1, 2  # TF32 is reserved (not built)
APF_OBJ_POWER, APF_OBJ_SPLITTER = 1, 2

PRECISIONS = {"fp64": APF_FP64, "mixed": APF_MIXED_BF16X3, "bf16x3": APF_MIXED_BF16X3}
OBJECTIVES = {"power": APF_OBJ_POWER, "splitter": APF_OBJ_SPLITTER}

# Every symbol that include/*.h declares.
EXPORTS = ("apf_create", "apf_destroy", "apf_set_grid", "apf_set_eps", "apf_set_channels",
           "apf_get_channels", "apf_solve_S", "apf_solve_S_grad", "apf_grad_from_gamma",
           "apf_set_refinement", "apf_get_stats", "apf_set_profiling", "apf_get_profile",
           "apf_solve_S_noalloc", "apf_last_error", "apf_version", "apf_set_ridges", "apf_ridge_grad",
           "apf_substrate_orders", "apf_reflection", "apf_reverse_S", "apf_set_krylov",
           "apf_solve_S_grad_adjoint", "apf_set_schur_storage", "apf_solve_S_grad_batch",
           "apf_set_elimination",
           "apf_sno_create", "apf_sno_destroy", "apf_sno_num_params", "apf_sno_set_params",
           "apf_sno_get_params", "apf_sno_forward", "apf_sno_gradients", "apf_sno_train_step")


class APFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"apf error {code}: {msg}")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("refine_iters", ctypes.c_int), ("residual", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_boundary", ctypes.c_double),
                ("ms_eliminate", ctypes.c_double), ("ms_fields", ctypes.c_double),
                ("ms_readout", ctypes.c_double), ("ms_gradient", ctypes.c_double),
                ("kernel_launches", ctypes.c_longlong), ("workspace_bytes", ctypes.c_longlong),
                ("leaf_fallbacks", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(ctypes.Structure):
    _fields_ = [("gemm_launches", ctypes.c_longlong), ("gemm_ms", ctypes.c_double),
                ("gemm_alg_flops", ctypes.c_double), ("gemm_hw_flops", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PML(ctypes.Structure):
    _fields_ = [("R0", ctypes.c_double), ("power", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libapf.so not found at {path}; build it with "
                           "`python -m paper_2306_09257_gb300.build`")
    L = ctypes.CDLL(path)
    vp, ip, dp, i, d = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.apf_create.argtypes = [ctypes.POINTER(vp), i, i]
    L.apf_destroy.argtypes = [vp]
    L.apf_destroy.restype = None
    L.apf_set_grid.argtypes = [vp, i, i, i, i, d, ctypes.POINTER(PML)]
    L.apf_set_eps.argtypes = [vp, dp, i, i, d, d, vp]
    L.apf_set_channels.argtypes = [vp, ip, i, ip, i]
    L.apf_get_channels.argtypes = [vp, ip, ip, ip, ip]
    L.apf_solve_S.argtypes = [vp, dp, vp]
    L.apf_solve_S_grad.argtypes = [vp, i, ctypes.POINTER(ctypes.c_double), i, dp, ctypes.POINTER(ctypes.c_double), dp, vp]
    L.apf_solve_S_grad_adjoint.argtypes = L.apf_solve_S_grad.argtypes
    L.apf_solve_S_grad_batch.argtypes = [ctypes.POINTER(vp), i, i, ctypes.POINTER(ctypes.c_double), i,
                                         ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(vp), vp]
    L.apf_grad_from_gamma.argtypes = [vp, dp, dp, vp]
    L.apf_set_refinement.argtypes = [vp, d, i]
    L.apf_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    L.apf_set_profiling.argtypes = [vp, i]
    L.apf_get_profile.argtypes = [vp, ctypes.POINTER(Profile)]
    L.apf_solve_S_noalloc.argtypes = [i, i, i, i, d, ctypes.POINTER(PML), dp, i, i, d, d, ip, i, ip, i, dp, vp]
    L.apf_substrate_orders.argtypes = [vp, ip, ip]
    L.apf_set_krylov.argtypes = [vp, i]
    L.apf_set_schur_storage.argtypes = [vp, i]
    L.apf_set_elimination.argtypes = [vp, i, i]
    L.apf_reflection.argtypes = [vp, ip, i, dp, vp]
    L.apf_reverse_S.argtypes = [vp, dp, vp]
    L.apf_set_ridges.argtypes = [vp, dp, i, i, d, d, i, i, d, d, dp, vp]
    L.apf_ridge_grad.argtypes = [vp, dp, dp, vp]
    L.apf_last_error.argtypes = [vp]
    L.apf_last_error.restype = ctypes.c_char_p
    L.apf_version.argtypes = []
    _lib = L
    return L


def _ptr(a, dtype) -> int:
    """Raw pointer of a contiguous NumPy array or torch tensor of `dtype`."""
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags.c_contiguous:
            raise TypeError(f"need a C-contiguous {dtype} array")
        return a.ctypes.data
    import torch
    tmap = {np.float64: torch.float64, np.complex128: torch.complex128}
    if not isinstance(a, torch.Tensor) or a.dtype != tmap[np.dtype(dtype).type] or not a.is_contiguous():
        raise TypeError(f"need a contiguous {dtype} array or tensor")
    return a.data_ptr()


def _stream_of(*arrays, device=None):
    """The stream a call is ordered on: torch's current stream of the device
    of the first CUDA tensor argument, else (when torch is in use and has
    initialised CUDA) torch's current stream of `device`, else the legacy
    default stream (None)."""
    for a in arrays:
        if a is not None and not isinstance(a, np.ndarray):
            import torch
            if isinstance(a, torch.Tensor) and a.is_cuda:
                return ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    torch = sys.modules.get("torch")
    if device is not None and torch is not None and torch.cuda.is_initialized():
        return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    return None


class Solver:
    """One APF context on one GPU."""

    def __init__(self, device: int = 0, precision: str = "fp64"):
        self._L = load_library()
        self._h = ctypes.c_void_p()
        rc = self._L.apf_create(ctypes.byref(self._h), int(device), PRECISIONS[precision])
        if rc != APF_OK:
            raise APFError(rc, self._L.apf_last_error(None).decode())
        self.precision = precision
        self.device = device
        self.nx = self.h = None
        self.n_edges = 0
        self.version = 0  # bumped by every call that changes the stored fields

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.apf_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int, allow=()):
        if rc != APF_OK and rc not in allow:
            raise APFError(rc, self._L.apf_last_error(self._h).decode())
        return rc

    def set_grid(self, nx, ny, npml_bot, npml_top, lambda_px, R0=1e-8, power=3.0):
        p = PML(R0, power)
        self._check(self._L.apf_set_grid(self._h, nx, ny, npml_bot, npml_top, float(lambda_px), ctypes.byref(p)))
        self.nx = nx

    def set_eps(self, eps_slab, eps_sub: float, eps_clad: float, j0: int = -1):
        h = int(eps_slab.shape[0])
        if isinstance(eps_slab, np.ndarray):
            eps_slab = np.ascontiguousarray(eps_slab, dtype=np.float64)
        # a CUDA tensor is read in order on torch's current stream (after the ops that wrote it)
        self._check(self._L.apf_set_eps(self._h, _ptr(eps_slab, np.float64), int(j0), h,
                                        float(eps_sub), float(eps_clad), _stream_of(eps_slab, device=self.device)))
        self.h = h
        self.version += 1

    def set_ridges(self, edges, h: int, eps_ridge: float, eps_bg: float, eps_sub: float, eps_clad: float,
                   mirror: bool = True, j0: int = -1, eps_out=None):
        """Slab permittivity from ridge edge positions (paper Sec. 3; see
        apf_set_ridges), set as by set_eps.  Returns the h x nx slab (a new
        host array when eps_out is None; nothing is copied out when eps_out
        is False)."""
        if isinstance(edges, np.ndarray) or not hasattr(edges, "data_ptr"):
            edges = np.ascontiguousarray(edges, dtype=np.float64)
        if eps_out is False:
            eps, eps_p = None, None
        else:
            eps = np.empty((int(h), self.nx), dtype=np.float64) if eps_out is None else eps_out
            eps_p = _ptr(eps, np.float64)
        self._check(self._L.apf_set_ridges(self._h, _ptr(edges, np.float64), int(edges.shape[0]),
                                           1 if mirror else 0, float(eps_ridge), float(eps_bg), int(j0), int(h),
                                           float(eps_sub), float(eps_clad), eps_p,
                                           _stream_of(edges, eps if eps_out is not None else None, device=self.device)))
        self.h = int(h)
        self.n_edges = int(edges.shape[0])
        self.version += 1
        return eps

    def ridge_grad(self, grad_eps, out=None):
        """df/d(edge positions) of the last set_ridges from a pixel gradient."""
        if isinstance(grad_eps, np.ndarray):
            grad_eps = np.ascontiguousarray(grad_eps, dtype=np.float64)
        g = np.empty(self.n_edges, dtype=np.float64) if out is None else out
        st = _stream_of(grad_eps, g, device=self.device)
        self._check(self._L.apf_ridge_grad(self._h, _ptr(grad_eps, np.float64), _ptr(g, np.float64), st))
        return g

    def set_channels(self, m_in: Optional[Sequence[int]] = None, m_out: Optional[Sequence[int]] = None):
        def arr(v):
            if v is None:
                return None, 0
            a = (ctypes.c_int * len(v))(*[int(x) for x in v])
            return a, len(v)
        ai, ni = arr(m_in)
        ao, no = arr(m_out)
        self._check(self._L.apf_set_channels(self._h, ai, ni, ao, no))

    def channels(self):
        ni, no = ctypes.c_int(), ctypes.c_int()
        self._check(self._L.apf_get_channels(self._h, ctypes.byref(ni), ctypes.byref(no), None, None))
        mi = (ctypes.c_int * ni.value)()
        mo = (ctypes.c_int * no.value)()
        self._check(self._L.apf_get_channels(self._h, None, None, mi, mo))
        return np.array(mi[:], dtype=np.int64), np.array(mo[:], dtype=np.int64)

    def substrate_orders(self) -> np.ndarray:
        """Orders propagating in the substrate (the reflection channels)."""
        n = ctypes.c_int()
        self._check(self._L.apf_substrate_orders(self._h, ctypes.byref(n), None))
        m = (ctypes.c_int * n.value)()
        self._check(self._L.apf_substrate_orders(self._h, None, m))
        return np.array(m[:], dtype=np.int64)

    def reflection(self, m_ref: Optional[Sequence[int]] = None, out=None):
        """Reflection block of the last solve (see apf_reflection): rows =
        substrate orders m_ref (default: all of substrate_orders()), columns =
        inputs."""
        mr = self.substrate_orders() if m_ref is None else np.asarray(m_ref)
        mi, _ = self.channels()
        R = np.empty((len(mr), len(mi)), dtype=np.complex128) if out is None else out
        arr = (ctypes.c_int * len(mr))(*[int(v) for v in mr])
        st = _stream_of(R, device=self.device)
        self._check(self._L.apf_reflection(self._h, arr, len(mr), _ptr(R, np.complex128), st))
        return R

    def reverse_S(self, out=None):
        """Transmission from the cladding side of the last solve (see
        apf_reverse_S): rows = substrate orders m_in, columns = cladding
        orders m_out."""
        mi, mo = self.channels()
        S = np.empty((len(mi), len(mo)), dtype=np.complex128) if out is None else out
        st = _stream_of(S, device=self.device)
        self._check(self._L.apf_reverse_S(self._h, _ptr(S, np.complex128), st))
        return S

    def set_refinement(self, tol: float, max_iters: int):
        self._check(self._L.apf_set_refinement(self._h, float(tol), int(max_iters)))

    def set_schur_storage(self, segment_rows: int):
        """Mixed mode: 0 stores every slab inverse; k > 0 keeps one segment of
        k rows and recomputes the others from float32 checkpoints (see
        apf_set_schur_storage)."""
        self._check(self._L.apf_set_schur_storage(self._h, int(segment_rows)))
        self.version += 1

    def set_elimination(self, planes: int = 2, butterfly: bool = True):
        """Mixed mode: bf16 split planes of the elimination (2: bf16x3, 3:
        bf16x6) and the symmetric random butterfly transform of the slab
        blocks (see apf_set_elimination)."""
        self._check(self._L.apf_set_elimination(self._h, int(planes), 1 if butterfly else 0))
        self.version += 1

    def set_krylov(self, m: int):
        """Mixed mode: GMRES(m) refinement (0: plain refinement); see apf_set_krylov."""
        self._check(self._L.apf_set_krylov(self._h, int(m)))
        self.version += 1

    def _alloc_S(self):
        mi, mo = self.channels()
        return np.empty((len(mo), len(mi)), dtype=np.complex128)

    def solve_S(self, out=None, allow_noconv=False):
        S = self._alloc_S() if out is None else out
        st = _stream_of(S, device=self.device)
        self.version += 1
        self._check(self._L.apf_solve_S(self._h, _ptr(S, np.complex128), st),
                    allow=(APF_ENOCONV,) if allow_noconv else ())
        return S

    @staticmethod
    def objective_params(kind: str, orders: Sequence[int], target: float = 0.0):
        vals = [float(target), float(len(orders))] + [float(o) for o in orders]
        return OBJECTIVES[kind], (ctypes.c_double * len(vals))(*vals), len(vals)

    def solve_S_grad(self, kind: str, orders: Sequence[int], target: float = 0.0,
                     out_S=None, out_grad=None, allow_noconv=False):
        S = self._alloc_S() if out_S is None else out_S
        g = np.empty((self.h, self.nx), dtype=np.float64) if out_grad is None else out_grad
        oid, params, npar = self.objective_params(kind, orders, target)
        f = ctypes.c_double()
        st = _stream_of(S, g, device=self.device)
        self.version += 1
        self._check(self._L.apf_solve_S_grad(self._h, oid, params, npar, _ptr(S, np.complex128),
                                             ctypes.byref(f), _ptr(g, np.float64), st),
                    allow=(APF_ENOCONV,) if allow_noconv else ())
        return S, f.value, g

    def solve_S_grad_adjoint(self, kind: str, orders: Sequence[int], target: float = 0.0,
                             out_S=None, out_grad=None, allow_noconv=False):
        """S, f and df/deps by the conventional adjoint method (Eq. S1: a
        forward sweep, then an adjoint sweep with sources built from Gamma);
        the paper's baseline for APF, on the same elimination."""
        S = self._alloc_S() if out_S is None else out_S
        g = np.empty((self.h, self.nx), dtype=np.float64) if out_grad is None else out_grad
        oid, params, npar = self.objective_params(kind, orders, target)
        f = ctypes.c_double()
        st = _stream_of(S, g, device=self.device)
        self.version += 1
        self._check(self._L.apf_solve_S_grad_adjoint(self._h, oid, params, npar, _ptr(S, np.complex128),
                                                     ctypes.byref(f), _ptr(g, np.float64), st),
                    allow=(APF_ENOCONV,) if allow_noconv else ())
        return S, f.value, g

    def grad_from_gamma(self, Gamma, out=None):
        g = np.empty((self.h, self.nx), dtype=np.float64) if out is None else out
        if isinstance(Gamma, np.ndarray):
            Gamma = np.ascontiguousarray(Gamma, dtype=np.complex128)
        st = _stream_of(Gamma, g, device=self.device)
        self._check(self._L.apf_grad_from_gamma(self._h, _ptr(Gamma, np.complex128), _ptr(g, np.float64), st))
        return g

    def set_profiling(self, enable: bool = True):
        self._check(self._L.apf_set_profiling(self._h, 1 if enable else 0))

    def profile(self) -> dict:
        p = Profile()
        self._check(self._L.apf_get_profile(self._h, ctypes.byref(p)))
        return p.as_dict()

    def stats(self) -> dict:
        s = Stats()
        self._check(self._L.apf_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()


def solve_S_grad_batch(solvers: Sequence["Solver"], kind: str, orders: Sequence[int], target: float = 0.0,
                       out_S=None, out_grad=None, allow_noconv=False):
    """S, f and df/deps of several designs in one call (apf_solve_S_grad_batch):
    `solvers` share grid, slab rows, channels and settings, each holding its
    own permittivity.  Returns lists (S, f, grad) in solver order."""
    nb = len(solvers)
    L = solvers[0]._L
    S = [sv._alloc_S() for sv in solvers] if out_S is None else list(out_S)
    g = [np.empty((sv.h, sv.nx), dtype=np.float64) for sv in solvers] if out_grad is None else list(out_grad)
    oid, params, npar = Solver.objective_params(kind, orders, target)
    hs = (ctypes.c_void_p * nb)(*[sv._h.value for sv in solvers])
    sp = (ctypes.c_void_p * nb)(*[_ptr(x, np.complex128) for x in S])
    gp = (ctypes.c_void_p * nb)(*[_ptr(x, np.float64) for x in g])
    f = (ctypes.c_double * nb)()
    st = _stream_of(*S, *g, device=solvers[0].device)
    for sv in solvers:
        sv.version += 1
    rc = L.apf_solve_S_grad_batch(hs, nb, oid, params, npar, sp, f, gp, st)
    if rc != APF_OK and not (allow_noconv and rc == APF_ENOCONV):
        msgs = [L.apf_last_error(sv._h).decode() for sv in solvers]
        raise APFError(rc, "; ".join(m for m in msgs if m and m != "no error") or L.apf_last_error(None).decode())
    return S, list(f), g


def solver_for_workload(w, eps_slab, precision="fp64", device=0, m_in=None, m_out=None) -> Solver:
    s = Solver(device=device, precision=precision)
    s.set_grid(w.nx, w.ny, w.npml, w.npml, w.lambda_px)
    s.set_eps(eps_slab, w.eps_sub, w.eps_clad, j0=w.j0)
    s.set_channels(m_in, m_out)
    return s
