"""Spectral-convolution surrogate for line-search screening (Python side).

The network and its training run in libapf (include/apf_surrogate.h); this
module marshals tensors, initialises parameters from a seed, produces the
training pairs with the exact solver, and runs the screened optimiser.

Training pairs: slab permittivity -> efficiencies T_d of the relative
diffraction orders d = -2..2, averaged over the inputs,
    T_d = mean over inputs a with an output order m_a + d of |S_{a+d,a}|^2,
computed from the exact S of the solver (mixed precision, refined).
"""
from __future__ import annotations

import ctypes
import time
from typing import Sequence

import numpy as np
import torch

from . import apf as _apf
from . import workloads as W

ORDERS = (-2, -1, 0, 1, 2)


def _lib():
    L = _apf.load_library()
    if not getattr(L, "_sno_ready", False):
        vp, i, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        L.apf_sno_create.argtypes = [ctypes.POINTER(vp), i, i, i, i, i, i, i, i]
        L.apf_sno_destroy.argtypes = [vp]
        L.apf_sno_destroy.restype = None
        L.apf_sno_num_params.argtypes = [vp]
        L.apf_sno_num_params.restype = ctypes.c_longlong
        L.apf_sno_set_params.argtypes = [vp, vp]
        L.apf_sno_get_params.argtypes = [vp, vp]
        L.apf_sno_forward.argtypes = [vp, vp, i, vp, vp]
        L.apf_sno_gradients.argtypes = [vp, vp, vp, i, vp, ctypes.POINTER(f), vp]
        L.apf_sno_train_step.argtypes = [vp, vp, vp, i, f, ctypes.POINTER(f), vp]
        L._sno_ready = True
    return L


def param_layout(n_in_ch, width, modes, layers, n_out):
    """(name, shape) list in the order of the flat parameter vector."""
    return [("W0", (width, n_in_ch)), ("b0", (width,)), ("Wr", (layers, width, width, modes)),
            ("Wi", (layers, width, width, modes)), ("P", (layers, width, width)), ("c", (layers, width)),
            ("Wh", (n_out, width)), ("bh", (n_out,))]


def init_params(seed, n_in_ch, width, modes, layers, n_out) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in param_layout(n_in_ch, width, modes, layers, n_out):
        if name in ("b0", "c", "bh"):
            v = np.zeros(shape)
        elif name in ("Wr", "Wi"):
            v = rng.uniform(-1.0, 1.0, size=shape) / width
        else:
            v = rng.normal(size=shape) / np.sqrt(shape[-1])
        parts.append(v.ravel())
    return np.concatenate(parts).astype(np.float32)


class Surrogate:
    def __init__(self, n=1024, in_ch=12, width=48, modes=64, layers=4, n_out=5, max_batch=256, device=0, seed=0):
        self._L = _lib()
        self._h = ctypes.c_void_p()
        rc = self._L.apf_sno_create(ctypes.byref(self._h), device, n, in_ch, width, modes, layers, n_out, max_batch)
        if rc != 0:
            raise _apf.APFError(rc, self._L.apf_last_error(None).decode())
        self.shape = dict(n=n, in_ch=in_ch, width=width, modes=modes, layers=layers, n_out=n_out)
        self.max_batch = max_batch
        self.device = torch.device("cuda", device)
        self.nparams = int(self._L.apf_sno_num_params(self._h))
        self.set_params(init_params(seed, in_ch, width, modes, layers, n_out))

    def close(self):
        if self._h and self._h.value:
            self._L.apf_sno_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc):
        if rc != 0:
            raise _apf.APFError(rc, self._L.apf_last_error(None).decode())

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparams
        self._chk(self._L.apf_sno_set_params(self._h, p.ctypes.data))

    def params(self) -> np.ndarray:
        out = np.empty(self.nparams, np.float32)
        self._chk(self._L.apf_sno_get_params(self._h, out.ctypes.data))
        return out

    def _x(self, x):
        x = torch.as_tensor(x, dtype=torch.float32, device=self.device).contiguous()
        assert x.shape[1:] == (self.shape["in_ch"], self.shape["n"]), x.shape
        return x

    def forward(self, x) -> torch.Tensor:
        x = self._x(x)
        outs = []
        for b0 in range(0, x.shape[0], self.max_batch):
            xb = x[b0:b0 + self.max_batch]
            y = torch.empty((xb.shape[0], self.shape["n_out"]), dtype=torch.float32, device=self.device)
            st = ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
            self._chk(self._L.apf_sno_forward(self._h, xb.data_ptr(), xb.shape[0], y.data_ptr(), st))
            outs.append(y)
        return torch.cat(outs)

    def gradients(self, x, target):
        x = self._x(x)
        t = torch.as_tensor(target, dtype=torch.float32, device=self.device).contiguous()
        g = torch.empty(self.nparams, dtype=torch.float32, device=self.device)
        loss = ctypes.c_float()
        st = ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        self._chk(self._L.apf_sno_gradients(self._h, x.data_ptr(), t.data_ptr(), x.shape[0], g.data_ptr(),
                                            ctypes.byref(loss), st))
        return g.cpu().numpy(), loss.value

    def train_step(self, x, target, lr) -> float:
        x = self._x(x)
        t = torch.as_tensor(target, dtype=torch.float32, device=self.device).contiguous()
        loss = ctypes.c_float()
        st = ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)
        self._chk(self._L.apf_sno_train_step(self._h, x.data_ptr(), t.data_ptr(), x.shape[0], float(lr),
                                             ctypes.byref(loss), st))
        return loss.value


# ---------------------------------------------------------------------------
# training data from the exact solver
# ---------------------------------------------------------------------------
def pair_index(m_in, m_out, orders=ORDERS):
    """For each order d: (b indices, a indices) of the pairs m_out[b] - m_in[a] = d."""
    pos = {int(m): i for i, m in enumerate(m_out)}
    idx = []
    for d in orders:
        bs, as_ = [], []
        for a, m in enumerate(m_in):
            b = pos.get(int(m) + int(d))
            if b is not None:
                bs.append(b)
                as_.append(a)
        idx.append((torch.tensor(bs), torch.tensor(as_)))
    return idx


def efficiencies(S: torch.Tensor, idx) -> torch.Tensor:
    p = S.real ** 2 + S.imag ** 2
    return torch.stack([p[b.to(S.device), a.to(S.device)].mean() for b, a in idx])


def design(w, seed: int) -> np.ndarray:
    """Training design: the seeded filtered-threshold generator; odd seeds blend
    two generator designs with a random weight, to cover grey values."""
    e = w.eps_slab(seed)
    if seed % 2:
        rng = np.random.default_rng(seed + 7919)
        a = rng.uniform(0.2, 0.8)
        e = (1 - a) * e + a * w.eps_slab(seed + 104729)
    return e


def generate(w, seeds: Sequence[int], batch: int = 16, device: int = 0):
    """Exact efficiencies for the designs of `seeds`, `batch` designs per
    apf_solve_S_grad_batch call (every launch shared by the batch; the
    gradient it also returns is not used).  Returns (eps float32 (N, h, nx)
    on the device, targets float32 (N, 5) on the device, seconds)."""
    seeds = list(seeds)
    dev = torch.device("cuda", device)
    X = torch.empty((len(seeds), w.h, w.nx), dtype=torch.float32, device=dev)
    T = torch.empty((len(seeds), len(ORDERS)), dtype=torch.float32, device=dev)
    t0 = time.perf_counter()
    nb = max(1, min(batch, len(seeds), 16))
    sv = [_apf.solver_for_workload(w, design(w, seeds[0]), precision="mixed", device=device) for _ in range(nb)]
    mi, mo = sv[0].channels()
    idx = pair_index(mi, mo)
    S = [torch.empty((len(mo), len(mi)), dtype=torch.complex128, device=dev) for _ in range(nb)]
    G = [torch.empty((w.h, w.nx), dtype=torch.float64, device=dev) for _ in range(nb)]
    for j0 in range(0, len(seeds), nb):
        chunk = seeds[j0:j0 + nb]
        for b, sd in enumerate(chunk):
            e = design(w, sd)
            sv[b].set_eps(e, w.eps_sub, w.eps_clad, j0=w.j0)
            X[j0 + b] = torch.as_tensor(e, dtype=torch.float32, device=dev)
        k = len(chunk)
        _apf.solve_S_grad_batch(sv[:k], "power", ORDERS, 0.0, out_S=S[:k], out_grad=G[:k])
        for b in range(k):
            T[j0 + b] = efficiencies(S[b], idx).float()
    torch.cuda.synchronize()
    for s in sv:
        s.close()
    return X, T, time.perf_counter() - t0


def train(sno: Surrogate, X, T, epochs=20, batch=128, lr=2e-3, seed=0, log=None):
    n = X.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    steps = 0
    t0 = time.perf_counter()
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g).to(X.device)
        lr_ep = lr * 0.5 * (1 + np.cos(np.pi * ep / epochs))
        tot = 0.0
        for i in range(0, n - batch + 1, batch):
            sel = perm[i:i + batch]
            tot += sno.train_step(X[sel], T[sel], lr_ep)
            steps += 1
        losses.append(tot / max(1, n // batch))
        if log:
            log(f"epoch {ep} loss {losses[-1]:.3e}")
    return dict(steps=steps, seconds=time.perf_counter() - t0, losses=losses)


def proxy_objective(Tbar: torch.Tensor, counts: torch.Tensor, target: float) -> torch.Tensor:
    """Beam-splitter objective (Eq. 5) with every pair of order d replaced by
    the order's mean efficiency: sum_d n_d (T_d - t)^2."""
    return ((Tbar - target) ** 2 * counts).sum(-1)


def main(argv=None):
    """Surrogate study on the 1024 x 240 grid: exact training pairs from the
    mixed solver, training in libapf, held-out error against the exact
    efficiencies, and the screened line search against plain backtracking.
    Prints one JSON line."""
    import argparse
    import json

    from . import optim

    ap = argparse.ArgumentParser()
    ap.add_argument("--designs", type=int, default=20000)
    ap.add_argument("--holdout", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=128)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--batch-designs", type=int, default=16)
    ap.add_argument("--opt-iters", type=int, default=10)
    ap.add_argument("--starts", type=int, default=3)
    a = ap.parse_args(argv)
    w = W.MID
    X, T, t_gen = generate(w, range(1_000_000, 1_000_000 + a.designs), batch=a.batch_designs)
    n_tr = a.designs - a.holdout
    sno = Surrogate(n=w.nx, in_ch=w.h, width=48, modes=64, layers=4, n_out=5, max_batch=256, seed=0)
    tr = train(sno, X[:n_tr], T[:n_tr], epochs=a.epochs, batch=a.batch, lr=a.lr)
    pred = sno.forward(X[n_tr:])
    err = (pred - T[n_tr:])
    mse = float((err ** 2).mean())
    base = float(((T[:n_tr].mean(0, keepdim=True) - T[n_tr:]) ** 2).mean())
    rel = float(torch.linalg.norm(err) / torch.linalg.norm(T[n_tr:]))
    # inference rate on 64 candidates
    cand = X[n_tr:n_tr + 64]
    sno.forward(cand)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(20):
        sno.forward(cand)
    torch.cuda.synchronize()
    t_inf = (time.perf_counter() - t0) / 20
    runs = []
    for k in range(a.starts):
        eps0 = np.clip(w.eps_slab(2_000_000 + k), 1.0, 2.25)
        s = _apf.solver_for_workload(w, eps0, precision="mixed")
        _, hp = optim.optimize(s, eps0, w.eps_sub, w.eps_clad, w.j0, "splitter", list(ORDERS), 0.18,
                               iters=a.opt_iters)
        _, hs = optim.optimize_screened(s, sno, eps0, w.eps_sub, w.eps_clad, w.j0, list(ORDERS), 0.18,
                                        iters=a.opt_iters)
        s.close()
        runs.append({"plain": {"f": hp.f, "exact_solves": hp.evals, "seconds": hp.seconds,
                               "iters_per_s": hp.iters_per_second},
                     "screened": {"f": hs.f, "exact_solves": hs.evals, "seconds": hs.seconds,
                                  "iters_per_s": hs.iters_per_second, "screen_seconds": hs.screen_seconds}})
    out = {"workload": w.name, "designs": a.designs, "holdout": a.holdout,
           "data_seconds": t_gen, "data_rate_designs_per_s": a.designs / t_gen,
           "train": {"steps": tr["steps"], "seconds": tr["seconds"], "final_loss": tr["losses"][-1]},
           "heldout_mse": mse, "mean_predictor_mse": base, "heldout_rel_error": rel,
           "inference_ms_64_candidates": 1e3 * t_inf, "optimisation": runs}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
