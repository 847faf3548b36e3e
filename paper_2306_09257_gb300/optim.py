"""Gradient-descent optimisation of the slab permittivity with the
backtracking (Armijo) line search of the paper's supplement (Sec. 4, Eq. S2):
start from gamma_max, shrink by tau = 1/2 until
    f(x_new) <= f(x) - c1 * ||x_new - x||^2 / gamma,    c1 = 1e-2,
which is Eq. (S2) when no bound is active (x_new - x = -gamma grad f).  The
permittivity is kept in [eps_lo, eps_hi] by projection.  Every trial point is
one APF evaluation that returns f and grad f together, so the gradient of the
accepted point is reused by the next iteration.
"""
from __future__ import annotations

import dataclasses
import time
from typing import List, Sequence

import numpy as np


@dataclasses.dataclass
class History:
    f: List[float]
    evals: int
    seconds: float
    gammas: List[float]

    @property
    def iters_per_second(self) -> float:
        return (len(self.f) - 1) / self.seconds if self.seconds > 0 else 0.0


def optimize(solver, eps0: np.ndarray, eps_sub: float, eps_clad: float, j0: int, kind: str,
             orders: Sequence[int], target: float, iters: int, gamma_max: float = None,
             tau: float = 0.5, c1: float = 1e-2, eps_lo: float = 1.0, eps_hi: float = 2.25,
             max_backtracks: int = 12):
    eps = np.clip(np.asarray(eps0, np.float64).copy(), eps_lo, eps_hi)
    t0 = time.perf_counter()
    solver.set_eps(eps, eps_sub, eps_clad, j0=j0)
    _, f, g = solver.solve_S_grad(kind, orders, target)
    evals = 1
    hist = History([f], 0, 0.0, [])
    if gamma_max is None:
        gamma_max = 0.25 / max(float(np.abs(g).max()), 1e-30)
    for _ in range(iters):
        gamma = gamma_max
        accepted = False
        for _ in range(max_backtracks):
            trial = np.clip(eps - gamma * g, eps_lo, eps_hi)
            solver.set_eps(trial, eps_sub, eps_clad, j0=j0)
            _, ft, gt = solver.solve_S_grad(kind, orders, target)
            evals += 1
            if ft <= f - c1 * float(np.sum((trial - eps) ** 2)) / gamma:
                eps, f, g = trial, ft, gt
                accepted = True
                break
            gamma *= tau
        hist.gammas.append(gamma if accepted else 0.0)
        hist.f.append(f)
        if not accepted:
            break
    hist.evals = evals
    hist.seconds = time.perf_counter() - t0
    return eps, hist


def optimize_screened(solver, sno, eps0: np.ndarray, eps_sub: float, eps_clad: float, j0: int,
                      orders: Sequence[int], target: float, iters: int, gamma_max: float = None,
                      n_candidates: int = 64, span: float = 2.0 ** 6, tau: float = 0.5, c1: float = 1e-2,
                      eps_lo: float = 1.0, eps_hi: float = 2.25, max_backtracks: int = 12):
    """Line search screened by the surrogate: every iteration scores
    n_candidates step sizes, log-spaced from gamma_max / span to
    gamma_max * span, with the surrogate's efficiencies plugged into the
    beam-splitter objective; the exact solve judges the best one with the
    same Armijo test as `optimize`, and if it fails backtracking by tau
    continues from there.  The exact solve is therefore still the arbiter of
    every accepted step; the surrogate lets the search try steps longer than
    gamma_max without paying exact solves for the ones it rejects."""
    import torch

    from . import surrogate as SG
    eps = np.clip(np.asarray(eps0, np.float64).copy(), eps_lo, eps_hi)
    t0 = time.perf_counter()
    solver.set_eps(eps, eps_sub, eps_clad, j0=j0)
    _, f, g = solver.solve_S_grad("splitter", orders, target)
    mi, mo = solver.channels()
    counts = torch.tensor([len(b) for b, _ in SG.pair_index(mi, mo, SG.ORDERS)], dtype=torch.float32,
                          device=sno.device)
    evals = 1
    hist = History([f], 0, 0.0, [])
    if gamma_max is None:
        gamma_max = 0.25 / max(float(np.abs(g).max()), 1e-30)
    gammas = gamma_max * span ** np.linspace(1.0, -1.0, n_candidates)
    screen_s = 0.0
    for _ in range(iters):
        ts = time.perf_counter()
        e_t = torch.as_tensor(eps, dtype=torch.float32, device=sno.device)
        g_t = torch.as_tensor(g, dtype=torch.float32, device=sno.device)
        gam = torch.as_tensor(gammas, dtype=torch.float32, device=sno.device)[:, None, None]
        cand = torch.clamp(e_t[None] - gam * g_t[None], eps_lo, eps_hi)
        pred = SG.proxy_objective(sno.forward(cand), counts, target)
        gamma = float(gammas[int(torch.argmin(pred))])
        screen_s += time.perf_counter() - ts
        accepted = False
        for _ in range(max_backtracks):
            trial = np.clip(eps - gamma * g, eps_lo, eps_hi)
            solver.set_eps(trial, eps_sub, eps_clad, j0=j0)
            _, ft, gt = solver.solve_S_grad("splitter", orders, target)
            evals += 1
            if ft <= f - c1 * float(np.sum((trial - eps) ** 2)) / gamma:
                eps, f, g = trial, ft, gt
                accepted = True
                break
            gamma *= tau
        hist.gammas.append(gamma if accepted else 0.0)
        hist.f.append(f)
        if not accepted:
            break
    hist.evals = evals
    hist.seconds = time.perf_counter() - t0
    hist.screen_seconds = screen_s
    return eps, hist
