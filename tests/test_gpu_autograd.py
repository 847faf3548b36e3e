"""autograd wrapper, finite differences and the line-search optimiser on the GPU."""
import numpy as np
import pytest

import oracle as O
from paper_2306_09257_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_09257_gb300 import apf, autograd, build
    build.build_lib()
    apf.load_library()
    return torch, apf, autograd


def small(nx=32, h=2, seed=0):
    return W.small_workload(nx, 70, 20, 9.0, h), W.iid_eps(h, nx, seed, 1.0, 3.0)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_autograd_backward_equals_builtin_gradient(env, prec, tol):
    torch, apf, AG = env
    w = W.TINY
    eps = w.eps_slab(5)
    s = apf.solver_for_workload(w, eps, precision=prec)
    mi, mo = s.channels()
    _, f_ref, g_ref = s.solve_S_grad("splitter", [-2, -1, 0, 1, 2], 0.18)
    x = torch.tensor(eps, device="cuda", requires_grad=True)
    S = AG.scattering(x, s, w.eps_sub, w.eps_clad, w.j0)
    mask = AG.relative_order_mask(mi, mo, [-2, -1, 0, 1, 2], device="cuda")
    loss = AG.splitter_loss(S, mask, 0.18)
    loss.backward()
    assert abs(loss.item() - f_ref) <= 1e-9 * abs(f_ref)
    g = x.grad.cpu().numpy()
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) <= tol


def test_gradcheck_tiny(env):
    torch, apf, AG = env
    w, eps = small()
    s = apf.solver_for_workload(w, eps, precision="fp64")
    mi, mo = s.channels()
    mask = AG.relative_order_mask(mi, mo, [-1, 0, 1], device="cuda")

    def f(x):
        return AG.splitter_loss(AG.scattering(x, s, w.eps_sub, w.eps_clad, w.j0), mask, 0.3)

    x = torch.tensor(eps, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(f, (x,), eps=1e-6, atol=1e-7, rtol=1e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_central_fd_on_16_pixels(env, prec):
    """Central differences (step 1e-6 in eps) on 16 seeded pixels of the
    1024 x 240 workload against the single-elimination gradient."""
    torch, apf, AG = env
    w = W.MID
    eps = w.eps_slab(3)
    s = apf.solver_for_workload(w, eps, precision=prec)
    if prec == "mixed":
        s.set_refinement(1e-13, 12)
    orders = [-2, -1, 0, 1, 2]
    _, f0, g = s.solve_S_grad("splitter", orders, 0.18)
    rng = np.random.default_rng(16)
    pix = [(int(rng.integers(w.h)), int(rng.integers(w.nx))) for _ in range(16)]
    h = 1e-6
    fd = []
    for (j, x) in pix:
        vals = []
        for sgn in (1, -1):
            e = eps.copy()
            e[j, x] += sgn * h
            s.set_eps(e, w.eps_sub, w.eps_clad, j0=w.j0)
            vals.append(s.solve_S_grad("splitter", orders, 0.18)[1])
        fd.append((vals[0] - vals[1]) / (2 * h))
    fd = np.array(fd)
    ga = np.array([g[j, x] for j, x in pix])
    err = np.linalg.norm(fd - ga) / np.linalg.norm(ga)
    assert err < 1e-5, err


def test_armijo_line_search_decreases_f(env):
    torch, apf, AG = env
    from paper_2306_09257_gb300 import optim
    w = W.TINY
    eps0 = np.clip(w.eps_slab(7), 1.0, 2.25)
    s = apf.solver_for_workload(w, eps0, precision="mixed")
    eps, hist = optim.optimize(s, eps0, w.eps_sub, w.eps_clad, w.j0, "splitter", [-1, 1], 0.25, iters=8)
    assert len(hist.f) >= 3
    assert all(b <= a for a, b in zip(hist.f, hist.f[1:]))
    assert hist.f[-1] < hist.f[0]
    assert eps.min() >= 1.0 and eps.max() <= 2.25
