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


ORDERS = [-2, -1, 0, 1, 2]


@pytest.mark.parametrize("prec,tol_s,tol_g", [("fp64", 1e-10, 1e-10), ("mixed", 1e-6, 1e-5)])
@pytest.mark.parametrize("seed", [0, 3, 9])
def test_autograd_matches_oracle(env, prec, tol_s, tol_g, seed):
    """S(eps) -> Eq. 5 loss in torch -> .backward() against the oracle's S, f
    and its conventional-adjoint gradient (Eq. S1) on the 64 x 100 grid: the
    whole autograd chain (forward solve, Gamma = conj(dL/dS)/2, the library's
    adjoint contraction) closed against the independent CPU reference."""
    torch, apf, AG = env
    w = W.TINY
    eps = w.eps_slab(seed)
    sol, f_ref, _, g_ref = O.f_and_grad(O.problem_from_workload(w, eps), "splitter", ORDERS, 0.18)
    s = apf.solver_for_workload(w, eps, precision=prec)
    mi, mo = s.channels()
    assert list(mi) == list(sol.pb.inputs()) and list(mo) == list(sol.pb.outputs())
    x = torch.tensor(eps, device="cuda", requires_grad=True)
    S = AG.scattering(x, s, w.eps_sub, w.eps_clad, w.j0)
    loss = AG.splitter_loss(S, AG.relative_order_mask(mi, mo, ORDERS, device="cuda"), 0.18)
    loss.backward()
    S_h = S.detach().cpu().numpy()
    g = x.grad.cpu().numpy()
    assert np.linalg.norm(S_h - sol.S) / np.linalg.norm(sol.S) <= tol_s
    assert np.max(np.abs(S_h - sol.S)) <= tol_s * np.max(np.abs(sol.S))
    assert abs(loss.item() - f_ref) <= max(tol_s, 1e-12) * 10 * abs(f_ref)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) <= tol_g
    assert np.max(np.abs(g - g_ref)) <= tol_g * np.max(np.abs(g_ref))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_ridge_autograd_matches_oracle(env, prec, tol):
    """The ridge wrapper (edges -> slab -> S -> Eq. 5 loss, backward to the
    edges) against the oracle: its pixel gradient pushed through the oracle's
    edge Jacobian (oracle.grad_edges) on the 64 x 100 grid."""
    torch, apf, AG = env
    w = W.TINY
    edges = W.ridge_edges(w.nx, W.ridge_count(w), 4, mirror=True)
    eps_r, eps_b = 13.69, 1.0
    eps = O.eps_from_edges(w.nx, w.h, edges, True, eps_r, eps_b)
    _, f_ref, _, g_pix = O.f_and_grad(O.problem_from_workload(w, eps), "splitter", ORDERS, 0.18)
    g_ref = O.grad_edges(g_pix, w.nx, edges, True, eps_r, eps_b)
    s = apf.Solver(0, prec)
    s.set_grid(w.nx, w.ny, w.npml, w.npml, w.lambda_px)
    s.set_ridges(edges, w.h, eps_r, eps_b, w.eps_sub, w.eps_clad, mirror=True, j0=w.j0)
    s.set_channels(None, None)
    mi, mo = s.channels()
    t = torch.tensor(edges, device="cuda", requires_grad=True)
    S = AG.ridge_scattering(t, s, w.h, eps_r, eps_b, w.eps_sub, w.eps_clad, mirror=True, j0=w.j0)
    loss = AG.splitter_loss(S, AG.relative_order_mask(mi, mo, ORDERS, device="cuda"), 0.18)
    loss.backward()
    g = t.grad.cpu().numpy()
    assert abs(loss.item() - f_ref) <= 1e-8 * abs(f_ref)
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) <= tol


def test_set_eps_reads_device_input_in_stream_order(env):
    """eps written by torch ops queued on a side stream behind a long matmul,
    then set_eps with no host synchronization: the library must read the
    finished values (in order on torch's current stream), so S matches the
    oracle's S of the intended eps."""
    torch, apf, AG = env
    w = W.TINY
    eps = w.eps_slab(2)
    sol = O.solve_S(O.problem_from_workload(w, eps))
    s = apf.solver_for_workload(w, np.full_like(eps, 1.5), precision="fp64")
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        a = torch.randn(4096, 4096, device="cuda", dtype=torch.float64)
        busy = (a @ a).sum() * 0.0  # keeps the side stream busy for a while
        x = torch.full(eps.shape, 7.0, dtype=torch.float64, device="cuda")
        x.copy_(torch.as_tensor(eps, device="cuda") + busy)
        s.set_eps(x, w.eps_sub, w.eps_clad, j0=w.j0)
        S = s.solve_S()
    assert np.linalg.norm(S - sol.S) / np.linalg.norm(sol.S) <= 1e-10


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


def test_multistart_on_one_gpu(env):
    """Multi-start beam-splitter optimisation (Sec. 3) through the replica
    helpers on one rank: every start is a seeded design optimised by the
    Armijo line search on the GPU; the gathered best is the minimum final f
    and every history decreases."""
    torch, apf, AG = env
    from paper_2306_09257_gb300 import replicas
    w = W.TINY
    s = apf.solver_for_workload(w, w.eps_slab(0), precision="mixed")
    res = replicas.multistart(
        lambda st: replicas.optimize_start(s, w, st, "splitter", [-1, 1], 0.25, iters=4), 3)
    assert [r[0] for r in res["runs"]] == [0, 1, 2]
    assert res["best_f"] == min(r[2] for r in res["runs"])
    assert all(h[-1] < h[0] for _, _, _, h in res["runs"])
    assert res["best_design"].shape == (w.h, w.nx)


@pytest.mark.slow
def test_central_fd_on_16_pixels_xlarge(env):
    """The differentiation workload itself (8192 x 280, 20 x 8192 slab, 513 x
    513 channels): central differences of the beam-splitter f (step 1e-6 in
    eps) on 16 seeded pixels against the single-elimination gradient.  The
    solves are refined to 1e-13 (float64 accuracy of S), so f's rounding noise
    over 2h stays far below the gradient; the bound allows for the O(h^2)
    truncation and that noise."""
    torch, apf, AG = env
    w = W.XLARGE
    eps = w.eps_slab(3)
    s = apf.solver_for_workload(w, eps, precision="mixed")
    s.set_refinement(1e-13, 40)
    orders = [-2, -1, 0, 1, 2]
    _, f0, g = s.solve_S_grad("splitter", orders, 0.18, allow_noconv=True)
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
            vals.append(s.solve_S_grad("splitter", orders, 0.18, allow_noconv=True)[1])
        fd.append((vals[0] - vals[1]) / (2 * h))
    fd = np.array(fd)
    ga = np.array([g[j, x] for j, x in pix])
    err = np.linalg.norm(fd - ga) / np.linalg.norm(ga)
    print(f"xlarge FD check: rel err {err:.2e}, |g| {np.linalg.norm(ga):.3e}")
    assert err < 1e-4, err
