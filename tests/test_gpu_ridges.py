"""Ridge edge-position parametrization on the GPU (paper Sec. 3, Eq. 5)
against the oracle: the slab permittivity, the chain rule to the edges, and
S + df/d(edges) end to end; the autograd path against differences."""
import numpy as np
import pytest

import oracle as O
from paper_2306_09257_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ORDERS = [-2, -1, 0, 1, 2]
TOL = {"fp64": (1e-10, 1e-10), "mixed": (1e-6, 1e-5)}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def apf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_09257_gb300 import apf as A, build
    build.build_lib()
    A.load_library()
    return A


def grid_solver(apf, w, precision="fp64"):
    s = apf.Solver(0, precision)
    s.set_grid(w.nx, w.ny, w.npml, w.npml, w.lambda_px)
    return s


@pytest.mark.parametrize("mirror", [True, False])
@pytest.mark.parametrize("w", [W.TINY, W.MID], ids=["64", "1024"])
def test_ridge_eps_matches_oracle(apf, w, mirror):
    s = grid_solver(apf, w)
    e = W.ridge_edges(w.nx, W.ridge_count(w), 5, mirror=mirror)
    eps = s.set_ridges(e, w.h, 4.0, 1.0, w.eps_sub, w.eps_clad, mirror=mirror, j0=w.j0)
    ref = O.eps_from_edges(w.nx, w.h, e, mirror, 4.0, 1.0)
    assert np.max(np.abs(eps - ref)) <= 1e-14 * 4.0


def test_ridge_eps_device_buffers(apf):
    import torch
    w = W.MID
    s = grid_solver(apf, w)
    e = W.ridge_edges(w.nx, W.ridge_count(w), 9, mirror=True)
    out = torch.empty((w.h, w.nx), dtype=torch.float64, device="cuda")
    s.set_ridges(torch.as_tensor(e, device="cuda"), w.h, 13.69, 1.0, w.eps_sub, w.eps_clad, eps_out=out)
    ref = O.eps_from_edges(w.nx, w.h, e, True, 13.69, 1.0)
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-14 * 13.69


@pytest.mark.parametrize("mirror", [True, False])
def test_ridge_chain_rule_matches_oracle(apf, mirror):
    """The same seeded pixel gradient through apf_ridge_grad and the oracle's
    Jacobian; edges include exact pixel boundaries, the mirror plane and the
    period boundary."""
    import torch
    w = W.MID
    s = grid_solver(apf, w)
    e = W.ridge_edges(w.nx, 20, 3, mirror=mirror)
    e[0] = -w.nx / 2.0            # period boundary
    e[3] = np.floor(e[3])          # on a pixel boundary
    if mirror:
        e[-1] = 0.0                # on the mirror plane
    s.set_ridges(e, w.h, 13.69, 1.0, w.eps_sub, w.eps_clad, mirror=mirror)
    g = np.random.default_rng(1).standard_normal((w.h, w.nx))
    ge = s.ridge_grad(g)
    ref = O.grad_edges(g, w.nx, e, mirror, 13.69, 1.0)
    assert rel(ge, ref) <= 1e-13
    gd = torch.empty(len(e), dtype=torch.float64, device="cuda")
    s.ridge_grad(torch.as_tensor(g, device="cuda"), out=gd)
    assert rel(gd.cpu().numpy(), ref) <= 1e-13


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("mirror", [True, False])
def test_ridge_S_and_edge_gradient(apf, prec, mirror):
    w = W.TINY
    e = W.ridge_edges(w.nx, 3, 21, mirror=mirror, min_gap=2.5)
    eps = O.eps_from_edges(w.nx, w.h, e, mirror, 4.0, 1.0)
    sol, f_ref, _, g_ref = O.f_and_grad(O.problem_from_workload(w, eps), "splitter", ORDERS, 0.18)
    ge_ref = O.grad_edges(g_ref, w.nx, e, mirror, 4.0, 1.0)
    s = grid_solver(apf, w, prec)
    s.set_ridges(e, w.h, 4.0, 1.0, w.eps_sub, w.eps_clad, mirror=mirror, j0=w.j0)
    s.set_channels(None, None)
    S, f, g = s.solve_S_grad("splitter", ORDERS, 0.18)
    ge = s.ridge_grad(g)
    ts, tg = TOL[prec]
    print(f"ridges {prec} mirror={mirror}: err S {rel(S, sol.S):.2e}, err dS/dedges {rel(ge, ge_ref):.2e}")
    assert rel(S, sol.S) <= ts
    assert rel(ge, ge_ref) <= tg


@pytest.mark.slow
def test_ridge_mid_grid_silicon(apf):
    """1024 x 240 grid, 40 a-Si ridges per half period (eps 13.69) in air on
    silica, mirror symmetric: S and df/d(edges) against the oracle."""
    w = W.MID
    e = W.ridge_edges(w.nx, W.ridge_count(w), 2, mirror=True)
    eps = O.eps_from_edges(w.nx, w.h, e, True, 13.69, 1.0)
    sol, f_ref, _, g_ref = O.f_and_grad(O.problem_from_workload(w, eps), "splitter", ORDERS, 0.18)
    ge_ref = O.grad_edges(g_ref, w.nx, e, True, 13.69, 1.0)
    for prec in ("fp64", "mixed"):
        s = grid_solver(apf, w, prec)
        s.set_ridges(e, w.h, 13.69, 1.0, w.eps_sub, w.eps_clad, j0=w.j0)
        s.set_channels(None, None)
        S, f, g = s.solve_S_grad("splitter", ORDERS, 0.18)
        ge = s.ridge_grad(g)
        ts, tg = TOL[prec]
        print(f"ridges mid {prec}: err S {rel(S, sol.S):.2e}, err dS/dedges {rel(ge, ge_ref):.2e}")
        assert rel(S, sol.S) <= ts and rel(ge, ge_ref) <= tg


def test_ridge_autograd_against_differences(apf):
    import torch
    from paper_2306_09257_gb300 import autograd as AG
    w = W.TINY
    s = grid_solver(apf, w)
    e0 = W.ridge_edges(w.nx, 3, 4, mirror=True, min_gap=2.5)
    s.set_ridges(e0, w.h, 4.0, 1.0, w.eps_sub, w.eps_clad, j0=w.j0)
    s.set_channels(None, None)
    mi, mo = s.channels()
    mask = AG.relative_order_mask(mi, mo, ORDERS, device="cuda")
    geom = dict(h=w.h, eps_ridge=4.0, eps_bg=1.0, eps_sub=w.eps_sub, eps_clad=w.eps_clad, j0=w.j0)

    def loss(edges):
        return AG.splitter_loss(AG.ridge_scattering(edges, s, **geom), mask, 0.18)

    e = torch.tensor(e0, dtype=torch.float64, device="cuda", requires_grad=True)
    L = loss(e)
    L.backward()
    step = 1e-4
    fd = []
    with torch.no_grad():
        for k in range(len(e0)):
            ep, em = e.detach().clone(), e.detach().clone()
            ep[k] += step
            em[k] -= step
            fd.append(((loss(ep) - loss(em)) / (2 * step)).item())
    fd = np.array(fd)
    assert rel(e.grad.cpu().numpy(), fd) <= 1e-6


def test_ridge_argument_errors(apf):
    w = W.TINY
    s = grid_solver(apf, w)
    with pytest.raises(apf.APFError) as ei:
        s.ridge_grad(np.zeros((w.h, w.nx)))
    assert ei.value.code == apf.APF_ESTATE
    for bad, mirror in (([-10.0, -12.0], True), ([-10.0, -8.0, -5.0], True), ([-40.0, -8.0], True),
                        ([-10.0, 3.0], True), ([-10.0, float("nan")], False)):
        with pytest.raises(apf.APFError) as ei:
            s.set_ridges(np.array(bad), w.h, 4.0, 1.0, w.eps_sub, w.eps_clad, mirror=mirror)
        assert ei.value.code == apf.APF_EINVAL


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_high_contrast_ridges_converge_at_defaults(apf, seed):
    """Amorphous-silicon ridges (eps 13.69, the paper's Sec. 3 material) in
    air on silica, 1024 x 240: the mixed path at the library's default
    refinement (tolerance 1e-10, 40 sweeps) converges (no APF_ENOCONV) and
    agrees with the float64 path."""
    w = W.MID
    e = W.ridge_edges(w.nx, W.ridge_count(w), seed, mirror=True)
    out = {}
    for prec in ("mixed", "fp64"):
        s = grid_solver(apf, w, prec)
        s.set_ridges(e, w.h, 13.69, 1.0, w.eps_sub, w.eps_clad, mirror=True, j0=w.j0, eps_out=False)
        s.set_channels(None, None)
        out[prec] = s.solve_S_grad("splitter", ORDERS, 0.18)
        if prec == "mixed":
            st = s.stats()
            assert st["residual"] <= 1e-10 and st["refine_iters"] <= 40, st
    assert rel(out["mixed"][0], out["fp64"][0]) <= 1e-8
    assert rel(out["mixed"][2], out["fp64"][2]) <= 1e-5
