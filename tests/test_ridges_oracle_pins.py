"""Pins of the ridge edge-position parametrization oracle (paper Sec. 3,
Eq. 5: p = ridge edge positions, mirror symmetry; Supplement Sec. 7 without
it), checked against closed forms, exact special cases and finite
differences of the oracle's own objective (not against the oracle's
derivative formula)."""
import numpy as np
import pytest

import oracle as O
from oracle import ridges as R
from paper_2306_09257_gb300 import workloads as W

EPS_R, EPS_B = 4.0, 1.0


@pytest.mark.parametrize("mirror", [True, False])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_covered_area_closed_form(mirror, seed):
    nx = 64
    e = W.ridge_edges(nx, 5, seed, mirror=mirror, min_gap=1.5)
    fill = O.fill_fraction(nx, e, mirror)
    width = float(np.sum(e[1::2] - e[0::2]))
    assert abs(fill.sum() - (2 if mirror else 1) * width) <= 1e-12 * nx
    assert fill.min() >= 0.0 and fill.max() <= 1.0 + 1e-15


@pytest.mark.parametrize("seed", [0, 3])
def test_mirror_symmetry_exact(seed):
    nx = 128
    e = W.ridge_edges(nx, 9, seed, mirror=True)
    eps = O.eps_from_edges(nx, 3, e, True, EPS_R, EPS_B)
    assert np.array_equal(eps, eps[:, ::-1])
    assert np.array_equal(eps[0], eps[2])


def test_integer_aligned_ridge():
    nx = 16
    eps = O.eps_from_edges(nx, 1, [-3.0, 2.0], False, EPS_R, EPS_B)[0]
    want = np.full(nx, EPS_B)
    want[5:10] = EPS_R  # [-3, 2) + nx/2 = pixels 5..9
    assert np.array_equal(eps, want)
    # a ridge inside one pixel covers exactly its width
    eps = O.eps_from_edges(nx, 1, [0.2, 0.7], False, EPS_R, EPS_B)[0]
    assert abs(eps[8] - (EPS_B + 0.5 * (EPS_R - EPS_B))) <= 1e-15
    assert np.count_nonzero(eps != EPS_B) == 1


def _fd_jacobian(nx, e, mirror, step, one_sided=False):
    J = np.zeros((len(e), nx))
    for k in range(len(e)):
        ep, em = np.array(e, float), np.array(e, float)
        ep[k] += step
        if not one_sided:
            em[k] -= step
        fp = O.eps_from_edges(nx, 1, ep, mirror, EPS_R, EPS_B)[0]
        fm = O.eps_from_edges(nx, 1, em, mirror, EPS_R, EPS_B)[0]
        J[k] = (fp - fm) / (step if one_sided else 2 * step)
    return J


@pytest.mark.parametrize("mirror", [True, False])
def test_jacobian_against_differences(mirror):
    nx = 48
    e = W.ridge_edges(nx, 4, 7, mirror=mirror)
    J = O.deps_dedges(nx, e, mirror, EPS_R, EPS_B)
    assert np.allclose(J, _fd_jacobian(nx, e, mirror, 1e-6), atol=1e-7, rtol=0)


def test_jacobian_one_sided_at_pixel_boundaries():
    # edges on integer positions: the derivative is the right-sided one
    nx = 32
    e = [-12.0, -9.0, -5.0, -2.0]
    J = O.deps_dedges(nx, e, True, EPS_R, EPS_B)
    assert np.allclose(J, _fd_jacobian(nx, e, True, 1e-6, one_sided=True), atol=1e-7, rtol=0)


def _tiny_problem(eps):
    return O.problem_from_workload(W.TINY, eps)


@pytest.mark.parametrize("mirror", [True, False])
def test_chain_rule_against_objective_differences(mirror):
    """df/dt from the pixel adjoint gradient and the ridge Jacobian against
    central differences of f itself (64 x 100 grid, Eq. 5 objective)."""
    w = W.TINY
    e = W.ridge_edges(w.nx, 3, 11, mirror=mirror, min_gap=2.5)
    orders = [-2, -1, 0, 1, 2]

    def f_of(edges):
        eps = O.eps_from_edges(w.nx, w.h, edges, mirror, EPS_R, EPS_B)
        return O.f_and_grad(_tiny_problem(eps), "splitter", orders, 0.18)

    _, f0, _, g = f_of(e)
    ge = O.grad_edges(g, w.nx, e, mirror, EPS_R, EPS_B)
    step = 1e-4
    fd = np.zeros(len(e))
    for k in range(len(e)):
        ep, em = np.array(e), np.array(e)
        ep[k] += step
        em[k] -= step
        fd[k] = (f_of(ep)[1] - f_of(em)[1]) / (2 * step)
    assert np.linalg.norm(ge - fd) <= 1e-6 * np.linalg.norm(fd), (ge, fd)


def test_planted_mirror_sign_mistake_is_caught(monkeypatch):
    """A plausible slip (the image edge's contribution with the wrong sign)
    must fail the difference pin."""
    nx = 48
    e = W.ridge_edges(nx, 4, 7, mirror=True)

    def wrong(nx_, edges, mirror, er, eb):
        J = np.zeros((len(edges), nx_))
        for k, t in enumerate(edges):
            s = -1.0 if k % 2 == 0 else 1.0
            J[k, R.edge_pixel(nx_, t)] += s * (er - eb)
            J[k, R.image_pixel(nx_, t)] -= s * (er - eb)
        return J

    J = wrong(nx, e, True, EPS_R, EPS_B)
    assert not np.allclose(J, _fd_jacobian(nx, e, True, 1e-6), atol=1e-7, rtol=0)


@pytest.mark.parametrize("mirror", [True, False])
def test_ridge_edge_generator_contract(mirror):
    """Input generator: sorted edges inside the half (or whole) period, every
    gap and both end margins at least min_gap, reproducible per seed."""
    for w in (W.TINY, W.MID, W.LARGE):
        n = W.ridge_count(w)
        e = W.ridge_edges(w.nx, n, 7, mirror=mirror)
        lo, hi = -w.nx / 2.0, (0.0 if mirror else w.nx / 2.0)
        assert e.shape == (2 * n,)
        assert np.all(np.diff(e) >= 2.0 - 1e-12)
        assert e[0] - lo >= 2.0 - 1e-12 and hi - e[-1] >= 2.0 - 1e-12
        assert np.array_equal(e, W.ridge_edges(w.nx, n, 7, mirror=mirror))
        assert not np.array_equal(e, W.ridge_edges(w.nx, n, 8, mirror=mirror))
    assert (W.ridge_count(W.MID), W.ridge_count(W.LARGE)) == (40, 133)
