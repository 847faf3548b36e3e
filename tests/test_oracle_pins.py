"""Pins for the CPU oracle: checks against facts the paper and the mathematics
fix, independent of the oracle's own formulas.

* 1-D reduction: a slab of uniform eps makes every row x-uniform, so each
  Fourier order decouples into a tridiagonal problem along y, solved here by
  LAPACK's banded solver (library routine), not by the 2D assembly.
* Homogeneous medium: S is diagonal with the plane-wave phase
  exp(i k_y (j_out - j_src)), up to PML reflection (closed form).
* Flux conservation for real eps: sum |t|^2 + sum |r|^2 = 1 (lossless).
* Reciprocity (A = A^T, the symmetry the paper uses for dA/dp):
  S_rev(-a <- -b) = S(b <- a).
* Cyclic x-shift and mirror invariants (exact).
* Gradient: central finite differences; the midpoint-Taylor cubic remainder of
  the paper's gradient validation (Supplement Sec. 3, Fig. S3); brute-force
  single-pixel dS from the derivative identity stated before Eq. (2).
* Wirtinger derivative of Eq. (5) (the formula printed after it): first-order
  change of f under a small complex perturbation of S.
"""
import math

import numpy as np
import pytest
from scipy.linalg import solve_banded

import oracle as O
from paper_2306_09257_gb300 import workloads as W


def small_problem(nx=32, ny=110, npml=30, lam=9.0, h=4, seed=0, eps_sub=2.25,
                  eps_clad=1.0, eps_slab=None):
    if eps_slab is None:
        eps_slab = W.iid_eps(h, nx, seed, 1.0, 4.0)
    j0 = npml + (ny - 2 * npml - h) // 2
    return O.Problem(nx=nx, ny=ny, npml_bot=npml, npml_top=npml, lambda_px=lam,
                     eps_slab=np.asarray(eps_slab, float), j0=j0, eps_sub=eps_sub,
                     eps_clad=eps_clad)


def grazing_margin(pb):
    """Smallest k_y over the orders used on both sides (grazing => PML reflects)."""
    ky1, _ = O.ky_nu(pb.nx, pb.k, pb.eps_clad, pb.outputs())
    ky2, _ = O.ky_nu(pb.nx, pb.k, pb.eps_sub, O.propagating_orders(pb.nx, pb.k, pb.eps_sub))
    return min(ky1.min(), ky2.min())


def test_layout_has_no_grazing_orders():
    pb = small_problem()
    assert grazing_margin(pb) > 0.2


def thomas_1d(pb, m, eps_slab_value):
    """Tridiagonal problem along y for Fourier order m, written from the
    operator's definition and solved with LAPACK gbsv (solve_banded); returns
    the projection on the output row."""
    e = field_1d(pb, m, eps_slab_value)
    _, nu_out = O.ky_nu(pb.nx, pb.k, pb.eps_clad, [m])
    return math.sqrt(nu_out[0]) * e[pb.j_out]


def field_1d(pb, m, eps_slab_value):
    """The field along y of the decoupled 1-D problem of Fourier order m for
    a unit-flux source on the source row."""
    ny, k = pb.ny, pb.k
    lam_m = 2.0 - 2.0 * math.cos(2.0 * math.pi * m / pb.nx)
    eps = np.full(ny, pb.eps_sub)
    eps[pb.j0:pb.j0 + pb.h] = eps_slab_value
    eps[pb.j0 + pb.h:] = pb.eps_clad
    s = np.array([O.stretch(float(j), pb) for j in range(ny)])
    sh = np.array([O.stretch(j - 0.5, pb) for j in range(ny + 1)])
    ab = np.zeros((3, ny), complex)
    ab[1] = s * (lam_m - k * k * eps) + 1.0 / sh[1:] + 1.0 / sh[:-1]
    ab[0, 1:] = -1.0 / sh[1:-1]   # super-diagonal A[j, j+1]
    ab[2, :-1] = -1.0 / sh[1:-1]  # sub-diagonal A[j+1, j]
    rhs = np.zeros(ny, complex)
    _, nu_in = O.ky_nu(pb.nx, k, pb.eps_sub, [m])
    rhs[pb.j_src] = -2j * math.sqrt(nu_in[0])
    return solve_banded((1, 1), ab, rhs)


def test_uniform_slab_matches_1d_banded_solve():
    pb = small_problem(eps_slab=np.full((4, 32), 3.1))
    sol = O.solve_S(pb)
    S = sol.S
    m = pb.inputs()
    diag = np.array([thomas_1d(pb, int(mm), 3.1) for mm in m])
    assert np.max(np.abs(np.diag(S) - diag)) < 1e-12 * np.max(np.abs(diag)) + 1e-13
    off = S - np.diag(np.diag(S))
    assert np.max(np.abs(off)) < 1e-12


def test_uniform_slab_reflection_matches_1d_banded_solve():
    """The reflection block of a uniform slab is diagonal, and each entry is
    the decoupled 1-D problem's source-row field, projected with the
    substrate flux normalisation, minus the incident wave."""
    pb = small_problem(eps_slab=np.full((4, 32), 3.1))
    sol = O.solve_S(pb)
    m = pb.inputs()
    R = O.reflection(sol, m)
    _, nu = O.ky_nu(pb.nx, pb.k, pb.eps_sub, m)
    diag = np.array([math.sqrt(nu[i]) * field_1d(pb, int(mm), 3.1)[pb.j_src] - 1.0 for i, mm in enumerate(m)])
    assert np.max(np.abs(np.diag(R) - diag)) < 1e-12 * max(1.0, np.max(np.abs(diag)))
    assert np.max(np.abs(R - np.diag(np.diag(R)))) < 1e-12
    # a slab of contrast 3.1 / 2.25 / 1 reflects measurably
    assert np.min(np.abs(diag)) > 1e-3


def test_homogeneous_medium_closed_form():
    pb = small_problem(eps_sub=1.0, eps_clad=1.0, eps_slab=np.ones((4, 32)))
    sol = O.solve_S(pb)
    ky, _ = O.ky_nu(pb.nx, pb.k, 1.0, pb.inputs())
    expect = np.exp(1j * ky * (pb.j_out - pb.j_src))
    # PML reflection of this profile at these angles is below 1e-4 in amplitude.
    assert np.max(np.abs(np.diag(sol.S) - expect)) < 2e-4
    assert np.max(np.abs(sol.S - np.diag(np.diag(sol.S)))) < 1e-12


def test_flux_conservation_lossless():
    pb = small_problem(seed=3)
    sol = O.solve_S(pb)
    R = O.reflection(sol)
    flux = (np.abs(sol.S) ** 2).sum(0) + (np.abs(R) ** 2).sum(0)
    assert np.max(np.abs(flux - 1.0)) < 2e-4
    # and a non-trivial scatterer: energy really leaves the specular order
    assert np.min(np.abs(np.diag(sol.S))) < 0.95


def test_reciprocity():
    pb = small_problem(seed=1)
    S = O.solve_S(pb).S
    Sr = O.solve_reverse_S(pb)
    pin = {int(m): i for i, m in enumerate(pb.inputs())}
    pout = {int(m): i for i, m in enumerate(pb.outputs())}
    for b, mb in enumerate(pb.outputs()):
        for a, ma in enumerate(pb.inputs()):
            assert abs(Sr[pin[-int(ma)], pout[-int(mb)]] - S[b, a]) < 1e-12


def test_reflection_reciprocity():
    """A = A^T: the reflection block satisfies R(m_b <- m_a) = R(-m_a <- -m_b)
    on a scattering slab (orders propagating in the substrate, a set closed
    under m -> -m)."""
    pb = small_problem(seed=4)
    sol = O.solve_S(pb)
    orders = O.propagating_orders(pb.nx, pb.k, pb.eps_sub)
    R = O.reflection(sol, orders)
    pin = {int(m): i for i, m in enumerate(pb.inputs())}
    pref = {int(m): i for i, m in enumerate(orders)}
    checked = 0
    for b, mb in enumerate(orders):
        for a, ma in enumerate(pb.inputs()):
            if -int(mb) in pin:
                assert abs(R[pref[-int(ma)], pin[-int(mb)]] - R[b, a]) < 1e-12
                checked += 1
    assert checked >= len(pb.inputs()) ** 2
    assert np.max(np.abs(R)) > 1e-3  # the slab really reflects


@pytest.mark.parametrize("shift", [1, 7])
def test_cyclic_shift_invariant(shift):
    pb = small_problem(seed=2)
    S = O.solve_S(pb).S
    pb2 = small_problem(eps_slab=np.roll(pb.eps_slab, shift, axis=1))
    S2 = O.solve_S(pb2).S
    ma, mb = pb.inputs()[None, :], pb.outputs()[:, None]
    phase = np.exp(2j * np.pi * (ma - mb) * shift / pb.nx)
    assert np.max(np.abs(S2 - S * phase)) < 1e-12


def test_mirror_invariant():
    pb = small_problem(seed=4)
    S = O.solve_S(pb).S
    mir = pb.eps_slab[:, (-np.arange(pb.nx)) % pb.nx]
    S2 = O.solve_S(small_problem(eps_slab=mir)).S
    m = pb.inputs()  # symmetric set, ascending -> index of -m is reversed index
    assert np.array_equal(m, -m[::-1])
    assert np.max(np.abs(S2[::-1, ::-1] - S)) < 1e-12


def test_wirtinger_derivative_of_eq5():
    rng = np.random.default_rng(0)
    pb = small_problem()
    m = pb.inputs()
    S = rng.normal(size=(len(m), len(m))) + 1j * rng.normal(size=(len(m), len(m)))
    S *= 0.3
    for kind, t in (("power", 0.0), ("splitter", 0.18)):
        f0, G = O.objective(S, kind, m, m, [-2, -1, 0, 1, 2], t)
        d = 1e-7 * (rng.normal(size=S.shape) + 1j * rng.normal(size=S.shape))
        f1, _ = O.objective(S + d, kind, m, m, [-2, -1, 0, 1, 2], t)
        lin = 2.0 * np.real(np.sum(G * d))
        # remainder is second order in |d| ~ 1e-7
        assert abs((f1 - f0) - lin) < 1e-5 * abs(lin)


def test_relative_pairs_small_example():
    pairs = O.relative_pairs(np.array([-1, 0, 1]), np.array([-2, -1, 0, 1]), [1])
    # input -1 -> output 0 (index 2); input 0 -> output 1 (index 3); input 1 -> 2 absent
    assert pairs == [(2, 0), (3, 1)]


def _f(pb, kind, orders, t):
    S = O.solve_S(pb).S
    return O.objective(S, kind, pb.inputs(), pb.outputs(), orders, t)[0]


@pytest.mark.parametrize("kind,orders,t", [("power", [0], 0.0),
                                           ("splitter", [-2, -1, 0, 1, 2], 0.18)])
def test_gradient_central_fd(kind, orders, t):
    pb = small_problem(seed=5)
    sol, f, G, g = O.f_and_grad(pb, kind, orders, t)
    rng = np.random.default_rng(11)
    hstep = 1e-6
    for _ in range(6):
        j, x = int(rng.integers(pb.h)), int(rng.integers(pb.nx))
        ep, em = pb.eps_slab.copy(), pb.eps_slab.copy()
        ep[j, x] += hstep
        em[j, x] -= hstep
        fd = (_f(small_problem(eps_slab=ep), kind, orders, t)
              - _f(small_problem(eps_slab=em), kind, orders, t)) / (2 * hstep)
        assert abs(fd - g[j, x]) < 1e-6 * np.max(np.abs(g)) + 1e-9


def test_midpoint_taylor_remainder_is_cubic():
    """|f(p+dp) - f(p) - grad f(p+dp/2).dp| = O(|dp|^3) (Supplement Sec. 3)."""
    pb = small_problem(seed=6)
    rng = np.random.default_rng(7)
    direction = rng.normal(size=pb.eps_slab.shape)
    direction /= np.linalg.norm(direction)
    f0 = _f(pb, "splitter", [-1, 1], 0.5)
    res = []
    steps = [4e-2, 2e-2, 1e-2]
    for s in steps:
        dp = s * direction
        f1 = _f(small_problem(eps_slab=pb.eps_slab + dp), "splitter", [-1, 1], 0.5)
        mid = small_problem(eps_slab=pb.eps_slab + dp / 2)
        _, _, _, gmid = O.f_and_grad(mid, "splitter", [-1, 1], 0.5)
        res.append(abs(f1 - f0 - np.sum(gmid * dp)))
    slopes = np.diff(np.log(res)) / np.diff(np.log(steps))
    assert np.all(slopes > 2.6) and np.all(slopes < 3.4), slopes


def test_brute_force_single_pixel_dS():
    pb = small_problem(seed=8)
    sol = O.solve_S(pb)
    j, x = 2, 13
    dS = O.dS_deps_pixel(sol, j, x)
    hstep = 1e-6
    ep, em = pb.eps_slab.copy(), pb.eps_slab.copy()
    ep[j, x] += hstep
    em[j, x] -= hstep
    fd = (O.solve_S(small_problem(eps_slab=ep)).S - O.solve_S(small_problem(eps_slab=em)).S) / (2 * hstep)
    assert np.max(np.abs(fd - dS)) < 1e-7 * np.max(np.abs(dS))
