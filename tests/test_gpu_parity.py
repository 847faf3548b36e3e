"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (rel-Frobenius over all of S and all slab pixels of df/deps):
float64 mode 1e-10 on S and on the gradient; mixed mode 1e-6 on S and 1e-5
on the gradient.  Beside the norm, every element is checked: the largest
absolute difference must stay within the same tolerance times the largest
reference entry, so one wrong small entry (a near-grazing order, one pixel)
cannot hide inside the norm.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2306_09257_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
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


def close(got, ref, tol):
    """rel-Frobenius and element-wise max-abs agreement within tol."""
    got, ref = np.asarray(got), np.asarray(ref)
    e_fro = rel(got, ref)
    e_max = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert e_fro <= tol and e_max <= tol, (e_fro, e_max, tol)
    return e_fro


def make_solver(apf, pb, precision):
    s = apf.Solver(device=0, precision=precision)
    s.set_grid(pb.nx, pb.ny, pb.npml_bot, pb.npml_top, pb.lambda_px, R0=pb.R0, power=pb.power)
    s.set_eps(pb.eps_slab, pb.eps_sub, pb.eps_clad, j0=pb.j0)
    s.set_channels(None if pb.m_in is None else list(pb.m_in), None if pb.m_out is None else list(pb.m_out))
    return s


PRECS = ["fp64", "mixed"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_S_and_grad(apf, prec, seed):
    w = W.TINY
    pb = O.problem_from_workload(w, w.eps_slab(seed))
    orders = [-2, -1, 0, 1, 2]
    sol, f_ref, _, g_ref = O.f_and_grad(pb, "splitter", orders, 0.18)
    s = make_solver(apf, pb, prec)
    mi, mo = s.channels()
    assert np.array_equal(mi, pb.inputs()) and np.array_equal(mo, pb.outputs())
    S, f, g = s.solve_S_grad("splitter", orders, 0.18)
    ts, tg = TOL[prec]
    print(f"parity tiny seed {seed} {prec}: err S {rel(S, sol.S):.2e}, err grad {rel(g, g_ref):.2e}")
    close(S, sol.S, ts)
    close(g, g_ref, tg)
    assert abs(f - f_ref) <= ts * abs(f_ref) * 10


@pytest.mark.parametrize("prec", PRECS)
def test_tiny_power_objective(apf, prec):
    w = W.TINY
    pb = O.problem_from_workload(w, w.eps_slab(3))
    sol, f_ref, _, g_ref = O.f_and_grad(pb, "power", [0], 0.0)
    s = make_solver(apf, pb, prec)
    S, f, g = s.solve_S_grad("power", [0])
    ts, tg = TOL[prec]
    close(S, sol.S, ts)
    close(g, g_ref, tg)


# Ragged and edge cases: one leaf (nx=32), several leaves (nx=128), a single
# slab row, two rows, unequal PMLs, an off-centre slab, channel subsets.
EDGE = [
    dict(nx=32, ny=90, nb=20, nt=20, lam=9.0, h=3, j0=-1, m_in=None, m_out=None),
    dict(nx=128, ny=80, nb=12, nt=17, lam=11.3, h=5, j0=30, m_in=None, m_out=None),
    dict(nx=64, ny=70, nb=15, nt=15, lam=8.0, h=1, j0=-1, m_in=None, m_out=None),
    dict(nx=64, ny=70, nb=10, nt=25, lam=8.0, h=2, j0=-1, m_in=[-3, 0, 2], m_out=[-2, -1, 0, 1, 4]),
    dict(nx=256, ny=64, nb=8, nt=8, lam=23.0, h=7, j0=-1, m_in=None, m_out=None),
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("case", range(len(EDGE)))
def test_edge_cases(apf, prec, case):
    c = EDGE[case]
    eps = W.iid_eps(c["h"], c["nx"], 100 + case, 1.0, 3.0)
    j0 = c["j0"] if c["j0"] >= 0 else c["nb"] + (c["ny"] - c["nb"] - c["nt"] - c["h"]) // 2
    pb = O.Problem(nx=c["nx"], ny=c["ny"], npml_bot=c["nb"], npml_top=c["nt"], lambda_px=c["lam"],
                   eps_slab=eps, j0=j0, eps_sub=2.25, eps_clad=1.0,
                   m_in=None if c["m_in"] is None else np.array(c["m_in"]),
                   m_out=None if c["m_out"] is None else np.array(c["m_out"]))
    sol, f_ref, _, g_ref = O.f_and_grad(pb, "splitter", [-1, 0, 1], 0.3)
    s = make_solver(apf, pb, prec)
    S, f, g = s.solve_S_grad("splitter", [-1, 0, 1], 0.3)
    ts, tg = TOL[prec]
    close(S, sol.S, ts)
    close(g, g_ref, tg)


@pytest.mark.parametrize("prec", PRECS)
def test_mid_against_golden(apf, prec):
    """1024 x 240, 103 x 103 channels, against oracle values written by
    tests/golden/make_golden.py."""
    ref = np.load(os.path.join(HERE, "golden", "mid_1024x240_seed0.npz"))
    w = W.MID
    eps = w.eps_slab(0)
    assert np.array_equal(eps, ref["eps"])
    from paper_2306_09257_gb300 import apf as A
    s = A.solver_for_workload(w, eps, precision=prec)
    S, f, g = s.solve_S_grad("splitter", [-2, -1, 0, 1, 2], 0.18)
    ts, tg = TOL[prec]
    print(f"parity mid {prec}: err S {rel(S, ref['S']):.2e}, err grad {rel(g, ref['grad']):.2e}")
    close(S, ref["S"], ts)
    close(g, ref["grad"], tg)


@pytest.mark.parametrize("prec", PRECS)
def test_grad_from_gamma_and_device_buffers(apf, prec):
    """Caller-supplied Gamma after solve_S equals the built-in objective path;
    device (torch) buffers give the same result as host buffers."""
    import torch
    w = W.TINY
    pb = O.problem_from_workload(w, w.eps_slab(4))
    s = make_solver(apf, pb, prec)
    S_h, f, g_h = s.solve_S_grad("power", [0, 1])
    _, G = O.objective(S_h, "power", pb.inputs(), pb.outputs(), [0, 1])
    S2 = s.solve_S()
    g2 = s.grad_from_gamma(G)
    assert rel(g2, g_h) <= 1e-12
    S_d = torch.empty(S_h.shape, dtype=torch.complex128, device="cuda")
    g_d = torch.empty(g_h.shape, dtype=torch.float64, device="cuda")
    s.solve_S_grad("power", [0, 1], out_S=S_d, out_grad=g_d)
    assert rel(S_d.cpu().numpy(), S_h) <= 1e-13 and rel(g_d.cpu().numpy(), g_h) <= 1e-12
    eps_d = torch.tensor(pb.eps_slab, device="cuda")
    s.set_eps(eps_d, pb.eps_sub, pb.eps_clad, j0=pb.j0)
    S3 = s.solve_S()
    assert rel(S3, S2) <= 1e-13


def test_errors_are_reported(apf):
    s = apf.Solver(0, "fp64")
    with pytest.raises(apf.APFError) as e:
        s.solve_S(out=np.empty((1, 1), np.complex128))
    assert e.value.code == apf.APF_ESTATE
    with pytest.raises(apf.APFError) as e:
        s.set_grid(100, 100, 20, 20, 16.0)  # not a power of two
    assert e.value.code == apf.APF_EINVAL
    s.set_grid(64, 100, 20, 20, 16.0)
    bad = np.ones((6, 64))
    bad[2, 5] = np.nan
    with pytest.raises(apf.APFError) as e:
        s.set_eps(bad, 2.25, 1.0)
    assert e.value.code == apf.APF_EINVAL
    with pytest.raises(apf.APFError):
        s.set_eps(np.ones((70, 64)), 2.25, 1.0)  # slab overlaps source row
    s.set_eps(np.ones((6, 64)) * 2.0, 2.25, 1.0)
    with pytest.raises(apf.APFError):
        s.set_channels([40], None)  # evanescent input
    s.set_channels()
    with pytest.raises(apf.APFError):
        s.solve_S_grad("power", [])  # no orders
