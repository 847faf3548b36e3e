"""The conventional adjoint method of the paper's supplement (Sec. 1, Eq. S1)
on the GPU (apf_solve_S_grad_adjoint) against the CPU oracle, which computes
its gradient by exactly that method with SuperLU solves, and against the
library's single-elimination (APF) gradient."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2306_09257_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ORDERS = [-2, -1, 0, 1, 2]
TOL = {"fp64": (1e-10, 1e-10), "mixed": (1e-6, 1e-5)}


def close(got, ref, tol):
    got, ref = np.asarray(got), np.asarray(ref)
    e_fro = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    e_max = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert e_fro <= tol and e_max <= tol, (e_fro, e_max, tol)
    return e_fro


@pytest.fixture(scope="module")
def apf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_09257_gb300 import apf as A, build
    build.build_lib()
    A.load_library()
    return A


def solver(apf, pb, prec):
    s = apf.Solver(0, prec)
    s.set_grid(pb.nx, pb.ny, pb.npml_bot, pb.npml_top, pb.lambda_px, R0=pb.R0, power=pb.power)
    s.set_eps(pb.eps_slab, pb.eps_sub, pb.eps_clad, j0=pb.j0)
    s.set_channels(None if pb.m_in is None else list(pb.m_in), None if pb.m_out is None else list(pb.m_out))
    return s


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adjoint_method_matches_oracle(apf, prec, seed):
    w = W.TINY
    pb = O.problem_from_workload(w, w.eps_slab(seed))
    sol, f_ref, _, g_ref = O.f_and_grad(pb, "splitter", ORDERS, 0.18)
    s = solver(apf, pb, prec)
    S, f, g = s.solve_S_grad_adjoint("splitter", ORDERS, 0.18)
    ts, tg = TOL[prec]
    close(S, sol.S, ts)
    close(g, g_ref, tg)
    assert abs(f - f_ref) <= 10 * ts * abs(f_ref)


# more inputs than outputs (the two passes need 2 n_in field columns), fewer,
# a single slab row, and several 32-blocks
CASES = [
    dict(nx=64, ny=70, nb=10, nt=25, lam=8.0, h=2, m_in=[-4, -3, -1, 0, 2, 3, 5], m_out=[-1, 0, 1]),
    dict(nx=64, ny=70, nb=15, nt=15, lam=8.0, h=1, m_in=[0], m_out=None),
    dict(nx=128, ny=80, nb=12, nt=17, lam=11.3, h=5, m_in=None, m_out=None),
]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_adjoint_method_edge_cases(apf, prec, case):
    c = CASES[case]
    eps = W.iid_eps(c["h"], c["nx"], 200 + case, 1.0, 3.0)
    j0 = c["nb"] + (c["ny"] - c["nb"] - c["nt"] - c["h"]) // 2
    pb = O.Problem(nx=c["nx"], ny=c["ny"], npml_bot=c["nb"], npml_top=c["nt"], lambda_px=c["lam"],
                   eps_slab=eps, j0=j0, eps_sub=2.25, eps_clad=1.0,
                   m_in=None if c["m_in"] is None else np.array(c["m_in"]),
                   m_out=None if c["m_out"] is None else np.array(c["m_out"]))
    sol, f_ref, _, g_ref = O.f_and_grad(pb, "power", [-1, 0, 1], 0.0)
    s = solver(apf, pb, prec)
    S, f, g = s.solve_S_grad_adjoint("power", [-1, 0, 1])
    ts, tg = TOL[prec]
    close(S, sol.S, ts)
    close(g, g_ref, tg)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_method_mid_against_golden_and_apf(apf, prec):
    """1024 x 240, 103 x 103 channels: against the stored oracle values, and
    against the single-elimination gradient of the same context (the two
    methods compute the same derivative; they differ only in how many
    sweeps and which products)."""
    ref = np.load(os.path.join(HERE, "golden", "mid_1024x240_seed0.npz"))
    w = W.MID
    eps = w.eps_slab(0)
    s = apf.solver_for_workload(w, eps, precision=prec)
    S_a, f_a, g_a = s.solve_S_grad_adjoint("splitter", ORDERS, 0.18)
    S_p, f_p, g_p = s.solve_S_grad("splitter", ORDERS, 0.18)
    ts, tg = TOL[prec]
    close(S_a, ref["S"], ts)
    close(g_a, ref["grad"], tg)
    close(g_a, g_p, tg)
    assert abs(f_a - f_p) <= 10 * ts * abs(f_p)


def test_adjoint_fields_are_not_reused_for_gamma(apf):
    """After the adjoint method the stored fields are forward + adjoint-method
    columns: grad_from_gamma and reverse_S refuse them until the next APF
    solve; the reflection block (forward fields only) still works."""
    w = W.TINY
    pb = O.problem_from_workload(w, w.eps_slab(4))
    s = solver(apf, pb, "fp64")
    S, f, g = s.solve_S_grad_adjoint("power", [0])
    R_a = s.reflection()
    with pytest.raises(apf.APFError) as e:
        s.grad_from_gamma(np.zeros_like(S))
    assert e.value.code == apf.APF_ESTATE
    with pytest.raises(apf.APFError) as e:
        s.reverse_S()
    assert e.value.code == apf.APF_ESTATE
    S2 = s.solve_S()
    assert np.linalg.norm(S2 - S) <= 1e-13 * np.linalg.norm(S)
    assert np.linalg.norm(s.reflection() - R_a) <= 1e-13 * np.linalg.norm(R_a)
    s.grad_from_gamma(np.zeros_like(S))
