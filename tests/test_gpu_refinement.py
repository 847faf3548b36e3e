"""Mixed-mode refinement by restarted GMRES (apf_set_krylov): parity with the
oracle, agreement with plain refinement on high-contrast ridge designs (the
designs that refine slowly), argument checks."""
import numpy as np
import pytest

import oracle as O
from paper_2306_09257_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ORDERS = [-2, -1, 0, 1, 2]


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


@pytest.mark.parametrize("m", [2, 3])
def test_gmres_parity_with_oracle(apf, m):
    w = W.TINY
    pb = O.problem_from_workload(w, w.eps_slab(1))
    sol, f_ref, _, g_ref = O.f_and_grad(pb, "splitter", ORDERS, 0.18)
    s = apf.solver_for_workload(w, w.eps_slab(1), precision="mixed")
    s.set_krylov(m)
    S, f, g = s.solve_S_grad("splitter", ORDERS, 0.18)
    assert rel(S, sol.S) <= 1e-6 and rel(g, g_ref) <= 1e-5
    assert s.stats()["residual"] <= 1e-10


def ridge_solver(apf, w, seed, m):
    s = apf.Solver(0, "mixed")
    s.set_grid(w.nx, w.ny, w.npml, w.npml, w.lambda_px)
    s.set_ridges(W.ridge_edges(w.nx, W.ridge_count(w), seed, mirror=True), w.h, 13.69, 1.0, w.eps_sub,
                 w.eps_clad, j0=w.j0, eps_out=False)
    s.set_channels(None, None)
    s.set_krylov(m)
    return s


@pytest.mark.parametrize("seed", [502, 701])
def test_gmres_on_slowly_refining_ridge_designs(apf, seed):
    """4096 x 260 grid, a-Si ridges: the two seeded designs that need the most
    plain refinement sweeps.  Both refinements must reach 1e-10 and agree."""
    w = W.LARGE
    out = {}
    for m in (0, 3):
        s = ridge_solver(apf, w, seed, m)
        S, f, g = s.solve_S_grad("splitter", ORDERS, 0.18)
        st = s.stats()
        out[m] = (S, g, st["refine_iters"], st["residual"])
        s.close()
    print(f"ridge seed {seed}: plain {out[0][2]} sweeps (residual {out[0][3]:.1e}), "
          f"GMRES(3) {out[3][2]} preconditioner applications (residual {out[3][3]:.1e})")
    assert out[0][3] <= 1e-10 and out[3][3] <= 1e-10
    assert rel(out[3][0], out[0][0]) <= 1e-8
    assert rel(out[3][1], out[0][1]) <= 1e-6


def test_set_krylov_arguments_and_reallocation(apf):
    w = W.TINY
    s = apf.solver_for_workload(w, w.eps_slab(0), precision="mixed")
    S0 = s.solve_S()
    with pytest.raises(apf.APFError) as ei:
        s.set_krylov(9)
    assert ei.value.code == apf.APF_EINVAL
    s.set_krylov(2)          # re-creates the workspace
    S1 = s.solve_S()
    s.set_krylov(0)
    S2 = s.solve_S()
    assert rel(S1, S0) <= 1e-9 and rel(S2, S0) <= 1e-9
    s64 = apf.solver_for_workload(w, w.eps_slab(0), precision="fp64")
    with pytest.raises(apf.APFError) as ei:
        s64.set_krylov(2)
    assert ei.value.code == apf.APF_EINVAL


@pytest.mark.parametrize("planes,butterfly", [(3, False), (2, True), (3, True)])
def test_elimination_options_against_golden(planes, butterfly):
    """The elimination options (bf16x6 products, the symmetric random
    butterfly transform of the slab blocks) change only the approximate
    factorization: after refinement S and grad f match the stored oracle
    values on the 1024 x 240 grid at the mixed-mode tolerances."""
    import os
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_09257_gb300 import apf, build
    from paper_2306_09257_gb300 import workloads as W
    build.build_lib()
    ref = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mid_1024x240_seed0.npz"))
    w = W.MID
    s = apf.solver_for_workload(w, w.eps_slab(0), precision="mixed")
    s.set_elimination(planes, butterfly)
    S, f, g = s.solve_S_grad("splitter", [-2, -1, 0, 1, 2], 0.18)
    assert np.linalg.norm(S - ref["S"]) / np.linalg.norm(ref["S"]) <= 1e-6
    assert np.linalg.norm(g - ref["grad"]) / np.linalg.norm(ref["grad"]) <= 1e-5
    assert s.stats()["residual"] <= 1e-10
