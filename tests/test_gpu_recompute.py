"""Recomputation of the slab Schur blocks (apf_set_schur_storage): keeping
one segment of packed inverses plus float32 checkpoints must give results
bit-identical to storing all h inverses (the recomputation repeats the same
deterministic kernels on the same inputs), and must match the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2306_09257_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ORDERS = [-2, -1, 0, 1, 2]


@pytest.fixture(scope="module")
def apf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_09257_gb300 import apf as A, build
    build.build_lib()
    A.load_library()
    return A


def run(apf, w, eps, seg, method="apf", krylov=0, tol=1e-10):
    s = apf.solver_for_workload(w, eps, precision="mixed")
    s.set_refinement(tol, 40)
    if krylov:
        s.set_krylov(krylov)
    s.set_schur_storage(seg)
    fn = s.solve_S_grad if method == "apf" else s.solve_S_grad_adjoint
    out = [fn("splitter", ORDERS, 0.18) for _ in range(2)]  # the second replays the captured graphs
    st = s.stats()
    s.close()
    return out, st


@pytest.mark.parametrize("seg", [1, 2, 4, 5])
def test_recompute_is_bit_identical_tiny(apf, seg):
    w = W.TINY
    eps = w.eps_slab(1)
    (a, _), st_a = run(apf, w, eps, 0)
    (b1, b2), st_b = run(apf, w, eps, seg)
    for b in (b1, b2):
        assert np.array_equal(a[0], b[0]) and a[1] == b[1] and np.array_equal(a[2], b[2])
    assert st_b["refine_iters"] == st_a["refine_iters"]
    assert st_b["workspace_bytes"] < st_a["workspace_bytes"]


@pytest.mark.parametrize("seg,method,krylov", [(5, "apf", 0), (3, "adjoint", 0), (4, "apf", 3)])
def test_recompute_is_bit_identical_mid(apf, seg, method, krylov):
    """1024 x 240 (h = 12, so a ragged last segment for seg 5), also through the
    conventional adjoint method's two passes and the GMRES refinement."""
    w = W.MID
    eps = w.eps_slab(2)
    (a, _), _ = run(apf, w, eps, 0, method, krylov)
    (b1, b2), _ = run(apf, w, eps, seg, method, krylov)
    for b in (b1, b2):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])


def test_recompute_matches_oracle(apf):
    w = W.TINY
    eps = w.eps_slab(6)
    sol, f_ref, _, g_ref = O.f_and_grad(O.problem_from_workload(w, eps), "splitter", ORDERS, 0.18)
    (r, _), _ = run(apf, w, eps, 2)
    S, f, g = r
    assert np.linalg.norm(S - sol.S) / np.linalg.norm(sol.S) <= 1e-6
    assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) <= 1e-5


def test_schur_storage_arguments(apf):
    s = apf.Solver(0, "fp64")
    with pytest.raises(apf.APFError) as e:
        s.set_schur_storage(2)
    assert e.value.code == apf.APF_EINVAL
    s.set_schur_storage(0)
    m = apf.Solver(0, "mixed")
    with pytest.raises(apf.APFError):
        m.set_schur_storage(-1)


def test_batch_recompute_is_bit_identical(apf):
    """Three 1024 x 240 designs in one batched call: recomputing the slab
    inverses in segments of 5 rows (ragged last segment, h = 12) gives the
    same bits as storing them, design by design."""
    w = W.MID
    eps = [w.eps_slab(sd) for sd in (3, 4, 5)]

    def batch(seg):
        sv = []
        for e in eps:
            s = apf.Solver(0, "mixed")
            s.set_grid(w.nx, w.ny, w.npml, w.npml, w.lambda_px)
            s.set_eps(e, w.eps_sub, w.eps_clad, j0=w.j0)
            s.set_schur_storage(seg)
            s.set_channels(None, None)
            s.set_refinement(1e-10, 40)
            sv.append(s)
        out = apf.solve_S_grad_batch(sv, "splitter", ORDERS, 0.18)
        ws = [s.stats()["workspace_bytes"] for s in sv]
        for s in sv:
            s.close()
        return out, ws

    (Sa, fa, ga), wa = batch(0)
    (Sb, fb, gb), wb = batch(5)
    for d in range(len(eps)):
        assert np.array_equal(Sa[d], Sb[d]) and fa[d] == fb[d] and np.array_equal(ga[d], gb[d])
        assert wb[d] < wa[d]
