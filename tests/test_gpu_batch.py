"""Several designs in one call (apf_solve_S_grad_batch): every launch of the
mixed elimination, sweeps and gradient serves all designs of the batch.  Each
design's results must match the oracle, the stored oracle values, and the
same design solved alone."""
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


@pytest.fixture(scope="module")
def apf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_09257_gb300 import apf as A, build
    build.build_lib()
    A.load_library()
    return A


def solvers(apf, w, eps_list, prec):
    return [apf.solver_for_workload(w, e, precision=prec) for e in eps_list]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_matches_oracle_tiny(apf, prec):
    w = W.TINY
    seeds = [0, 1, 2]
    eps = [w.eps_slab(sd) for sd in seeds]
    sv = solvers(apf, w, eps, prec)
    S, f, g = apf.solve_S_grad_batch(sv, "splitter", ORDERS, 0.18)
    ts, tg = TOL[prec]
    for b, sd in enumerate(seeds):
        sol, f_ref, _, g_ref = O.f_and_grad(O.problem_from_workload(w, eps[b]), "splitter", ORDERS, 0.18)
        close(S[b], sol.S, ts)
        close(g[b], g_ref, tg)
        assert abs(f[b] - f_ref) <= 10 * ts * abs(f_ref)


def test_batch_mid_against_golden_and_single(apf):
    """1024 x 240, four designs (seed 0 first): design 0 against the stored
    oracle values; every design against the same design solved alone (the
    batch shares the launches, so tile shapes and therefore rounding may
    differ slightly; refinement brings both to the same tolerance)."""
    import torch
    ref = np.load(os.path.join(HERE, "golden", "mid_1024x240_seed0.npz"))
    w = W.MID
    eps = [w.eps_slab(sd) for sd in (0, 5, 6, 7)]
    sv = solvers(apf, w, eps, "mixed")
    S_d = [torch.empty((103, 103), dtype=torch.complex128, device="cuda") for _ in eps]
    g_d = [torch.empty((w.h, w.nx), dtype=torch.float64, device="cuda") for _ in eps]
    S, f, g = apf.solve_S_grad_batch(sv, "splitter", ORDERS, 0.18, out_S=S_d, out_grad=g_d)
    ts, tg = TOL["mixed"]
    close(S[0].cpu().numpy(), ref["S"], ts)
    close(g[0].cpu().numpy(), ref["grad"], tg)
    for b in range(len(eps)):
        one = apf.solver_for_workload(w, eps[b], precision="mixed")
        S1, f1, g1 = one.solve_S_grad("splitter", ORDERS, 0.18)
        close(S[b].cpu().numpy(), S1, 1e-8)
        close(g[b].cpu().numpy(), g1, 1e-5)
        assert sv[b].stats()["residual"] <= 1e-10
    # the contexts keep their fields: grad_from_gamma after the batch
    _, G = O.objective(S[1].cpu().numpy(), "splitter", sv[1].channels()[0], sv[1].channels()[1], ORDERS, 0.18)
    close(sv[1].grad_from_gamma(G), g[1].cpu().numpy(), 1e-12)


def test_batch_with_recompute_and_butterfly(apf):
    """Two designs with recomputed slab inverses: the batch's recomputations
    are shared launches too, and the results equal the stored case bit for
    bit."""
    w = W.MID
    eps = [w.eps_slab(sd) for sd in (8, 9)]
    a = solvers(apf, w, eps, "mixed")
    b = solvers(apf, w, eps, "mixed")
    for s in b:
        s.set_schur_storage(5)
    Sa, fa, ga = apf.solve_S_grad_batch(a, "splitter", ORDERS, 0.18)
    Sb, fb, gb = apf.solve_S_grad_batch(b, "splitter", ORDERS, 0.18)
    for i in range(2):
        assert np.array_equal(Sa[i], Sb[i]) and np.array_equal(ga[i], gb[i])


def test_batch_rejects_mismatched_contexts(apf):
    w = W.TINY
    s0 = apf.solver_for_workload(w, w.eps_slab(0), precision="mixed")
    s1 = apf.solver_for_workload(w, w.eps_slab(1), precision="mixed", m_in=[0, 1], m_out=[0, 1])
    with pytest.raises(apf.APFError) as e:
        apf.solve_S_grad_batch([s0, s1], "power", [0])
    assert e.value.code == apf.APF_EINVAL
    with pytest.raises(apf.APFError) as e:
        apf.solve_S_grad_batch([s0, s0], "power", [0])
    assert e.value.code == apf.APF_EINVAL


def test_threads_take_turns(apf):
    """Four host threads, each with its own context and stream, solving 1024 x
    240 designs at once: the library runs one solve at a time on the GPU
    (the others wait on the host), and each design's S and gradient are
    bit-identical to the same design solved alone."""
    import threading

    import torch
    w = W.MID
    seeds = [0, 1, 2, 3]
    eps = [w.eps_slab(sd) for sd in seeds]
    sv = solvers(apf, w, eps, "mixed")
    alone = [s.solve_S_grad("splitter", ORDERS, 0.18) for s in sv]
    L = apf.load_library()
    L.apf_debug_inflight_peak.argtypes = [apf.ctypes.c_int]
    L.apf_debug_inflight_peak(1)
    out, errs = [None] * len(sv), []

    def worker(b):
        try:
            with torch.cuda.stream(torch.cuda.Stream()):
                for _ in range(2):
                    out[b] = sv[b].solve_S_grad("splitter", ORDERS, 0.18)
        except BaseException as e:  # noqa: BLE001
            errs.append(e)
    ths = [threading.Thread(target=worker, args=(b,)) for b in range(len(sv))]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    assert not errs, errs
    peak = L.apf_debug_inflight_peak(0)
    assert peak == 1, peak
    for b in range(len(sv)):
        assert np.array_equal(out[b][0], alone[b][0])
        assert np.array_equal(out[b][2], alone[b][2])
        assert out[b][1] == alone[b][1]
