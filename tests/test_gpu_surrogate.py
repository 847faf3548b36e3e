"""Surrogate kernels against the float64 CPU reference, and what the trained
surrogate gains in the line search."""
import numpy as np
import pytest

from oracle import surrogate_ref as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_09257_gb300 import apf, build, surrogate
    build.build_lib()
    apf.load_library()
    return torch, surrogate


SHP = dict(in_ch=3, width=8, modes=16, layers=3, n_out=5)


def test_forward_and_gradients_match_reference(env):
    torch, SG = env
    n, B = 128, 6
    sno = SG.Surrogate(n=n, max_batch=16, seed=3, **SHP)
    p = SG.init_params(3, SHP["in_ch"], SHP["width"], SHP["modes"], SHP["layers"], SHP["n_out"])
    p = (p * 3.0).astype(np.float32)  # larger weights: a non-trivial network
    sno.set_params(p)
    rng = np.random.default_rng(0)
    x = rng.uniform(1.0, 2.25, size=(B, SHP["in_ch"], n)).astype(np.float32)
    t = rng.uniform(0, 0.5, size=(B, SHP["n_out"])).astype(np.float32)
    y = sno.forward(x).cpu().numpy()
    loss_ref, g_ref, y_ref = R.loss_and_grads(p, x.astype(np.float64), t.astype(np.float64), **SHP)
    assert np.linalg.norm(y - y_ref) / np.linalg.norm(y_ref) < 1e-4
    g, loss = sno.gradients(x, t)
    assert abs(loss - loss_ref) < 1e-4 * abs(loss_ref)
    off = 0
    for name, shape in SG.param_layout(SHP["in_ch"], SHP["width"], SHP["modes"], SHP["layers"], SHP["n_out"]):
        k = int(np.prod(shape))
        a, b = g[off:off + k], g_ref[off:off + k]
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b) + 1e-7, name
        off += k


def test_training_reduces_loss(env):
    torch, SG = env
    n = 128
    sno = SG.Surrogate(n=n, max_batch=64, seed=1, **SHP)
    rng = np.random.default_rng(1)
    x = rng.uniform(1.0, 2.25, size=(64, SHP["in_ch"], n)).astype(np.float32)
    # a smooth target that depends on the Fourier content of the input
    t = np.stack([np.abs(np.fft.rfft(x[:, 0], axis=-1)[:, k]) / n for k in range(5)], 1).astype(np.float32)
    l0 = sno.train_step(x, t, 1e-3)
    for _ in range(200):
        l1 = sno.train_step(x, t, 1e-3)
    assert l1 < 0.2 * l0


def test_trained_surrogate_in_the_line_search(env):
    """Train on exact efficiencies of 1024 x 240 designs, then compare the
    screened line search with plain backtracking from the same start: the
    surrogate must beat the mean predictor on held-out designs, and the
    screened search must need fewer exact solves per accepted step."""
    torch, SG = env
    from paper_2306_09257_gb300 import apf, optim, workloads as W
    w = W.MID
    X, T, secs = SG.generate(w, range(10_000, 10_640), batch=16)
    sno = SG.Surrogate(n=w.nx, in_ch=w.h, width=48, modes=64, layers=4, n_out=5, max_batch=128, seed=0)
    tr, te = slice(0, 576), slice(576, 640)
    SG.train(sno, X[tr], T[tr], epochs=40, batch=64, lr=2e-3)
    pred = sno.forward(X[te])
    mse = float(((pred - T[te]) ** 2).mean())
    base = float(((T[tr].mean(0, keepdim=True) - T[te]) ** 2).mean())
    print(f"data {secs:.1f} s, held-out mse {mse:.3e} vs mean predictor {base:.3e}")
    assert mse < 0.7 * base
    eps0 = np.clip(w.eps_slab(123), 1.0, 2.25)
    s = apf.solver_for_workload(w, eps0, precision="mixed")
    _, h_plain = optim.optimize(s, eps0, w.eps_sub, w.eps_clad, w.j0, "splitter", [-2, -1, 0, 1, 2], 0.18, iters=6)
    _, h_scr = optim.optimize_screened(s, sno, eps0, w.eps_sub, w.eps_clad, w.j0, [-2, -1, 0, 1, 2], 0.18, iters=6)
    per_plain = h_plain.evals / max(1, len(h_plain.f) - 1)
    per_scr = h_scr.evals / max(1, len(h_scr.f) - 1)
    print(f"plain: f {h_plain.f[0]:.4f} -> {h_plain.f[-1]:.4f}, {per_plain:.2f} solves/step, "
          f"{h_plain.iters_per_second:.2f} it/s; screened: f -> {h_scr.f[-1]:.4f}, {per_scr:.2f} solves/step, "
          f"{h_scr.iters_per_second:.2f} it/s")
    assert h_scr.f[-1] < h_scr.f[0]
    # the gain: a larger decrease of f per exact solve than plain backtracking
    gain_plain = (h_plain.f[0] - h_plain.f[-1]) / h_plain.evals
    gain_scr = (h_scr.f[0] - h_scr.f[-1]) / h_scr.evals
    print(f"decrease of f per exact solve: plain {gain_plain:.4f}, screened {gain_scr:.4f}")
    assert gain_scr > gain_plain
