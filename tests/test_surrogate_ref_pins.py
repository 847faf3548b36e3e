"""Pins for the float64 surrogate reference: closed forms of its spectral
layer and finite differences of its gradient."""
import numpy as np
import torch

from oracle import surrogate_ref as R


def test_single_mode_passes_identity_mixing():
    """With W = identity on every kept mode, P = 0, c = 0, the spectral layer
    reproduces a band-limited input exactly (its modes are kept)."""
    n, M, C = 64, 8, 3
    x = np.arange(n)
    sig = np.cos(2 * np.pi * 3 * x / n + 0.4) + 0.2
    params = {"W0": torch.eye(C, dtype=torch.float64)[:, :1], "b0": torch.zeros(C, dtype=torch.float64),
              "Wr": torch.eye(C, dtype=torch.float64)[None, :, :, None].repeat(1, 1, 1, M),
              "Wi": torch.zeros(1, C, C, M, dtype=torch.float64), "P": torch.zeros(1, C, C, dtype=torch.float64),
              "c": torch.zeros(1, C, dtype=torch.float64), "Wh": torch.eye(C, dtype=torch.float64),
              "bh": torch.zeros(C, dtype=torch.float64)}
    xt = torch.tensor(sig[None, None, :])
    out = R.forward(params, xt, M)
    # single (last) layer has no activation: the pooled output is the mean of the input in channel 0
    assert abs(float(out[0, 0]) - sig.mean()) < 1e-12
    assert abs(float(out[0, 1])) < 1e-12


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    shp = dict(in_ch=2, width=4, modes=4, layers=2, n_out=3)
    n = 32
    from paper_2306_09257_gb300.surrogate import init_params
    p = init_params(1, shp["in_ch"], shp["width"], shp["modes"], shp["layers"], shp["n_out"])
    p = torch.tensor(p).to(torch.bfloat16).to(torch.float32).numpy()  # exactly representable
    x = rng.normal(size=(3, shp["in_ch"], n))
    t = rng.normal(size=(3, shp["n_out"]))
    loss, g, _ = R.loss_and_grads(p, x, t, **shp)
    pd = p.astype(np.float64)
    for k in rng.choice(p.size, 12, replace=False):
        h = 1e-6
        def f(v):
            q = pd.copy()
            q[k] = v
            params, _ = R.unpack(q, **shp, bf16_round=False)
            out = R.forward(params, torch.tensor(x), shp["modes"])
            return float(((out - torch.tensor(t)) ** 2).mean())
        fd = (f(pd[k] + h) - f(pd[k] - h)) / (2 * h)
        assert abs(fd - g[k]) < 1e-6 + 1e-5 * abs(g[k]), (k, fd, g[k])
