"""Float64 CPU reference of the spectral-convolution surrogate network (test
infrastructure only; the paper has no learned component).

Same flat parameter layout as include/apf_surrogate.h.  Written with plain
torch CPU ops: the truncated DFT is torch.fft.rfft cut to the first M modes,
the synthesis is the real part of the sum over the kept modes with weights
1/n (mode 0) and 2/n, and gradients come from torch autograd in float64.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F


def unpack(p, in_ch, width, modes, layers, n_out, bf16_round=True):
    if bf16_round:
        p = torch.as_tensor(np.asarray(p, dtype=np.float32)).to(torch.bfloat16).to(torch.float64)
    else:
        p = torch.as_tensor(np.asarray(p, dtype=np.float64))
    shapes = [("W0", (width, in_ch)), ("b0", (width,)), ("Wr", (layers, width, width, modes)),
              ("Wi", (layers, width, width, modes)), ("P", (layers, width, width)), ("c", (layers, width)),
              ("Wh", (n_out, width)), ("bh", (n_out,))]
    out, o = {}, 0
    for name, shp in shapes:
        k = int(np.prod(shp))
        out[name] = p[o:o + k].reshape(shp).clone()
        o += k
    assert o == p.numel()
    return out, shapes


def forward(params: dict, x: torch.Tensor, modes: int) -> torch.Tensor:
    n = x.shape[-1]
    h = torch.einsum("oi,bix->box", params["W0"], x) + params["b0"][:, None]
    L = params["Wr"].shape[0]
    for l in range(L):
        Xh = torch.fft.rfft(h, dim=-1)[..., :modes]
        W = params["Wr"][l] + 1j * params["Wi"][l]
        Y = torch.einsum("iom,bim->bom", W, Xh)
        # real part of the zero-padded inverse DFT of the kept modes, written
        # out (irfft's backward assumes a Hermitian spectrum, which the
        # complex mixing does not keep for the imaginary part of mode 0)
        m = torch.arange(modes, dtype=torch.float64)[:, None]
        x = torch.arange(n, dtype=torch.float64)[None, :]
        wgt = torch.where(m == 0, 1.0 / n, 2.0 / n)
        E = wgt * torch.exp(2j * np.pi * m * x / n)
        z = torch.einsum("bom,mx->box", Y, E).real + torch.einsum("oi,bix->box", params["P"][l], h) \
            + params["c"][l][:, None]
        h = F.gelu(z) if l < L - 1 else z
    return h.mean(-1) @ params["Wh"].T + params["bh"]


def loss_and_grads(p, x, target, in_ch, width, modes, layers, n_out):
    """Mean squared error and its gradient w.r.t. the flat parameters (at
    the bf16-rounded weights), float64."""
    params, shapes = unpack(p, in_ch, width, modes, layers, n_out)
    for v in params.values():
        v.requires_grad_(True)
    xt = torch.as_tensor(np.asarray(x), dtype=torch.float64)
    tt = torch.as_tensor(np.asarray(target), dtype=torch.float64)
    out = forward(params, xt, modes)
    loss = ((out - tt) ** 2).mean()
    loss.backward()
    g = torch.cat([params[name].grad.reshape(-1) for name, _ in shapes])
    return float(loss.detach()), g.numpy(), out.detach().numpy()
