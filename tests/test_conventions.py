"""Host-side conventions that need no GPU."""
import numpy as np
import torch

import oracle as O


def test_torch_complex_grad_is_twice_conj_wirtinger():
    """The autograd wrapper turns torch's dL/dS into the paper's Gamma = df/dS
    (Wirtinger, Eq. 1) as conj(g)/2; check that convention on Eq. (5)."""
    rng = np.random.default_rng(1)
    S = rng.normal(size=(5, 5)) + 1j * rng.normal(size=(5, 5))
    m = np.arange(-2, 3)
    f, G = O.objective(S, "splitter", m, m, [-1, 0, 1], 0.2)
    St = torch.tensor(S, requires_grad=True)
    p = St.real ** 2 + St.imag ** 2
    mask = torch.tensor(np.abs(m[:, None] - m[None, :]) <= 1)
    loss = ((p[mask] - 0.2) ** 2).sum()
    loss.backward()
    assert abs(loss.item() - f) < 1e-12
    assert np.allclose(np.conj(St.grad.numpy()) / 2, G, atol=1e-12)


def test_relative_order_mask_matches_oracle_pairs():
    from paper_2306_09257_gb300 import autograd as AG
    m_in, m_out = np.array([-2, 0, 1, 3]), np.array([-1, 0, 1, 2])
    mask = AG.relative_order_mask(m_in, m_out, [-1, 1]).numpy()
    pairs = sorted(O.relative_pairs(m_in, m_out, [-1, 1]))
    assert sorted(zip(*np.nonzero(mask))) == pairs
