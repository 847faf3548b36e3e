"""Kernel-level GPU checks against plain PyTorch references of the same op:
the bf16-split complex tensor-core GEMM and the mixed recursive inversion."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2306_09257_gb300 import apf, build
    build.build_lib()
    L = apf.load_library()
    f = ctypes.c_void_p
    L.apf_debug_cgemm.argtypes = [f, ctypes.c_int, ctypes.c_int, ctypes.c_int] + [f] * 6 + [ctypes.c_int]
    L.apf_debug_inv32.argtypes = [f, ctypes.c_int, f, f, ctypes.c_int]
    return torch, apf, L


def planar(torch, z):
    return z.real.float().contiguous(), z.imag.float().contiguous()


# (m, n, k): aligned, ragged m/n/k, and sizes that take the wide-tile two-CTA
# cluster kernel (aligned, and ragged in m, n and k).
SHAPES = [(128, 256, 64), (200, 130, 96), (37, 300, 40), (1024, 2048, 512), (1000, 3000, 264)]
TOL = {1: 1.5e-2, 2: 1e-4, 3: 3e-5}  # 3 planes: limited by the tensor-core fp32 accumulation


@pytest.mark.parametrize("nsplit", [1, 2, 3])
@pytest.mark.parametrize("shape", SHAPES)
def test_tc_cgemm_against_torch(env, shape, nsplit):
    torch, apf, L = env
    m, n, k = shape
    g = torch.Generator(device="cuda").manual_seed(m * 7 + n + k)
    A = torch.randn(m, k, dtype=torch.complex128, device="cuda", generator=g)
    B = torch.randn(k, n, dtype=torch.complex128, device="cuda", generator=g)
    Ar, Ai = planar(torch, A)
    Br, Bi = planar(torch, B)
    Cr = torch.full((m, n), float("nan"), device="cuda")
    Ci = torch.full((m, n), float("nan"), device="cuda")
    s = apf.Solver(0, "mixed")
    rc = L.apf_debug_cgemm(s._h, m, n, k, Ar.data_ptr(), Ai.data_ptr(), Br.data_ptr(), Bi.data_ptr(),
                           Cr.data_ptr(), Ci.data_ptr(), nsplit)
    assert rc == 0, L.apf_last_error(s._h)
    # reference: the same fp32 operands, product in float64
    ref = (Ar.double() + 1j * Ai.double()) @ (Br.double() + 1j * Bi.double())
    got = Cr.double() + 1j * Ci.double()
    err = (torch.linalg.norm(got - ref) / torch.linalg.norm(ref)).item()
    assert err < TOL[nsplit], err


# leaf = block size + 1000 * leaf kernel variant (128 blocks: 0 in-CTA Schur
# recursion over 32 x 32 Gauss-Jordan leaves, 3 single-level Gauss-Jordan);
# + 100000: through the symmetric random butterfly transform
@pytest.mark.parametrize("n,leaf", [(64, 64), (256, 64), (128, 128), (512, 128), (1024, 128), (1024, 3128),
                                    (512, 100128), (2048, 100128)])
def test_mixed_recursive_inverse(env, n, leaf):
    """Inverse of a complex-symmetric matrix shaped like a slab Schur block
    (diagonal ~4 - k^2 eps, periodic -1 neighbours, a dense symmetric
    perturbation) against torch.linalg.inv in float64."""
    torch, apf, L = env
    g = torch.Generator(device="cpu").manual_seed(n)
    P = torch.randn(n, n, dtype=torch.complex128, generator=g) * (0.3 / n ** 0.5)
    X = P + P.T
    idx = torch.arange(n)
    X[idx, idx] += 3.6 + 0.2j
    X[idx, (idx + 1) % n] -= 1.0
    X[idx, (idx - 1) % n] -= 1.0
    X = X.cuda()
    s = apf.Solver(0, "mixed")
    s.set_grid(n, 8 + 2 * 4 + 4, 4, 4, 8.0)
    s.set_eps(np.full((1, n), 1.5), 2.25, 1.0)
    s.set_channels([0], [0])
    re, im = planar(torch, X)
    rc = L.apf_debug_inv32(s._h, n, re.data_ptr(), im.data_ptr(), leaf)
    assert rc == 0, L.apf_last_error(s._h)
    Xi = re.double() + 1j * im.double()
    ref = torch.linalg.inv(X)
    err = (torch.linalg.norm(Xi - ref) / torch.linalg.norm(ref)).item()
    assert err < 3e-4, err


def test_leaf128_falls_back_on_singular_leading_block(env):
    """A complex-symmetric 128 x 128 block whose leading 64 x 64 sub-block is
    zero but which is itself well conditioned: the recursive in-CTA inversion
    must detect its failure and recover through the fully pivoted
    Gauss-Jordan, with no singular-pivot error."""
    torch, apf, L = env
    n = 128
    g = torch.Generator(device="cpu").manual_seed(5)
    P = torch.randn(n, n, dtype=torch.complex128, generator=g) * 0.01
    X = torch.zeros(n, n, dtype=torch.complex128)
    X[:64, 64:] = torch.eye(64)
    X[64:, :64] = torch.eye(64)
    X = X + P + P.T
    X[:64, :64] = 0.0
    X = X.cuda()
    s = apf.Solver(0, "mixed")
    s.set_grid(n, 8 + 2 * 4 + 4, 4, 4, 8.0)
    s.set_eps(np.full((1, n), 1.5), 2.25, 1.0)
    s.set_channels([0], [0])
    re, im = planar(torch, X)
    rc = L.apf_debug_inv32(s._h, n, re.data_ptr(), im.data_ptr(), 128)
    assert rc == 0, L.apf_last_error(s._h)
    Xi = re.double() + 1j * im.double()
    ref = torch.linalg.inv(X)
    err = (torch.linalg.norm(Xi - ref) / torch.linalg.norm(ref)).item()
    assert err < 3e-4, err
