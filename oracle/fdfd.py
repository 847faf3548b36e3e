"""CPU oracle for the scattering matrix and its gradient (test infrastructure).

THIS IS TEST INFRASTRUCTURE, NOT A PRODUCT PATH.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.
It shares no code with the CUDA path: the finite-difference operator, the PML,
the channels, the sources and the gradient are all written out here again,
from their definitions, in float64 / complex128 NumPy + SciPy.

What it computes (paper, Sec. 2):
  * A: the discretised 2D TM operator  -lap - (w/c)^2 eps  (Sec. 2, the TM
    example after Eq. 1), on a grid periodic in x with graded PMLs at both y
    ends, in the complex-symmetric stretched-coordinate form (A = A^T; the
    paper notes dA/dp is symmetric by reciprocity).
  * B, C, D: input sources and output projections of plane-wave channels
    (Sec. 2, S = C A^-1 B - D and Fig. 1a).
  * S = C A^-1 B - D by factoring A once and solving the M_in forward problems
    one column at a time.
  * grad f by the conventional adjoint method, Eq. (S1): one adjoint solve per
    input with source C_m^adj = sum_n (df/dS_nm) C_n, then
    df/dp_k = -sum_m 2 Re( C_m^adj A^-1 (dA/dp_k) A^-1 B_m ), with p_k the
    permittivity of slab pixel k so dA/dp_k = -(k0 dx)^2 e_k e_k^T (Eq. 2 with
    U_k = e_k).  That is 2 M_in sparse solves: the brute force the paper's
    method replaces.
  * f and df/dS for the two objectives used here: a sum of channel powers and
    the beam-splitter figure of merit, Eq. (5), with the Wirtinger derivative
    printed after it.

Readings of points the paper leaves open (the CUDA path takes the same ones):
  * Axes: x periodic (Bloch wave number 0), PML along y.
  * Scale: A carries a factor dx^2, so the gradient is per unit eps with
    dA/deps_k = -(k0 dx)^2.
  * PML: s(y) = 1 + i alpha (d/L)^p with d the depth into the PML measured
    from the half-integer interface row, L the PML thickness in pixels and
    alpha = -(p+1) ln(R0) / (2 k0dx sqrt(eps_side) L) (normal-incidence round
    trip reflection R0).  Dirichlet walls at rows -1 and ny.
  * Channels: Fourier orders u_m(x) = exp(2 pi i m x/nx)/sqrt(nx), propagating
    iff 0 < (k0dx)^2 eps/4 - sin^2(pi m/nx) < 1; k_y = 2 asin(sqrt(that)),
    nu = sin(k_y).
  * Unit-flux normalisation: source B_a = -2i sqrt(nu_a) u_{m_a} on row j_s
    (first non-PML row), projection C_b = sqrt(nu_b) u_{m_b}^H on row j_o
    (last non-PML row); D = 0 for transmission, D = I for reflection measured
    on row j_s.
  * Objective orders are relative diffraction orders d = m_out - m_in.

Parity pins: see tests/test_oracle_pins.py (uniform-slab 1-D Thomas solve,
homogeneous-medium closed form, flux conservation, reciprocity, cyclic shift
and mirror invariants, finite differences and the midpoint-Taylor cubic
remainder of the paper's gradient validation).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ---------------------------------------------------------------------------
# Problem description
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    nx: int
    ny: int
    npml_bot: int
    npml_top: int
    lambda_px: float
    eps_slab: np.ndarray          # (h, nx) float64
    j0: int                       # first slab row
    eps_sub: float
    eps_clad: float
    R0: float = 1e-8
    power: float = 3.0
    m_in: Optional[np.ndarray] = None    # input orders (default: cladding-propagating)
    m_out: Optional[np.ndarray] = None   # output orders (default: cladding-propagating)

    @property
    def k(self) -> float:
        """k0 * dx."""
        return 2.0 * math.pi / self.lambda_px

    @property
    def h(self) -> int:
        return int(self.eps_slab.shape[0])

    @property
    def j_src(self) -> int:
        return self.npml_bot

    @property
    def j_out(self) -> int:
        return self.ny - self.npml_top - 1

    def inputs(self) -> np.ndarray:
        if self.m_in is not None:
            return np.asarray(self.m_in, dtype=np.int64)
        return propagating_orders(self.nx, self.k, self.eps_clad)

    def outputs(self) -> np.ndarray:
        if self.m_out is not None:
            return np.asarray(self.m_out, dtype=np.int64)
        return propagating_orders(self.nx, self.k, self.eps_clad)


def problem_from_workload(w, eps_slab: np.ndarray, **kw) -> Problem:
    return Problem(nx=w.nx, ny=w.ny, npml_bot=w.npml, npml_top=w.npml,
                   lambda_px=w.lambda_px, eps_slab=np.asarray(eps_slab, np.float64),
                   j0=w.j0, eps_sub=w.eps_sub, eps_clad=w.eps_clad, **kw)


# ---------------------------------------------------------------------------
# Channels: discrete dispersion of the 5-point stencil in a uniform medium
# ---------------------------------------------------------------------------
def dispersion_q(nx: int, k: float, eps: float, m) -> np.ndarray:
    """q = sin^2(k_y/2) for order m: from 2cos(k_y) = 2 + lambda_m - k^2 eps with
    lambda_m = 2 - 2cos(2 pi m/nx) the eigenvalue of the periodic -d^2/dx^2."""
    m = np.asarray(m, dtype=np.float64)
    return (k * k * eps) / 4.0 - np.sin(np.pi * m / nx) ** 2


def propagating_orders(nx: int, k: float, eps: float) -> np.ndarray:
    m = np.arange(-(nx // 2), nx - nx // 2)
    q = dispersion_q(nx, k, eps, m)
    return m[(q > 0.0) & (q < 1.0)].astype(np.int64)


def ky_nu(nx: int, k: float, eps: float, m):
    q = dispersion_q(nx, k, eps, m)
    if np.any(q <= 0.0) or np.any(q >= 1.0):
        raise ValueError("order not propagating in this medium")
    ky = 2.0 * np.arcsin(np.sqrt(q))
    return ky, np.sin(ky)


def plane_wave(nx: int, m: int) -> np.ndarray:
    x = np.arange(nx)
    return np.exp(2j * np.pi * m * x / nx) / math.sqrt(nx)


# ---------------------------------------------------------------------------
# Grid: PML stretch factors and the permittivity map
# ---------------------------------------------------------------------------
def stretch(y: float, pb: Problem) -> complex:
    """Complex coordinate stretch s(y) at integer or half-integer row y."""
    lo = pb.npml_bot - 0.5           # bottom PML / interior interface
    hi = pb.ny - pb.npml_top - 0.5   # interior / top PML interface
    if y < lo and pb.npml_bot > 0:
        L, d, eps = pb.npml_bot, lo - y, pb.eps_sub
    elif y > hi and pb.npml_top > 0:
        L, d, eps = pb.npml_top, y - hi, pb.eps_clad
    else:
        return 1.0 + 0.0j
    alpha = -(pb.power + 1.0) * math.log(pb.R0) / (2.0 * pb.k * math.sqrt(eps) * L)
    return 1.0 + 1j * alpha * (d / L) ** pb.power


def eps_map(pb: Problem) -> np.ndarray:
    e = np.empty((pb.ny, pb.nx), dtype=np.float64)
    e[: pb.j0, :] = pb.eps_sub
    e[pb.j0: pb.j0 + pb.h, :] = pb.eps_slab
    e[pb.j0 + pb.h:, :] = pb.eps_clad
    return e


def check_layout(pb: Problem) -> None:
    if not (pb.j_src < pb.j0 and pb.j0 + pb.h <= pb.j_out):
        raise ValueError("source row, slab and output row overlap")


# ---------------------------------------------------------------------------
# Operator A (complex symmetric), sources B, projections C
# ---------------------------------------------------------------------------
def assemble_A(pb: Problem, eps: Optional[np.ndarray] = None) -> sp.csc_matrix:
    """Row (j, x) -> index j*nx + x.  For unknown E at (x, j):
        s_j [ 2E - E(x-1) - E(x+1) - k^2 eps E ]
      + (1/s_{j+1/2} + 1/s_{j-1/2}) E - E(j+1)/s_{j+1/2} - E(j-1)/s_{j-1/2}
    which is -d2/dx2 - d/dy (1/s) d/dy - k^2 eps, multiplied through by s_j
    (stretched-coordinate PML in symmetric form), times dx^2."""
    nx, ny, k = pb.nx, pb.ny, pb.k
    if eps is None:
        eps = eps_map(pb)
    s_int = np.array([stretch(float(j), pb) for j in range(ny)])
    s_half = np.array([stretch(j - 0.5, pb) for j in range(ny + 1)])  # s at j-1/2
    rows, cols, vals = [], [], []
    idx = np.arange(nx)
    for j in range(ny):
        base = j * nx
        sj = s_int[j]
        up, dn = 1.0 / s_half[j + 1], 1.0 / s_half[j]
        diag = sj * (2.0 - k * k * eps[j]) + up + dn
        rows.append(base + idx); cols.append(base + idx); vals.append(diag.astype(complex))
        for dx in (-1, 1):
            rows.append(base + idx); cols.append(base + (idx + dx) % nx)
            vals.append(np.full(nx, -sj, dtype=complex))
        if j + 1 < ny:
            rows.append(base + idx); cols.append(base + nx + idx); vals.append(np.full(nx, -up, complex))
        if j - 1 >= 0:
            rows.append(base + idx); cols.append(base - nx + idx); vals.append(np.full(nx, -dn, complex))
    r = np.concatenate(rows); c = np.concatenate(cols); v = np.concatenate(vals)
    N = nx * ny
    return sp.coo_matrix((v, (r, c)), shape=(N, N)).tocsc()


def source_matrix(pb: Problem, orders, row: int, eps_side: float) -> np.ndarray:
    """Columns: unit-flux line sources -2i sqrt(nu) u_m on one row."""
    orders = np.asarray(orders)
    _, nu = ky_nu(pb.nx, pb.k, eps_side, orders)
    B = np.zeros((pb.nx * pb.ny, len(orders)), dtype=complex)
    for a, m in enumerate(orders):
        B[row * pb.nx:(row + 1) * pb.nx, a] = -2j * math.sqrt(nu[a]) * plane_wave(pb.nx, int(m))
    return B


def projection_matrix(pb: Problem, orders, row: int, eps_side: float) -> np.ndarray:
    """Rows: flux-normalised projections sqrt(nu) u_m^H on one row."""
    orders = np.asarray(orders)
    _, nu = ky_nu(pb.nx, pb.k, eps_side, orders)
    C = np.zeros((len(orders), pb.nx * pb.ny), dtype=complex)
    for b, m in enumerate(orders):
        C[b, row * pb.nx:(row + 1) * pb.nx] = math.sqrt(nu[b]) * np.conj(plane_wave(pb.nx, int(m)))
    return C


# ---------------------------------------------------------------------------
# S = C A^-1 B - D, one forward problem per input
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Solution:
    S: np.ndarray              # (M_out, M_in)
    X: np.ndarray              # A^-1 B, (N, M_in)
    lu: object
    B: np.ndarray
    C: np.ndarray
    pb: Problem


def solve_S(pb: Problem) -> Solution:
    check_layout(pb)
    A = assemble_A(pb)
    lu = spla.splu(A)
    m_in, m_out = pb.inputs(), pb.outputs()
    B = source_matrix(pb, m_in, pb.j_src, pb.eps_sub)
    C = projection_matrix(pb, m_out, pb.j_out, pb.eps_clad)
    X = np.empty_like(B)
    for a in range(B.shape[1]):
        X[:, a] = lu.solve(B[:, a])
    S = C @ X
    return Solution(S=S, X=X, lu=lu, B=B, C=C, pb=pb)


def reflection(sol: Solution, orders=None) -> np.ndarray:
    """r = C_ref A^-1 B - I on the source row (orders propagating in the
    substrate; defaults to all of them)."""
    pb = sol.pb
    if orders is None:
        orders = propagating_orders(pb.nx, pb.k, pb.eps_sub)
    Cr = projection_matrix(pb, orders, pb.j_src, pb.eps_sub)
    R = Cr @ sol.X
    m_in = pb.inputs()
    for a, m in enumerate(m_in):
        hit = np.nonzero(np.asarray(orders) == m)[0]
        if len(hit):
            R[hit[0], a] -= 1.0
    return R


def solve_reverse_S(pb: Problem) -> np.ndarray:
    """Transmission for waves incident from the cladding side: sources on row
    j_out (cladding), projections on row j_src (substrate).  Rows/cols are
    indexed by the orders of pb.inputs() (as outputs) and pb.outputs() (as
    inputs)."""
    A = assemble_A(pb)
    lu = spla.splu(A)
    B = source_matrix(pb, pb.outputs(), pb.j_out, pb.eps_clad)
    C = projection_matrix(pb, pb.inputs(), pb.j_src, pb.eps_sub)
    X = np.column_stack([lu.solve(B[:, a]) for a in range(B.shape[1])])
    return C @ X


# ---------------------------------------------------------------------------
# Objectives f(S) and their Wirtinger derivatives Gamma = df/dS
# ---------------------------------------------------------------------------
def relative_pairs(m_in, m_out, orders: Sequence[int]):
    """(b, a) index pairs with m_out[b] - m_in[a] in `orders` (terms whose
    output order is not in the output set are dropped)."""
    pos = {int(m): i for i, m in enumerate(m_out)}
    pairs = []
    for a, ma in enumerate(m_in):
        for d in orders:
            b = pos.get(int(ma) + int(d))
            if b is not None:
                pairs.append((b, a))
    return pairs


def objective(S: np.ndarray, kind: str, m_in, m_out, orders, target: float = 0.0):
    """kind 'power':    f = sum_{(b,a)} |S_ba|^2,             Gamma = S*
       kind 'splitter': f = sum_{(b,a)} (|S_ba|^2 - t)^2,      Gamma = 2(|S|^2 - t) S*
       (Eq. 5 and the derivative printed after it)."""
    G = np.zeros_like(S)
    f = 0.0
    for b, a in relative_pairs(m_in, m_out, orders):
        p = abs(S[b, a]) ** 2
        if kind == "power":
            f += p
            G[b, a] += np.conj(S[b, a])
        elif kind == "splitter":
            f += (p - target) ** 2
            G[b, a] += 2.0 * (p - target) * np.conj(S[b, a])
        else:
            raise ValueError(kind)
    return f, G


# ---------------------------------------------------------------------------
# Gradient: conventional adjoint method, Eq. (S1)
# ---------------------------------------------------------------------------
def grad_eps_adjoint(sol: Solution, Gamma: np.ndarray) -> np.ndarray:
    """df/deps for every slab pixel, shape (h, nx).

    For each input m: adjoint row vector C_m^adj = sum_n Gamma[n, m] C_n; the
    row C_m^adj A^-1 is obtained by solving A^T lam = (C_m^adj)^T.  Then
    df/deps_k = -sum_m 2 Re(lam_m[k] * dA_kk/deps_k * x_m[k]) with
    dA_kk/deps_k = -s_k (k0dx)^2 = -(k0dx)^2 in the slab."""
    pb = sol.pb
    k2 = pb.k ** 2
    sl = slice(pb.j0 * pb.nx, (pb.j0 + pb.h) * pb.nx)
    g = np.zeros(pb.h * pb.nx)
    for m in range(sol.B.shape[1]):
        cadj = Gamma[:, m] @ sol.C                       # row vector (N,)
        lam = sol.lu.solve(cadj, trans="T")              # A^T lam = cadj^T
        g += -2.0 * np.real(lam[sl] * (-k2) * sol.X[sl, m])
    return g.reshape(pb.h, pb.nx)


def dS_deps_pixel(sol: Solution, j: int, x: int) -> np.ndarray:
    """Brute-force dS/deps for one slab pixel from the definition
    dS = -C A^-1 (dA) A^-1 B (the identity stated before Eq. 2)."""
    pb = sol.pb
    kidx = (pb.j0 + j) * pb.nx + x
    CAinv = np.vstack([sol.lu.solve(sol.C[b], trans="T") for b in range(sol.C.shape[0])])
    return -(CAinv[:, kidx:kidx + 1] * (-pb.k ** 2)) @ sol.X[kidx:kidx + 1, :]


def f_and_grad(pb: Problem, kind: str, orders, target: float = 0.0):
    sol = solve_S(pb)
    f, G = objective(sol.S, kind, pb.inputs(), pb.outputs(), orders, target)
    return sol, f, G, grad_eps_adjoint(sol, G)
