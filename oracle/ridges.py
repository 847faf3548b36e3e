"""Ridge edge-position parametrization (CPU oracle; test infrastructure only).

The paper's beam splitter (Sec. 3, Eq. 5) is parametrized by the edge
positions p = {y_1, ..., y_N} of ridges in half a period, with the other half
fixed by mirror symmetry {y_{N+1}, ..., y_{2N}} = -{y_N, ..., y_1}; without
mirror symmetry (Supplement Sec. 7) all 2N edges are free.  The paper does not
state how an edge that falls inside a pixel is discretized.  Reading used here:
a pixel's permittivity is linear in the length of it that ridges cover,

    eps_x = eps_bg + (eps_ridge - eps_bg) * sum_ridges |[a, b] & [x - nx/2, x + 1 - nx/2)|,

with positions t measured from the mirror plane x = nx/2, ridges [t_{2i}, t_{2i+1}]
and, with mirror symmetry, their images [-t_{2i+1}, -t_{2i}].  Every slab row has
the same profile (the ridges span the slab height).  d eps_x / d t_k is then
+-(eps_ridge - eps_bg) at the pixel holding the edge (minus for a ridge's left
edge, plus for its right edge) and at the pixel holding its mirror image, zero
elsewhere: dA/dp_k has rank h (the column of slab pixels under the edge), the
r_k > 1 case of Eq. 2.  At an edge that sits exactly on a pixel boundary the
derivative taken is the one for increasing t: the edge moves into the pixel to
its right, floor(t + nx/2), and its mirror image (at -t, moving left) into the
pixel to the image's left, ceil(nx/2 - t) - 1 (both periodic).

The chain rule df/dt_k = sum_{j,x} (df/deps_{j,x}) (d eps_x / d t_k) is written
out as a dense Jacobian product.
"""
from __future__ import annotations

import math

import numpy as np


def ridge_intervals(edges, mirror: bool):
    """[(a, b), ...] for the ridges of the edge list, mirror images appended."""
    e = [float(v) for v in edges]
    if len(e) % 2:
        raise ValueError("edge count must be even")
    iv = [(e[2 * i], e[2 * i + 1]) for i in range(len(e) // 2)]
    if mirror:
        iv += [(-b, -a) for (a, b) in iv]
    return iv


def fill_fraction(nx: int, edges, mirror: bool) -> np.ndarray:
    """Covered length of each pixel [x, x+1) (positions shifted by nx/2)."""
    fill = np.zeros(nx)
    c = nx / 2.0
    for (a, b) in ridge_intervals(edges, mirror):
        for x in range(nx):
            lo, hi = x - c, x + 1 - c
            fill[x] += max(0.0, min(b, hi) - max(a, lo))
    return fill


def eps_from_edges(nx: int, h: int, edges, mirror: bool, eps_ridge: float, eps_bg: float) -> np.ndarray:
    """Slab permittivity (h x nx) of the ridge pattern."""
    row = eps_bg + (eps_ridge - eps_bg) * fill_fraction(nx, edges, mirror)
    return np.tile(row, (h, 1))


def edge_pixel(nx: int, t: float) -> int:
    """Pixel that an edge at t enters as t increases (periodic)."""
    return int(math.floor(t + nx / 2.0)) % nx


def image_pixel(nx: int, t: float) -> int:
    """Pixel that the mirror image (at -t) of an edge at t enters as t
    increases: the image moves left (periodic)."""
    return (int(math.ceil(nx / 2.0 - t)) - 1) % nx


def deps_dedges(nx: int, edges, mirror: bool, eps_ridge: float, eps_bg: float) -> np.ndarray:
    """Jacobian J[k, x] = d eps_x / d t_k of one slab row."""
    e = [float(v) for v in edges]
    d = eps_ridge - eps_bg
    J = np.zeros((len(e), nx))
    for k, t in enumerate(e):
        sign = -1.0 if k % 2 == 0 else 1.0  # left edge of its ridge: covering shrinks as t grows
        J[k, edge_pixel(nx, t)] += sign * d
        if mirror:
            # the image edge sits at -t and moves the opposite way; it bounds
            # the image ridge on the other side, so the sign is the same
            J[k, image_pixel(nx, t)] += sign * d
    return J


def grad_edges(grad_eps: np.ndarray, nx: int, edges, mirror: bool, eps_ridge: float, eps_bg: float) -> np.ndarray:
    """df/dt = J (sum over slab rows of df/deps)."""
    col = np.asarray(grad_eps, dtype=np.float64).reshape(-1, nx).sum(axis=0)
    return deps_dedges(nx, edges, mirror, eps_ridge, eps_bg) @ col
