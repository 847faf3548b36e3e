"""Seeded synthetic workloads: grid shapes and permittivity maps.

This module holds only input generation (grid sizes, random numbers, the
filtered-threshold permittivity recipe).  It contains none of the method's
arithmetic, so both the CPU oracle and the CUDA path may import it.

The paper's metasurface (Sec. 3: periodic ridges on a substrate, 20-pixel
PMLs in the non-periodic direction, many plane-wave input angles) is stood in
for by five synthetic workloads.  The x axis here is the periodic axis
(the paper's y), and the PMLs sit at both ends of the y axis (the paper's z).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    """One grid/slab configuration (all lengths in pixels)."""

    name: str
    nx: int            # period, pixels (periodic x)
    ny: int            # rows including both PMLs
    npml: int          # PML rows at each y end
    lambda_px: float   # vacuum wavelength in pixels
    h: int             # design-slab rows
    eps_sub: float     # substrate (bottom) permittivity
    eps_clad: float    # cladding (top) permittivity
    eps_kind: str      # "iid" (uniform in [lo, hi]) or "filtered"
    eps_lo: float = 1.0
    eps_hi: float = 4.0

    @property
    def j0(self) -> int:
        """First slab row: the slab is centred between the two PMLs."""
        return self.npml + (self.ny - 2 * self.npml - self.h) // 2

    def eps_slab(self, seed: int) -> np.ndarray:
        """Slab permittivity, shape (h, nx), float64, row-major [row][x]."""
        if self.eps_kind == "iid":
            return iid_eps(self.h, self.nx, seed, self.eps_lo, self.eps_hi)
        return filtered_threshold_eps(self.h, self.nx, seed)


# Tiny: iid eps in [1, 4], 9 channels.
TINY = Workload("tiny_64x100", 64, 100, 20, 16.0, 6, 2.25, 1.0, "iid", 1.0, 4.0)
# Mid: filtered-threshold eps, 103 channels.
MID = Workload("mid_1024x240", 1024, 240, 30, 20.0, 12, 2.25, 1.0, "filtered")
# Precision study size: 343 channels.
LARGE = Workload("large_4096x260", 4096, 260, 30, 24.0, 16, 2.25, 1.0, "filtered")
# Differentiation study size: 513 channels.
XLARGE = Workload("xlarge_8192x280", 8192, 280, 30, 32.0, 20, 2.25, 1.0, "filtered")

WORKLOADS = {w.name: w for w in (TINY, MID, LARGE, XLARGE)}


def small_workload(nx: int, ny: int, npml: int, lambda_px: float, h: int,
                   eps_sub: float = 2.25, eps_clad: float = 1.0,
                   kind: str = "iid") -> Workload:
    """A custom small case (used for ragged / edge-case tests)."""
    return Workload(f"custom_{nx}x{ny}_h{h}", nx, ny, npml, lambda_px, h,
                    eps_sub, eps_clad, kind)


def iid_eps(h: int, nx: int, seed: int, lo: float = 1.0, hi: float = 4.0) -> np.ndarray:
    """Independent uniform permittivity per slab pixel."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(h, nx)).astype(np.float64)


def filtered_threshold_eps(h: int, nx: int, seed: int, sigma: float = 3.0,
                           ramp_px: int = 2, eps_min: float = 1.0,
                           contrast: float = 1.25) -> np.ndarray:
    """Binary-like metasurface pattern: uniform noise, Gaussian filter
    (sigma px; periodic in x, mirrored in y), threshold at 0.5, then a
    ramp_px-wide box filter so edges ramp linearly; eps = eps_min + contrast*rho.
    """
    from scipy import ndimage

    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, 1.0, size=(h, nx))
    g = ndimage.gaussian_filter(u, sigma=sigma, mode=("reflect", "wrap"))
    b = (g > 0.5).astype(np.float64)
    rho = ndimage.uniform_filter(b, size=ramp_px, mode=("reflect", "wrap"))
    return (eps_min + contrast * rho).astype(np.float64)


def ridge_edges(nx: int, n_ridges: int, seed: int, mirror: bool = True, min_gap: float = 2.0) -> np.ndarray:
    """Seeded ridge edge positions (pixels, measured from the mirror plane x = nx/2).

    The paper's metasurface (Sec. 3) is parametrized by the two edge positions
    of each ridge; with mirror symmetry only the ridges of one half period are
    free.  Returns 2 n_ridges sorted positions t_0 < t_1 < ... in
    [-nx/2, 0] (mirror) or [-nx/2, nx/2] (no mirror); ridge i spans
    [t_{2i}, t_{2i+1}].  Neighbouring edges (ridge widths and gaps) are at least
    `min_gap` apart, as are the outermost edges from the interval ends, so the
    mirrored and the periodic neighbours never overlap.
    """
    lo, hi = -nx / 2.0, (0.0 if mirror else nx / 2.0)
    n = 2 * n_ridges
    free = (hi - lo) - (n + 1) * min_gap
    if free <= 0:
        raise ValueError("too many ridges for the interval and gap")
    u = np.sort(np.random.default_rng(seed).uniform(0.0, free, n))
    return lo + min_gap * (np.arange(n) + 1) + u


def ridge_count(w: "Workload") -> int:
    """Ridges per half period for a workload: one ridge per ~0.64 wavelength,
    the paper's 80-ridge, 25.5-wavelength beam splitter (Sec. 3) scaled to the
    grid's period."""
    return max(1, int(round(w.nx / (2 * 0.64 * w.lambda_px))))
