"""CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does: it runs
entirely in the CUDA library and fails loudly when that library is missing.
"""
from .fdfd import (Problem, Solution, assemble_A, dS_deps_pixel, eps_map,
                   f_and_grad, grad_eps_adjoint, ky_nu, objective, plane_wave,
                   problem_from_workload, projection_matrix, propagating_orders,
                   reflection, relative_pairs, solve_reverse_S, solve_S,
                   source_matrix, stretch)
from .ridges import (deps_dedges, edge_pixel, eps_from_edges, fill_fraction,
                     grad_edges, image_pixel, ridge_intervals)

__all__ = [
    "Problem", "Solution", "assemble_A", "dS_deps_pixel", "eps_map", "f_and_grad",
    "grad_eps_adjoint", "ky_nu", "objective", "plane_wave", "problem_from_workload",
    "projection_matrix", "propagating_orders", "reflection", "relative_pairs",
    "solve_reverse_S", "solve_S", "source_matrix", "stretch",
    "deps_dedges", "edge_pixel", "eps_from_edges", "fill_fraction", "grad_edges", "image_pixel", "ridge_intervals",
]
