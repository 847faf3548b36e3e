"""GB300-native augmented-partial-factorization solver for 2D TM FDFD:
S = C A^-1 B - D and df/deps for every design pixel in one elimination.

Importing the package is light; the CUDA library is loaded by
``paper_2306_09257_gb300.apf`` on first use and fails loudly if missing.
"""
__all__ = ["workloads"]
