"""Write oracle reference values for the GPU parity tests at sizes where the
oracle takes too long to run inside a test.  Calls only ``oracle/`` (and the
seeded input generators); never the CUDA path.

    python tests/golden/make_golden.py

mid_1024x240_seed0.npz: S (103 x 103) and df/deps (12 x 1024) of the
beam-splitter objective (Eq. 5; relative orders -2..2, target 0.18) for the
1024 x 240 workload, slab seed 0, plus the orders and f.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2306_09257_gb300 import workloads as W  # noqa: E402


def main():
    w = W.MID
    seed = 0
    eps = w.eps_slab(seed)
    pb = O.problem_from_workload(w, eps)
    t = time.time()
    sol, f, G, g = O.f_and_grad(pb, "splitter", [-2, -1, 0, 1, 2], 0.18)
    print(f"oracle {w.name} seed {seed}: {time.time() - t:.1f} s, f = {f:.12g}")
    np.savez_compressed(os.path.join(HERE, f"{w.name}_seed{seed}.npz"), S=sol.S, grad=g, f=f,
                        m_in=pb.inputs(), m_out=pb.outputs(), eps=eps)


if __name__ == "__main__":
    main()
