"""Writes tests/golden/poisson5d_full.txt: the FP64 oracle's relative L2 error against
the manufactured solution on the test set for the full 5-D Poisson configuration
(32,768 + 4,096 rows x 4,096 features, sigma = 3, weight 100).  The oracle is plain
single-threaded C (assembly, unblocked Householder QR, back substitution), so this
takes tens of minutes; the GPU full-size test reads the stored value.
``python tests/golden/make_poisson5d_full.py``."""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2602_10541_gb300 import workloads as wl  # noqa: E402


def main():
    oracle.build()
    w = wl.poisson5d()
    t0 = time.time()
    A_int = oracle.assemble(w.x_int, w.alpha, w.coef, w.W, w.b, w.scale)
    A_bc = oracle.assemble(w.x_bc, np.zeros((1, w.d), np.int32), [1.0], w.W, w.b, w.scale,
                           row_weight=w.lam_bc)
    f = oracle.problem_source(w.problem, w.x_int, w.params)
    g = oracle.problem_exact(w.problem, w.x_bc, w.params)
    beta = oracle.lstsq(np.vstack([A_int, A_bc]), np.concatenate([f, w.lam_bc * g]), mu=w.mu)
    u = oracle.eval_u(w.x_test, w.W, w.b, w.scale, beta)
    ue = oracle.problem_exact(w.problem, w.x_test, w.params)
    err = float(np.linalg.norm(u - ue) / np.linalg.norm(ue))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "poisson5d_full.txt")
    with open(out, "w") as fh:
        fh.write("# FP64 oracle, poisson5d at full size (32768 + 4096 rows x 4096 features): relative L2\n")
        fh.write("# error of u against the manufactured solution on the 5000-point test set.\n")
        fh.write(f"# written by tests/golden/make_poisson5d_full.py in {time.time() - t0:.0f} s\n")
        fh.write(f"oracle_rel_l2_vs_exact {err:.6e}\n")
    print(err)


if __name__ == "__main__":
    main()
