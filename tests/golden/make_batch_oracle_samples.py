"""Write tests/golden/batch_oracle_samples.txt: the CPU oracle's solutions of the
64-instance batched workload (m in {255, 511, 1023, 2047}, s in {64, 128, 256},
ETR3 / GBDF3 / GAM4, fde_inputs.config_batch), reduced to what a test can compare
against at full size: for every instance with m >= 1023 and for instances 0-7, the
2-norm and max-norm of the solution, its values at 128 seeded positions and its
inner products with 8 seeded normal vectors (fde_inputs.check_sample).

The solutions are the oracle's FP64 Strang-preconditioned flexible GMRES(20)
(oracle.solve_strang_gmres, Sec. 3.2 with the dense DFT along time and one LAPACK
LU per frequency block) to a true relative residual of 1e-11 (the oracle's FP64 floor
is 2e-13 - 6e-12 at m = 2047, so a tighter tolerance would not terminate); the file
records the residual each reached (under the oracle's own Kronecker matvec).  Four
instances whose floor lies above 1e-11 (GAM4 at m = 2047, s = 256, alpha 1.76 and
1.85; ETR3 at m = 2047, s = 64, alpha 1.70 and 1.71) stop at maxit = 1500 with their
reached residual, 1.0e-11 to 2.1e-11, recorded as "converged 0".  Only oracle/ and
the input generators are used.  A full run takes about an hour on 8 cores:

    python tests/golden/make_batch_oracle_samples.py [--workers 4]
"""
from __future__ import annotations

import argparse
import os
import sys
import time
from concurrent.futures import ProcessPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch_oracle_samples.txt")


def selected():
    import fde_inputs as fi
    probs = fi.config_batch()
    return [i for i, p in enumerate(probs) if p.m >= 1023 or i < 8]


def solve(i: int):
    import numpy as np

    import fde_inputs as fi
    import oracle as O
    prob = fi.config_batch()[i]
    t0 = time.time()
    x, its, ok, _ = O.solve_strang_gmres(prob, side="right", tol=1e-11, maxit=1500)
    J = O.j_of(prob)
    b = O.reduced_rhs(prob, J=J)
    res = float(np.linalg.norm(b - O.matvec(prob, x, J=J)) / np.linalg.norm(b))
    idx, probes = fi.check_sample(prob.n, fi.instance_seed(i))
    lines = [f"instance {i} m {prob.m} s {prob.s} scheme {prob.family}{prob.mu} its {its} converged {int(ok)} "
             f"residual {res:.3e} norm2 {np.linalg.norm(x):.17e} norminf {np.abs(x).max():.17e}"]
    lines.append("proj " + " ".join(f"{v:.17e}" for v in probes @ x))
    for k in idx:
        lines.append(f"x {int(k)} {x[k]:.17e}")
    return i, lines, time.time() - t0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=4)
    args = ap.parse_args()
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "2")
    import fde_inputs as fi
    probs = fi.config_batch()
    todo = sorted(selected(), key=lambda i: -probs[i].m * probs[i].s)  # largest first
    done = {}
    with ProcessPoolExecutor(args.workers) as ex:
        for i, lines, dt in ex.map(solve, todo):
            done[i] = lines
            print(f"instance {i}: {dt:.0f} s, {lines[0]}", flush=True)
    with open(OUT, "w") as f:
        f.write("# CPU-oracle solutions of the 64-instance batched workload (fde_inputs.config_batch),\n"
                "# sampled: written by tests/golden/make_batch_oracle_samples.py (oracle/ only).\n"
                "# Per instance: a header line, 8 probe inner products, then 'x index value' lines.\n")
        for i in sorted(done):
            f.write("\n".join(done[i]) + "\n")


if __name__ == "__main__":
    main()
