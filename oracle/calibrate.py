"""Run the FP64 oracle to convergence on the benchmark workload and record
its Jacobi-PCG iteration count (used to scale the oracle's bounded timing
sample to one full solve).  Calls only the oracle; writes
oracle/iters_globular257.json.  Takes several minutes on one core.

    python -m oracle.calibrate
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import pb_inputs  # noqa: E402
from oracle import oracle as orc  # noqa: E402


def main():
    atoms = pb_inputs.globular_molecule(2000, seed=2)
    g = orc.place_grid(atoms, 257, 1.5)
    t0 = time.time()
    r = orc.solve_problem(atoms, g, eps_in=2.0, eps_out=80.0, ionic_strength_M=0.145,
                          bc=orc.BC_ZERO, rtol=1e-8, with_energy=False)
    out = {"workload": "globular 2000 atoms seed 2, 257^3, fill 1.5, eps 2/80, 0.145 M, zero BC",
           "rtol": 1e-8, "iters": int(r["iters"]), "true_rel_res": float(r["relres"]),
           "converged": bool(r["converged"]), "seconds": time.time() - t0,
           "n_cross": int(len(r["cross"]["ids"])), "h": g.h}
    with open(os.path.join(HERE, "iters_globular257.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(out)


if __name__ == "__main__":
    main()
