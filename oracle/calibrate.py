"""Run the FP64 oracle once, completely, on the benchmark workload (grid,
classification, crossing edges, coefficients, right-hand side, Jacobi-PCG to
a 1e-8 true residual, Coulomb terms and energies) and record its iteration
count and the measured seconds of the whole pass, with the machine it ran on.
The count scales the oracle's bounded timing sample to one full solve; the
seconds check that projection.  Calls only the oracle; writes
oracle/iters_globular257.json.  Takes a few minutes on one core.

    python -m oracle.calibrate
"""
import json
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import pb_inputs  # noqa: E402
from oracle import oracle as orc  # noqa: E402


def main():
    atoms = pb_inputs.globular_molecule(2000, seed=2)
    orc.build()
    t0 = time.perf_counter()
    g = orc.place_grid(atoms, 257, 1.5)
    r = orc.solve_problem(atoms, g, eps_in=2.0, eps_out=80.0, ionic_strength_M=0.145,
                          bc=orc.BC_ZERO, rtol=1e-8, with_energy=True)
    out = {"workload": "globular 2000 atoms seed 2, 257^3, fill 1.5, eps 2/80, 0.145 M, zero BC",
           "rtol": 1e-8, "iters": int(r["iters"]), "true_rel_res": float(r["relres"]),
           "converged": bool(r["converged"]), "seconds_full": time.perf_counter() - t0,
           "e_total": r["energy"]["e_total"], "n_cross": int(len(r["cross"]["ids"])), "h": g.h,
           "machine": platform.machine(), "cores_used": 1}
    with open(os.path.join(HERE, "iters_globular257.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(out)


if __name__ == "__main__":
    main()
