"""Writes the oracle's state after the full step counts of two configurations,
for the GPU FP64 parity tests that would otherwise spend minutes of CPU time
in the oracle:

  cylinder48_fp64_200steps.txt  2D cylinder, 48^2 cells on [-4,4]^2, 24^2
                                trapezoid velocities on [-5,5]^2, Kn 0.1, Ma 0.3,
                                200 steps from the freestream (every fluid cell)
  sphere24_fp64_50steps.txt     the 3D sphere downscaled to 24^3 cells and 12^3
                                velocities, 50 steps (every 7th fluid cell)

Each file holds the residual of the last step, F, Q, C_D, C_L and, per cell
kept, its index and W = (rho, rho U, rho E).  Only the CPU oracle runs here.

    python tests/golden/make_oracle_goldens.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2512_20252_gb300 import workloads as wl  # noqa: E402

CASES = {
    "cylinder48_fp64_200steps.txt": (wl.cylinder_48, 200, 1),
    "sphere24_fp64_50steps.txt": (wl.sphere_24, 50, 7),
}


def write(name, make, steps, every):
    case = make()
    o = oracle.OracleCase(case)
    res = o.step(steps)
    W, _ = o.moments()
    F, Q, CD, CL = o.forces()
    cells = np.nonzero(o.cell_types() == oracle.FLUID)[0][::every]
    with open(os.path.join(HERE, name), "w") as fh:
        fh.write(f"# oracle (oracle/ibdvm_oracle.c), {steps} steps, every {every} fluid cell(s); "
                 f"written by tests/golden/make_oracle_goldens.py\n")
        fh.write(f"residual {res:.17g}\n")
        fh.write("F " + " ".join(f"{x:.17g}" for x in F) + "\n")
        fh.write(f"Q {Q:.17g}\nCD {CD:.17g}\nCL {CL:.17g}\n")
        for c in cells:
            fh.write(f"{c} " + " ".join(f"{x:.17g}" for x in W[c]) + "\n")


if __name__ == "__main__":
    for name, (make, steps, every) in CASES.items():
        if len(sys.argv) > 1 and name not in sys.argv[1:]:
            continue
        write(name, make, steps, every)
        print("wrote", name)
