"""Write the oracle's regression values for the 32^3 particle (the FID, the
population and the MSD along x every 100 steps of 2000).  Calls only the
oracle and the input generators; run from the repository root:
    python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import lpc_inputs  # noqa: E402
import oracle  # noqa: E402


def main():
    inp = lpc_inputs.particle()
    res = oracle.run(oracle.pack_input(inp, oracle.MODE_EXACT), inp.uniform_rho0(), inp.steps, msd_axes=1)
    msd = res.msd(0)
    with open(os.path.join(HERE, "oracle_particle_32.txt"), "w") as f:
        f.write("# FP64 oracle, 32^3 particle (seed 1, 30 % solid, F ~ N(-2,1) kT, shift ~ N(-6,2) ppm),\n")
        f.write("# alpha = dt/tau = 0.005, exact weights, rho0 = 1 on pore sites; written by make_golden.py\n")
        f.write("# n  Re M(n)  Im M(n)  P(n)  MSD_x(n)\n")
        for n in range(0, inp.steps + 1, 100):
            f.write("%d %.17g %.17g %.17g %.17g\n" % (n, res.M[n].real, res.M[n].imag, res.P[n], msd[n]))


if __name__ == "__main__":
    main()
