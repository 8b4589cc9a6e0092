"""Whole-lattice parity at the full sizes of two workloads (every site and
every step compared, not sampled sites).

* Particle in electrolyte bath, 256^3 (FP32): the first 1000 of its 10 000
  steps, the FID of every step and its spectrum (a plain DFT, Eq. 9; by
  Parseval its relative error equals the FID's) and the final densities,
  against the FP64 oracle on the same FP32 weights.  The oracle takes about
  three minutes of host time per 1000 steps; ``LPC_FULL_PARITY=1`` runs the
  whole configured run of 10 000 steps (a 10 001-point spectrum).
* Supercapacitor slab, 2048 x 256 x 256 (BF16 weights, first moment along
  x, walls in x): the first 100 of its 5000 steps in the oracle's matched
  BF16 mode: the density profile along x (sum over y and z), MSD_x, the FID
  and the whole density field.  The oracle's 6.7e10 site updates of the
  first 500 steps take about ten minutes on the host, longer than the whole
  GPU suite should; ``LPC_FULL_PARITY=1`` runs those 500 steps instead.

Tolerance, from the arithmetic: the matched oracle takes the stay weight
s = 1 - sum_k w_k of the FP32 weights in FP64, the kernels in FP32, rounded
once: |s_f32 - s| <= 2^-25 for s in [0.5, 1).  Where many sites share one
rounding (the 87 % of the bath that is uniform bulk electrolyte, F = 0: all
weights alpha/6 and s_f32 - s = +4.9e-9) the bias does not average out, and
populations drift by up to n 2^-25 relative after n steps (3.0e-5 at
n = 1000); the other rounding errors are random and far smaller.  The bound
is max(1e-5, n 2^-25), and never above the 1e-4 that the method's results
are held to.
"""
import os

import numpy as np
import pytest

import lpc_inputs
import oracle
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _tol(steps):
    return min(1e-4, max(1e-5, steps * 2.0 ** -25))


def test_particle_in_bath_256_whole_lattice():
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.particle_in_bath()
    steps = 10000 if os.environ.get("LPC_FULL_PARITY") == "1" else 1000
    lat = Lattice.from_input(inp)
    lat.step(steps)
    M, P = lat.fid(), lat.population()
    rho = lat.density().astype(np.float64)
    info = lat.info()
    lat.close()
    o = H.oracle_run(inp, steps, oracle.MODE_F32, msd_axes=0)
    _, S_g = oracle.spectrum(M, inp.dt)
    _, S_o = oracle.spectrum(o.M, inp.dt)
    e = {"fid": H.rel_l2(M, o.M), "spectrum": H.rel_l2(S_g, S_o), "rho": H.rel_l2(rho, o.rho),
         "pop": float(np.max(np.abs(P / o.P - 1.0)))}
    print("256^3 bath, %d steps, kernel %d form %d:" % (steps, info["kernel"], info["static_form"]), e)
    tol = _tol(steps)
    assert e["fid"] <= tol and e["spectrum"] <= tol and e["rho"] <= tol and e["pop"] <= tol, e


def test_supercapacitor_2048x256x256_whole_lattice_matched_bf16():
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.supercapacitor()
    steps = 500 if os.environ.get("LPC_FULL_PARITY") == "1" else 100
    lat = Lattice.from_input(inp)
    lat.step(steps)
    M, P = lat.fid(), lat.population()
    rho = lat.density().astype(np.float64)
    msd = lat.msd(0)
    lat.close()
    o = H.oracle_run(inp, steps, oracle.MODE_BF16, msd_axes=1)
    prof_g = rho.sum(axis=(0, 1))
    prof_o = o.rho.sum(axis=(0, 1))
    msd_o = o.msd(0)
    e = {"fid": H.rel_l2(M, o.M), "rho": H.rel_l2(rho, o.rho), "profile": H.rel_l2(prof_g, prof_o),
         "profile_max": float(np.max(np.abs(prof_g - prof_o) / np.abs(prof_o))),
         "msd_x": float(np.max(np.abs(msd[10:] - msd_o[10:]) / np.abs(msd_o[10:]))),
         "pop": float(np.max(np.abs(P / o.P - 1.0)))}
    print("2048x256x256 slab, %d steps, matched BF16:" % steps, e)
    assert all(v <= _tol(steps) for v in e.values()), e
