"""Fixtures under tests/golden: the paper's printed constants against the
input recipe and the closed form of Eq. 7, and the oracle against its own
stored values for the 32^3 particle (a regression check; the values were
written by tests/golden/make_golden.py, which calls only the oracle)."""
import os

import numpy as np
import pytest

import lpc_inputs
import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _paper():
    vals = {}
    for line in open(os.path.join(GOLDEN, "paper_values.txt")):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            vals[name] = float(value)
    return vals


def test_input_recipe_uses_the_papers_constants():
    p = _paper()
    assert lpc_inputs.DT == p["dt"] and lpc_inputs.TAU == p["tau_1"] and lpc_inputs.NU0 == p["nu0"]
    assert lpc_inputs.ALPHA == pytest.approx(p["dt"] / p["tau_1"])


def test_eq7_diffusion_with_the_papers_constants():
    """D = alpha a^2 / (2 d dt) on a uniform lattice (Eq. 7), alpha = dt / tau."""
    p = _paper()
    for tau in (p["tau_1"], p["tau_2"]):
        alpha = p["dt"] / tau
        shape = (6, 6, 6)
        pk = oracle.pack(6, 6, 6, (1, 1, 1), alpha, p["dt"], 1.0, np.zeros(shape), np.zeros(shape),
                         np.zeros(shape, np.uint8))
        r = oracle.run(pk, np.ones(shape), 40, msd_axes=7)
        D = np.mean([oracle.diffusion(r.msd(a), p["dt"])[1:] for a in range(3)], axis=0)
        assert np.allclose(D, alpha / (2 * p["d_dim"] * p["dt"]), rtol=1e-12)


def test_film_geometry_matches_the_papers_particles():
    p = _paper()
    inp = lpc_inputs.film_supercapacitor(nx=152, ny=40, nz=40, electrode=60, bulk=32, radius=p["particle_r"],
                                         fraction=p["film_frac"])
    assert abs(inp.particles[:, :, :60].mean() - p["film_frac"]) <= 0.01


def test_oracle_regression_particle_32():
    rows = np.loadtxt(os.path.join(GOLDEN, "oracle_particle_32.txt"))
    inp = lpc_inputs.particle()
    res = oracle.run(oracle.pack_input(inp, oracle.MODE_EXACT), inp.uniform_rho0(), inp.steps, msd_axes=1)
    n = rows[:, 0].astype(int)
    assert np.allclose(res.M[n].real, rows[:, 1], rtol=1e-12, atol=0)
    assert np.allclose(res.M[n].imag, rows[:, 2], rtol=1e-12, atol=1e-12 * rows[0, 3])
    assert np.allclose(res.P[n], rows[:, 3], rtol=1e-12)
    assert np.allclose(res.msd(0)[n], rows[:, 4], rtol=1e-12, atol=1e-15)
