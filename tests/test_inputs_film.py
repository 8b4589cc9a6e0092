"""The film-electrode geometry (Sec. 4, Fig. 7 bottom): monodisperse porous
particles of radius 9 sites taking 38 % of each electrode slab, separated by
bulk-like electrolyte."""
import math

import numpy as np

import lpc_inputs
from tests import bruteforce as bf


def test_film_particles_fraction_radius_and_separation():
    e, b = 60, 32
    inp = lpc_inputs.film_supercapacitor(nx=2 * e + b, ny=40, nz=40, electrode=e, bulk=b)
    p = inp.particles
    for x0 in (0, e + b):
        assert abs(p[:, :, x0:x0 + e].mean() - 0.38) <= 0.01
    assert not p[:, :, e:e + b].any()
    # separated spheres: every particle is its own cluster of particle sites
    label, ncl = bf.pore_clusters((~p).astype(np.uint8), inp.periodic)
    vol = 4.0 / 3.0 * math.pi * 9.0 ** 3
    sizes = np.bincount(label[label >= 0].ravel())
    assert ncl == 24                                   # 2 x 2 x 3 spheres per electrode
    assert np.all(np.abs(sizes / vol - 1.0) <= 0.03)
    # fields: the pore-size map inside particles, bulk values outside
    assert np.all(inp.F[~p] == 0.0) and np.all(inp.omega[~p] == 0.0)
    assert np.all((inp.F[p] < 0.0) & (inp.F[p] > -4.0))
    assert np.all(inp.solid == 0)
    lab, names = lpc_inputs.region_labels(inp)
    assert names == ("electrode_minus", "bulk", "electrode_plus")


def test_film_is_seeded():
    a = lpc_inputs.film_supercapacitor(nx=152, ny=40, nz=40, electrode=60, bulk=32)
    b = lpc_inputs.film_supercapacitor(nx=152, ny=40, nz=40, electrode=60, bulk=32)
    assert np.array_equal(a.particles, b.particles) and np.array_equal(a.F, b.F)
