"""Seeded random configurations through every one-step schedule against the
matched-input FP64 oracle: ragged shapes (some below a tile, some spanning
several), periodic or walled axes, reservoir faces, per-link jump factors,
region labels, FP32 or BF16 weights and any set of MSD axes.  Tolerances as
in test_gpu_parity (relative L2 1e-5 against the matched oracle)."""
import numpy as np
import pytest

import lpc_inputs
import oracle
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _config(i):
    rng = np.random.default_rng(5000 + i)
    shape = (int(rng.integers(3, 24)), int(rng.integers(3, 40)), int(rng.integers(3, 140)))
    periodic = tuple(int(v) for v in rng.integers(0, 2, 3))
    inp = lpc_inputs.random_case(shape, 6000 + i, periodic=periodic, solid_frac=float(rng.uniform(0, 0.35)),
                                 F_sd=float(rng.uniform(0.2, 2.0)), shift_sd=float(rng.uniform(1, 40)),
                                 alpha=float(rng.uniform(0.2, 1.0)), msd_axes=int(rng.integers(0, 8)),
                                 weight_dtype=int(rng.integers(0, 2)))
    if rng.random() < 0.4:
        _, inp.alpha_links = lpc_inputs.symmetric_links(shape, 7000 + i, lo=0.1, hi=1.0)
    res = [None] * 6
    for f in range(4):
        if not periodic[f // 2] and rng.random() < 0.6:
            res[f] = (float(rng.normal(0, 1)), float(np.float32(rng.uniform(0.2, 2.0))),
                      complex(np.float32(rng.normal(0, 1)), np.float32(rng.normal(0, 1))))
    inp.reservoirs = tuple(res) if any(r is not None for r in res) else None
    nreg = int(rng.integers(0, 5))
    lab = lpc_inputs.random_regions(shape, 8000 + i, nreg) if nreg else None
    return inp, lab, nreg


@pytest.mark.parametrize("i", range(40))
def test_random_configuration_all_schedules(i):
    from paper_2603_22553_b300 import binding as B
    from paper_2603_22553_b300.lattice import Lattice, step_many
    inp, lab, nreg = _config(i)
    steps = 40
    pk = oracle.pack_input(inp, H.MODE_OF_DTYPE[inp.weight_dtype])
    o = oracle.run(pk, inp.uniform_rho0(), steps, msd_axes=inp.msd_axes,
                   region=lab, n_regions=nreg)
    kw = dict(region=lab, n_regions=nreg) if nreg else {}
    for sched in ("step1", "tb1", "batch"):
        lat = Lattice.from_input(inp, **kw)
        if sched == "tb1":
            lat.set_schedule(B.LPC_KERNEL_TB, 1)
        elif sched == "step1":
            lat.set_schedule(B.LPC_KERNEL_STEP1, 1)
        if sched == "batch":
            step_many([lat], [steps])
        else:
            lat.step(steps)
        assert H.rel_l2(lat.fid(), o.M) <= 1e-5, (i, sched)
        assert H.rel_l2(lat.population(), o.P) <= 1e-5, (i, sched)
        assert H.rel_l2(lat.density().astype(np.float64), o.rho) <= 1e-5, (i, sched)
        for a in range(3):
            if inp.msd_axes >> a & 1:
                ref = o.msd(a)
                assert np.max(np.abs(lat.msd(a) - ref)) <= 1e-5 * max(np.max(np.abs(ref)), 1e-30), (i, sched, a)
        for r in range(nreg):
            assert np.max(np.abs(lat.fid_region(r) - o.Mr[r])) <= 1e-5 * o.P[0], (i, sched, r)
        lat.close()
