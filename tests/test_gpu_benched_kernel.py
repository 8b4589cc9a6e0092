"""Parity of the kernel the benchmark times against the FP64 oracle.

The benchmarked path is the TMA-fed one-step kernel reading its static data
in link form (one signed weight per link and axis, rebuilt into in-, out- and
stay weights in the kernel).  ``lattice_set_static_form`` makes that form (or
the gather form) on lattices of any size, so:

* long runs (2000 steps) of 64^3-sized lattices in forced link form, and in
  forced gather form, are compared element by element with the oracle run on
  the same rounded weights (the matched-input mode): FID, populations,
  densities and magnetisation relative L2 <= 1e-5, MSD along every axis
  within 1e-5 relative for n >= 10;
* the 384^3 monolith (the benchmark's recipe at 0.42 of its sites, large
  enough for the automatic schedule to choose the link form itself) runs 250
  steps and its whole-lattice FID and population histories and final
  densities are compared with the oracle on the whole lattice.

The first moments mu_a take both signs and cancel over the lattice, so their
element-wise relative L2 is dominated by the rounding of small values; they
are held to 5e-5 (an FP32 emulation of the recursion with fused multiply-adds
lands at 5e-6 to 7e-6 after 2000 steps on a 36 x 40 x 48 lattice).
"""
import numpy as np
import pytest

import lpc_inputs
import oracle
from paper_2603_22553_b300 import binding as B
from tests import helpers as H

pytestmark = pytest.mark.gpu

FORM_CODE = {B.LPC_STATIC_GATHER: 1, B.LPC_STATIC_LINK: 2}

# (nz, ny, nx), periodic (x, y, z), MSD axes, weight type, static form, seed
LONG_CASES = [
    ((64, 64, 64), (1, 1, 1), 7, 0, B.LPC_STATIC_LINK, 301),
    ((48, 80, 72), (0, 1, 1), 1, 0, B.LPC_STATIC_LINK, 302),      # ragged tiles, x walls
    ((40, 70, 130), (1, 0, 0), 6, 0, B.LPC_STATIC_LINK, 303),     # three x tiles, y and z walls
    ((40, 72, 70), (1, 1, 1), 3, 1, B.LPC_STATIC_LINK, 304),      # BF16 weights
    ((64, 64, 64), (1, 1, 1), 7, 0, B.LPC_STATIC_GATHER, 305),
]


@pytest.mark.parametrize("shape,periodic,msd,wdt,form,seed", LONG_CASES)
def test_forced_static_form_2000_steps_against_the_oracle(shape, periodic, msd, wdt, form, seed):
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.random_case(shape, seed, periodic=periodic, solid_frac=0.25, F_sd=1.0, shift_sd=5.0,
                                 alpha=0.5, msd_axes=msd, weight_dtype=wdt)
    steps = 2000
    lat = Lattice.from_input(inp)
    lat.set_schedule(B.LPC_KERNEL_TB, 1)
    lat.set_static_form(form)
    info = lat.info()
    assert info["kernel"] == B.LPC_KERNEL_TB and info["block_steps"] == 1
    assert info["static_form"] == FORM_CODE[form]
    lat.step(steps)
    g = dict(M=lat.fid(), P=lat.population(), rho=lat.density().astype(np.float64), m=lat.magnetization())
    for a in range(3):
        if msd >> a & 1:
            g["msd%d" % a] = lat.msd(a)
            g["mu%d" % a] = lat.moment(a).astype(np.float64)
    assert lat.info()["static_form"] == FORM_CODE[form]
    lat.close()
    o = H.oracle_run(inp, steps, H.MODE_OF_DTYPE[wdt])
    errs = H.compare(g, o, msd, tol=1e-5)
    for a in range(3):
        if msd >> a & 1:
            errs["mu%d" % a] = H.rel_l2(g["mu%d" % a], o.mu[a])
            assert errs["mu%d" % a] <= 5e-5, errs
    print(shape, "form", form, errs)


def test_link_form_matches_gather_form_bit_for_bit():
    """Both static forms hold the same weights: states bit-identical, sums
    equal to FP32 summation order."""
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.random_case((33, 45, 97), 306, periodic=(1, 0, 1), solid_frac=0.3, alpha=0.8, msd_axes=5)
    out = []
    for form in (B.LPC_STATIC_LINK, B.LPC_STATIC_GATHER):
        lat = Lattice.from_input(inp)
        lat.set_schedule(B.LPC_KERNEL_TB, 1)
        lat.set_static_form(form)
        lat.step(37)
        out.append((lat.density(), lat.magnetization(), lat.moment(0), lat.moment(2), lat.fid(), lat.msd(2)))
        lat.close()
    a, b = out
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)
    assert np.allclose(a[4], b[4], rtol=1e-6, atol=1e-6 * abs(b[4][0]))
    assert np.allclose(a[5][1:], b[5][1:], rtol=1e-5)


def test_static_form_switch_mid_run_keeps_the_trajectory():
    """Switching the form between steps releases the old static data and makes
    the new one; the trajectory is the same as without the switch."""
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.random_case((20, 24, 80), 307, periodic=(1, 1, 1), alpha=0.6, msd_axes=0)
    a = Lattice.from_input(inp)
    a.set_schedule(B.LPC_KERNEL_TB, 1)
    a.step(40)
    b = Lattice.from_input(inp)
    b.set_schedule(B.LPC_KERNEL_TB, 1)
    b.set_static_form(B.LPC_STATIC_LINK)
    b.step(13)
    b.set_static_form(B.LPC_STATIC_GATHER)
    assert b.info()["static_form"] == 1
    b.step(14)
    b.set_static_form(B.LPC_STATIC_LINK)
    assert b.info()["static_form"] == 2
    b.step(13)
    assert np.array_equal(a.density(), b.density()) and np.array_equal(a.magnetization(), b.magnetization())
    a.close()
    b.close()


def test_link_form_rejected_where_it_cannot_hold_the_weights():
    """Per-link jump factors break the form's rule (one hop of every open link
    weighs alpha/6): the link form is refused, the gather form allowed."""
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.random_case((8, 8, 70), 308, periodic=(0, 1, 1), alpha=0.6, msd_axes=0)
    links = np.random.default_rng(309).uniform(0.2, 1.0, (3,) + inp.F.shape)
    lat = Lattice.from_input(inp, alpha_links=links)
    with pytest.raises(B.LPCError) as ei:
        lat.set_static_form(B.LPC_STATIC_LINK)
    assert ei.value.status == B.LPC_ERR_INVALID
    lat.set_static_form(B.LPC_STATIC_GATHER)      # allowed
    lat.close()


RES_ALL = ((-0.75, 1.25, 0.5 - 0.25j), (0.5, 0.625, 1.0 + 0.0j), (0.25, 0.75, 0.0j), (-1.5, 2.0, 0.0j),
           (-0.25, 1.5, 0.75 + 0.5j), (0.75, 0.5, 0.25 - 0.5j))


# (nz, ny, nx), periodic (x, y, z), reservoir faces, regions, MSD axes, weight type
RES_REG_CASES = [
    ((20, 36, 130), (0, 0, 1), (0, 1, 3), 3, 5, 0),        # x and y reservoirs, regions, MSD x and z
    ((24, 40, 128), (0, 1, 0), (0, 1, 4, 5), 3, 1, 1),     # x and z reservoirs, BF16, MSD x
    ((16, 48, 96), (1, 0, 1), (2,), 0, 2, 0),              # a lower y reservoir only, no regions
    ((18, 33, 70), (0, 1, 1), (1,), 2, 1, 0),              # an upper x reservoir only (lower x face a wall)
]


@pytest.mark.parametrize("shape,periodic,faces,nreg,msd,wdt", RES_REG_CASES)
def test_link_form_with_reservoirs_and_regions(shape, periodic, faces, nreg, msd, wdt):
    """Reservoir links follow the Metropolis rule too (one hop weighs alpha/6),
    so the link form holds lattices with reservoir faces; the links entering
    column 0 and row 0 come from the ghost sites.  Regions stage their labels
    beside the links.  States bit-identical to the gather form, sums to FP32
    summation order (the link form attributes MSD increments to the source
    site, as the region and reservoir sums need), and against the oracle."""
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.random_case(shape, 340 + len(faces), periodic=periodic, alpha=0.8, msd_axes=msd,
                                 weight_dtype=wdt)
    inp.reservoirs = tuple(RES_ALL[f] if f in faces else None for f in range(6))
    kw = {}
    lab = None
    if nreg:
        lab = lpc_inputs.random_regions(shape, 350, nreg)
        kw = dict(region=lab, n_regions=nreg)
    steps = 120
    out = {}
    for form in (B.LPC_STATIC_LINK, B.LPC_STATIC_GATHER):
        lat = Lattice.from_input(inp, **kw)
        lat.set_schedule(B.LPC_KERNEL_TB, 1)
        lat.set_static_form(form)
        assert lat.info()["static_form"] == FORM_CODE[form]
        lat.step(steps)
        r = dict(rho=lat.density(), m=lat.magnetization(), M=lat.fid(), P=lat.population())
        for a in range(3):
            if msd >> a & 1:
                r["mu%d" % a] = lat.moment(a)
                r["msd%d" % a] = lat.msd(a)
        for g in range(nreg):
            r["Mr%d" % g] = lat.fid_region(g)
            r["Pr%d" % g] = lat.population_region(g)
        out[form] = r
        lat.close()
    a, b = out[B.LPC_STATIC_LINK], out[B.LPC_STATIC_GATHER]
    for k in a:
        if k in ("rho", "m") or k.startswith("mu"):
            assert np.array_equal(a[k], b[k]), k
        else:
            assert np.allclose(a[k], b[k], rtol=1e-5, atol=1e-6 * abs(b["P"][0])), k
    pk = oracle.pack_input(inp, H.MODE_OF_DTYPE[wdt])
    o = oracle.run(pk, inp.uniform_rho0(), steps, msd_axes=msd, region=lab, n_regions=nreg)
    g = dict(a)
    g["rho"] = a["rho"].astype(np.float64)
    H.compare(g, o, msd, tol=1e-5)
    for r in range(nreg):
        assert H.rel_l2(a["Mr%d" % r], o.Mr[r]) <= 1e-5
        assert H.rel_l2(a["Pr%d" % r], o.Pr[r]) <= 1e-5


def test_monolith_384_link_form_whole_lattice_against_the_oracle():
    """The benchmark's monolith recipe at 384^3 (5.7e7 sites: the automatic
    schedule takes the TMA-fed one-step kernel in link form), 250 steps: the
    whole-lattice FID and population histories and the final densities
    against the FP64 oracle on the same FP32 weights."""
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.monolith(edge=384, msd_axes=0)
    steps = 250
    lat = Lattice.from_input(inp)
    lat.step(steps)
    info = lat.info()
    assert info["kernel"] == B.LPC_KERNEL_TB and info["block_steps"] == 1 and info["static_form"] == 2
    M, P = lat.fid(), lat.population()
    rho = lat.density()
    m = lat.magnetization()
    lat.close()
    o = H.oracle_run(inp, steps, oracle.MODE_F32, msd_axes=0)
    e = {"fid": H.rel_l2(M, o.M), "pop": float(np.max(np.abs(P / o.P - 1.0))),
         "rho": H.rel_l2(rho.astype(np.float64), o.rho), "m": H.rel_l2(m, o.m)}
    print("384^3 link form, 250 steps:", e)
    assert e["fid"] <= 1e-5 and e["pop"] <= 1e-5 and e["rho"] <= 1e-5 and e["m"] <= 1e-5, e
