"""GPU parity of reservoir faces and region-resolved sums against the FP64 oracle.

Reservoir faces (Sec. 3.2 item 1: field values fixed in the ghost layer of a
non-periodic face) and region labels (the spectra and diffusion of separate
parts of a system, Sec. 4) run through lattice_create_ex.  Tolerances as in
test_gpu_parity: relative L2 <= 1e-5 against the matched-input oracle (its
own FP32 roundings) and <= 1e-4 against the exact oracle; weights within one
unit in the last place of the oracle's rounding, with the same zero pattern.
Reservoir values are exactly representable in FP32, so the GPU's FP32 ghost
values equal the oracle's FP64 ones.
"""
import numpy as np
import pytest

import lpc_inputs
import oracle
from tests import helpers as H

pytestmark = pytest.mark.gpu

RES = ((-0.75, 1.25, 0.5 - 0.25j), (0.5, 0.625, 1.0 + 0.0j), None, (-1.5, 2.0, 0.0j), None, None)


def _lattice(inp, sched, **kw):
    from paper_2603_22553_b300 import binding as B
    from paper_2603_22553_b300.lattice import Lattice
    lat = Lattice.from_input(inp, **kw)
    if sched == "step1":
        lat.set_schedule(B.LPC_KERNEL_STEP1, 1)
    elif sched == "tb1":
        lat.set_schedule(B.LPC_KERNEL_TB, 1)
    return lat


def _advance(lat, sched, steps):
    from paper_2603_22553_b300.lattice import step_many
    if sched == "batch":
        step_many([lat], [steps])
    else:
        lat.step(steps)


def _read(lat, axes):
    g = dict(M=lat.fid(), P=lat.population(), rho=lat.density().astype(np.float64), m=lat.magnetization())
    for a in range(3):
        if axes >> a & 1:
            g["msd%d" % a] = lat.msd(a)
    return g


def _ulp_diff(a, b, bits):
    scale = np.where(b != 0, 2.0 ** (np.floor(np.log2(np.abs(np.where(b != 0, b, 1.0)))) - (bits - 1)), 1.0)
    return np.abs(a - b) / scale


def _compare_fid_pop(g, o, tol):
    assert H.rel_l2(g["M"], o.M) <= tol
    assert H.rel_l2(g["P"], o.P) <= tol
    assert H.rel_l2(g["rho"], o.rho) <= tol
    assert H.rel_l2(g["m"], o.m) <= tol


@pytest.mark.parametrize("sched", ["auto", "step1", "tb1", "batch"])
def test_reservoir_parity(sched):
    shape = (20, 36, 130)
    inp = lpc_inputs.random_case(shape, 301, periodic=(0, 0, 1), alpha=0.8, msd_axes=5)
    inp.reservoirs = RES
    lat = _lattice(inp, sched)
    pk = oracle.pack_input(inp, oracle.MODE_F32)
    w = lat.weights().reshape(6, -1).T.astype(np.float64)
    assert np.array_equal(w == 0, pk.w == 0), "link geometry differs"
    assert _ulp_diff(w, pk.w, 24).max() <= 1.0
    steps = 150
    _advance(lat, sched, steps)
    g = _read(lat, 5)
    o = oracle.run(pk, inp.uniform_rho0(), steps, msd_axes=5)
    _compare_fid_pop(g, o, 1e-5)
    for a in (0, 2):
        sl = slice(10, None)
        assert np.max(np.abs(g["msd%d" % a][sl] - o.msd(a)[sl]) / np.abs(o.msd(a)[sl])) <= 1e-5
    oe = oracle.run(oracle.pack_input(inp), inp.uniform_rho0(), steps, msd_axes=5)
    _compare_fid_pop(g, oe, 1e-4)
    # population flows through the reservoir faces: not conserved
    assert abs(g["P"][-1] / g["P"][0] - 1.0) > 1e-3
    lat.close()


@pytest.mark.parametrize("sched", ["step1", "tb1"])
def test_reservoir_grand_canonical_equilibrium(sched):
    """Reservoirs at the same (F_res, rho_res) on both x faces: the
    equilibration phase converges to rho_res exp(-(F - F_res)) on every pore
    site (all connected: no solids); the propagation phase then restarts with
    the reservoirs' own magnetisation m_res = 0 in the ghost layer (oracle run
    from the equilibrated populations)."""
    shape = (8, 16, 32)
    inp = lpc_inputs.random_case(shape, 302, periodic=(0, 1, 1), solid_frac=0.0, F_sd=0.7, alpha=1.0,
                                 msd_axes=0)
    F_res, rho_res = -0.5, 1.5
    inp.reservoirs = ((F_res, rho_res, 0.0), (F_res, rho_res, 0.0), None, None, None, None)
    lat = _lattice(inp, sched)
    # a fixed number of steps (threshold 0): the slowest mode, about
    # sin(pi (x + 1) / 33), decays at least like (1 - 0.6 (alpha / 6) (pi / 33)^2)^n,
    # below e^-30 over them; FP32 rounding keeps max |drho| near 1 ulp
    it, diff = lat.equilibrate(0.0, 40000, check_every=2000)
    assert it == 40000 and diff < 1e-5
    rho_eq = rho_res * np.exp(-(inp.F - F_res))
    rho = lat.density().astype(np.float64)
    # FP32 arithmetic: each step's rounding (about 6e-8 relative, biased by
    # the FP32 stay weight) accumulates in the slowest mode over 1/gap ~ 1e3
    # steps, a few 1e-5 at the fixed point (a numpy FP32 emulation of the same
    # recursion lands 4.7e-5 away): the 1e-4 density bound applies
    assert H.rel_l2(rho, rho_eq) <= 1e-4
    steps = 40
    lat.step(steps)
    pk = oracle.pack_input(inp, oracle.MODE_F32)
    o = oracle.run(pk, rho, steps, msd_axes=0)
    assert H.rel_l2(lat.fid(), o.M) <= 1e-5
    assert H.rel_l2(lat.population(), o.P) <= 1e-5
    # the reservoirs bring in no magnetisation: |M| falls below P
    assert abs(lat.fid()[-1]) < lat.population()[-1] * (1 - 1e-4)
    lat.close()


def test_reservoir_rejects_deep_temporal_blocks():
    from paper_2603_22553_b300 import binding as B
    inp = lpc_inputs.random_case((8, 16, 64), 303, periodic=(0, 1, 1), msd_axes=0)
    inp.reservoirs = RES[:2] + (None,) * 4
    lat = _lattice(inp, "auto", ghost=4)
    with pytest.raises(B.LPCError):
        lat.set_schedule(B.LPC_KERNEL_TB, 2)
    lat.close()


def _region_case(shape=(20, 36, 130), seed=311, n_regions=3, **kw):
    inp = lpc_inputs.random_case(shape, seed, periodic=(1, 0, 1), alpha=0.9, msd_axes=5, **kw)
    lab = lpc_inputs.random_regions(shape, seed + 1, n_regions)
    return inp, lab


@pytest.mark.parametrize("sched", ["auto", "step1", "tb1"])
def test_region_sums_parity(sched):
    inp, lab = _region_case()
    lat = _lattice(inp, sched, region=lab, n_regions=3)
    steps = 120
    lat.step(steps)
    o = oracle.run(oracle.pack_input(inp, oracle.MODE_F32), inp.uniform_rho0(), steps, msd_axes=5,
                   region=lab, n_regions=3)
    M, P = lat.fid(), lat.population()
    Mr = np.array([lat.fid_region(r) for r in range(3)])
    Pr = np.array([lat.population_region(r) for r in range(3)])
    for r in range(3):
        assert H.rel_l2(Mr[r], o.Mr[r]) <= 1e-5
        assert H.rel_l2(Pr[r], o.Pr[r]) <= 1e-5
        for a in (0, 2):
            ms = lat.msd_region(r, a)
            ref = np.concatenate([[0.0], np.cumsum(o.Dr[r, a])]) / o.P[0]
            assert np.max(np.abs(ms[10:] - ref[10:])) <= 1e-5 * np.max(np.abs(ref[10:]))
    # the regions partition the lattice
    assert np.max(np.abs(Mr.sum(axis=0) - M)) <= 1e-6 * P[0]
    assert np.max(np.abs(Pr.sum(axis=0) - P)) <= 1e-6 * P[0]
    for a in (0, 2):
        tot = sum(lat.msd_region(r, a) for r in range(3))
        assert np.max(np.abs(tot - lat.msd(a))) <= 1e-6 * np.max(np.abs(lat.msd(a)))
    lat.close()


def test_region_lattice_in_step_many_and_checkpoint():
    """A region lattice advanced by lattice_step_many beside a plain one gives
    the region sums of lattice_step_n; a checkpoint carries the region
    histories and resuming continues them bit for bit."""
    from paper_2603_22553_b300.lattice import step_many
    inp, lab = _region_case(shape=(12, 20, 70), seed=321, n_regions=2)
    plain = lpc_inputs.random_case((10, 18, 40), 322, msd_axes=5)
    a = _lattice(inp, "auto", region=lab, n_regions=2)
    b = _lattice(plain, "auto")
    step_many([a, b], [50, 30])
    c = _lattice(inp, "auto", region=lab, n_regions=2)
    c.step(50)
    for r in range(2):
        assert np.array_equal(a.fid_region(r), c.fid_region(r))
        assert np.array_equal(a.msd_region(r, 0), c.msd_region(r, 0))
    blob = c.get_state()
    c.step(20)
    d = _lattice(inp, "auto", region=lab, n_regions=2)
    d.set_state(blob)
    d.step(20)
    for r in range(2):
        assert np.array_equal(c.fid_region(r), d.fid_region(r))
        assert np.array_equal(c.population_region(r), d.population_region(r))
        assert np.array_equal(c.msd_region(r, 2), d.msd_region(r, 2))
    for lat in (a, b, c, d):
        lat.close()


def test_supercapacitor_slab_regions_and_reservoirs():
    """A scaled supercapacitor slab (electrode / bulk / electrode along x,
    BF16 weights, MSD along x) with reservoirs on both x faces and the three
    parts as regions: per-region FIDs, spectra (Parseval: the spectrum error
    equals the FID error) and MSD against the matched-input oracle."""
    from paper_2603_22553_b300 import downstream
    inp = lpc_inputs.supercapacitor(nx=160, ny=32, nz=24, electrode=64, bulk=32, steps=300)
    inp.alpha = 0.3
    inp.reservoirs = ((0.0, 1.0, 1.0), (0.0, 1.0, 1.0), None, None, None, None)
    lab, names = lpc_inputs.region_labels(inp)
    assert names == ("electrode_minus", "bulk", "electrode_plus")
    lat = _lattice(inp, "tb1", region=lab, n_regions=3)
    lat.step(inp.steps)
    o = oracle.run(oracle.pack_input(inp, oracle.MODE_BF16), inp.uniform_rho0(), inp.steps, msd_axes=1,
                   region=lab, n_regions=3)
    for r in range(3):
        Mr = lat.fid_region(r)
        assert H.rel_l2(Mr, o.Mr[r]) <= 1e-5
        _, _, S = downstream.spectrum(Mr, inp.dt)
        _, So = oracle.spectrum(o.Mr[r], inp.dt)
        assert H.rel_l2(S, So) <= 1e-5
    assert H.rel_l2(lat.fid(), o.M) <= 1e-5
    lat.close()


@pytest.mark.parametrize("msd_axes,wdt", [(0, 0), (1, 1), (7, 0)])
def test_fused_region_sums_match_the_separate_pass(msd_axes, wdt):
    """The one-step TMA kernel takes the region sums itself (labels staged with
    the static data): states are bit-identical to the same kernel without
    regions and its totals (there the sums over regions) agree to FP32
    summation order, as do the region sums with the separate region pass of
    the register-pipelined schedule; the checkpoint of a fused run resumes
    bit for bit."""
    from paper_2603_22553_b300 import binding as B
    shape = (40, 64, 200)
    inp = lpc_inputs.random_case(shape, 331, periodic=(1, 1, 0), alpha=0.7, msd_axes=msd_axes,
                                 weight_dtype=wdt)
    lab = lpc_inputs.random_regions(shape, 332, 4)
    steps = 64
    fused = _lattice(inp, "tb1", region=lab, n_regions=4)
    assert fused.info()["kernel"] == B.LPC_KERNEL_TB and fused.info()["block_steps"] == 1
    plain = _lattice(inp, "tb1")
    sep = _lattice(inp, "step1", region=lab, n_regions=4)
    for lat in (fused, plain, sep):
        lat.step(steps)
    assert np.array_equal(fused.density(), plain.density())
    assert np.array_equal(fused.density(), sep.density())
    P0 = fused.population()[0]
    assert np.max(np.abs(fused.fid() - plain.fid())) <= 1e-6 * P0
    assert np.max(np.abs(fused.population() - plain.population())) <= 1e-6 * P0
    for r in range(4):
        assert np.max(np.abs(fused.fid_region(r) - sep.fid_region(r))) <= 1e-6 * P0
        assert np.max(np.abs(fused.population_region(r) - sep.population_region(r))) <= 1e-6 * P0
        for a in range(3):
            if msd_axes >> a & 1:
                ref = sep.msd_region(r, a)
                assert np.max(np.abs(fused.msd_region(r, a) - ref)) <= 1e-6 * np.max(np.abs(ref))
                ref = plain.msd(a)
                assert np.max(np.abs(fused.msd(a) - ref)) <= 1e-6 * np.max(np.abs(ref))
    o = oracle.run(oracle.pack_input(inp, H.MODE_OF_DTYPE[wdt]), inp.uniform_rho0(), steps,
                   msd_axes=msd_axes, region=lab, n_regions=4)
    for r in range(4):
        assert H.rel_l2(fused.fid_region(r), o.Mr[r]) <= 1e-5
    blob = fused.get_state()
    fused.step(10)
    again = _lattice(inp, "tb1", region=lab, n_regions=4)
    again.set_state(blob)
    again.step(10)
    for r in range(4):
        assert np.array_equal(fused.fid_region(r), again.fid_region(r))
        assert np.array_equal(fused.population_region(r), again.population_region(r))
        for a in range(3):
            if msd_axes >> a & 1:
                assert np.array_equal(fused.msd_region(r, a), again.msd_region(r, a))
    for lat in (fused, plain, sep, again):
        lat.close()


RES_FACE = ((-0.75, 1.25, 0.5 - 0.25j), (0.5, 0.625, 1.0 + 0.0j), (0.25, 0.75, 0.0j), (-1.5, 2.0, 0.0j),
            (-0.25, 1.5, 0.75 + 0.5j), (0.75, 0.5, 0.25 - 0.5j))

# (nz, ny, nx), periodic (x, y, z), reservoir faces, regions, MSD axes, weight type
SOURCE_SUM_CASES = [
    ((12, 20, 97), (1, 1, 1), (), 3, 1, 0),           # periodic x; the last tile's last site is a lane's first
    ((10, 18, 131), (0, 1, 1), (0, 1), 2, 5, 1),       # x reservoirs, BF16, a last tile of 3 sites, MSD x and z
    ((10, 16, 64), (0, 0, 1), (0, 2), 0, 7, 0),        # reservoirs without regions, one full tile, every axis
    ((9, 20, 33), (0, 1, 1), (0, 1), 0, 1, 0),         # a single tile of 33 sites between two reservoirs
    ((8, 24, 100), (1, 0, 0), (2, 3, 4), 2, 3, 0),     # the last site is a lane's second; y and z reservoirs
]


@pytest.mark.parametrize("shape,periodic,faces,nreg,msd,wdt", SOURCE_SUM_CASES)
def test_source_attributed_msd_sums_of_the_one_step_tma_kernel(shape, periodic, faces, nreg, msd, wdt):
    """With regions or reservoir faces the MSD increments are summed over
    source sites from their out-weights; the one-step TMA kernel takes the x
    out-weights from the x neighbours' in-weights (the tile's two ends from a
    small edge array) and stages those of y and z.  Ragged last tiles that end
    on either site of a lane, periodic and reservoir x faces: states
    bit-identical to the register-pipelined schedule (separate region pass,
    out-weights read directly), totals and region sums equal to FP32
    summation order, and against the FP64 oracle."""
    from paper_2603_22553_b300 import binding as B
    inp = lpc_inputs.random_case(shape, 360 + shape[2], periodic=periodic, solid_frac=0.2, alpha=0.8,
                                 msd_axes=msd, weight_dtype=wdt)
    inp.reservoirs = tuple(RES_FACE[f] if f in faces else None for f in range(6))
    kw, lab = {}, None
    if nreg:
        lab = lpc_inputs.random_regions(shape, 361 + shape[2], nreg)
        kw = dict(region=lab, n_regions=nreg)
    steps = 50
    tma = _lattice(inp, "tb1", **kw)
    tma.set_static_form(B.LPC_STATIC_GATHER)
    ref = _lattice(inp, "step1", **kw)
    for lat in (tma, ref):
        lat.step(steps)
    info = tma.info()
    assert info["kernel"] == B.LPC_KERNEL_TB and info["block_steps"] == 1 and info["static_form"] == 1
    assert np.array_equal(tma.density(), ref.density()) and np.array_equal(tma.magnetization(), ref.magnetization())
    P0 = ref.population()[0]
    assert np.max(np.abs(tma.fid() - ref.fid())) <= 1e-6 * P0
    for a in range(3):
        if msd >> a & 1:
            assert np.array_equal(tma.moment(a), ref.moment(a))
            r = ref.msd(a)
            assert np.max(np.abs(tma.msd(a)[1:] - r[1:])) <= 1e-5 * np.max(np.abs(r[1:])), a
            for g in range(nreg):
                rr = ref.msd_region(g, a)
                assert np.max(np.abs(tma.msd_region(g, a) - rr)) <= 1e-5 * np.max(np.abs(rr)) + 1e-12, (g, a)
    pk = oracle.pack_input(inp, H.MODE_OF_DTYPE[wdt])
    o = oracle.run(pk, inp.uniform_rho0(), steps, msd_axes=msd, region=lab, n_regions=nreg)
    g = _read(tma, msd)
    _compare_fid_pop(g, o, 1e-5)
    for a in range(3):
        if msd >> a & 1:
            assert np.max(np.abs(g["msd%d" % a][10:] / o.msd(a)[10:] - 1.0)) <= 1e-5, a
    for r in range(nreg):
        assert H.rel_l2(tma.fid_region(r), o.Mr[r]) <= 1e-5
        for a in range(3):
            if msd >> a & 1:
                ms = tma.msd_region(r, a)
                rr = np.concatenate([[0.0], np.cumsum(o.Dr[r, a])]) / o.P[0]
                assert np.max(np.abs(ms[10:] - rr[10:])) <= 1e-5 * np.max(np.abs(rr[10:])), (r, a)
    for lat in (tma, ref):
        lat.close()


def test_kohn_vacf_and_region_diffusion_parity():
    """Eq. 4 (Kohn route) from a Boltzmann start and the diffusion of the
    particles of each region, from the GPU's histories (downstream) against
    the oracle's estimators on its own run."""
    from paper_2603_22553_b300 import binding as B
    from paper_2603_22553_b300 import downstream
    shape = (16, 24, 70)
    inp = lpc_inputs.random_case(shape, 341, periodic=(1, 0, 1), solid_frac=0.2, F_sd=1.0, alpha=0.8,
                                 msd_axes=7)
    lab = lpc_inputs.random_regions(shape, 342, 2)
    lat = _lattice(inp, "auto", region=lab, n_regions=2, init=B.LPC_INIT_BOLTZMANN)
    steps = 300
    lat.step(steps)
    rho_eq = oracle.boltzmann(inp.F, inp.solid)
    o = oracle.run(oracle.pack_input(inp, oracle.MODE_F32), rho_eq, steps, msd_axes=7, region=lab, n_regions=2)
    P0 = lat.population()[0]
    for a in range(3):
        Dg = downstream.kohn_diffusion(lat.msd(a), inp.dt)
        Do = oracle.kohn_diffusion(o.dmsd[a], o.P[0], inp.dt)
        assert np.max(np.abs(Dg - Do) / np.abs(Do)) <= 1e-4
        cg, co = downstream.vacf(lat.msd(a)), oracle.vacf(o.dmsd[a], o.P[0])
        assert np.max(np.abs(cg - co)) <= 1e-4 * co[0]
        for r in range(2):
            Drg = downstream.region_diffusion(lat.msd_region(r, a), lat.population_region(r), P0, inp.dt)
            Dro = oracle.region_diffusion(o.Dr[r, a], o.Pr[r], inp.dt)
            assert np.max(np.abs(Drg - Dro) / np.abs(Dro)) <= 1e-4
    lat.close()


def test_film_electrode_slab_parity():
    """A film-electrode slab (separated monodisperse particles in each
    electrode) with bulk reservoirs and three regions, BF16 weights and MSD
    along x: FID, populations and region FIDs against the matched oracle."""
    inp = lpc_inputs.film_supercapacitor(nx=152, ny=40, nz=40, electrode=60, bulk=32, steps=200)
    inp.alpha = 0.4
    inp.reservoirs = ((0.0, 1.0, 1.0), (0.0, 1.0, 1.0), None, None, None, None)
    lab, names = lpc_inputs.region_labels(inp)
    for sched in ("auto", "tb1"):
        lat = _lattice(inp, sched, region=lab, n_regions=3)
        lat.step(inp.steps)
        o = oracle.run(oracle.pack_input(inp, oracle.MODE_BF16), inp.uniform_rho0(), inp.steps, msd_axes=1,
                       region=lab, n_regions=3)
        assert H.rel_l2(lat.fid(), o.M) <= 1e-5
        assert H.rel_l2(lat.density().astype(np.float64), o.rho) <= 1e-5
        for r in range(3):
            assert H.rel_l2(lat.fid_region(r), o.Mr[r]) <= 1e-5
        lat.close()


@pytest.mark.parametrize("sched", ["tb1", "step1"])
def test_region_edge_cases(sched):
    """One region covering every site gives the totals (bit for bit in the
    fused kernel, where the totals are the sum over regions); a label that no
    site carries gives an all-zero history."""
    from paper_2603_22553_b300 import binding as B
    shape = (24, 48, 160)
    inp = lpc_inputs.random_case(shape, 351, periodic=(1, 1, 1), alpha=0.6, msd_axes=1)
    lab = np.zeros(shape, np.uint8)
    lat = _lattice(inp, sched, region=lab, n_regions=2)
    fused = lat.info()["kernel"] == B.LPC_KERNEL_TB
    lat.step(40)
    M, P = lat.fid(), lat.population()
    if fused:
        assert np.array_equal(lat.fid_region(0)[1:], M[1:])
        assert np.array_equal(lat.population_region(0)[1:], P[1:])
    else:
        assert np.max(np.abs(lat.fid_region(0) - M)) <= 1e-6 * P[0]
    assert np.all(lat.fid_region(1) == 0) and np.all(lat.population_region(1) == 0)
    assert np.all(lat.msd_region(1, 0) == 0)
    lat.close()


@pytest.mark.parametrize("sched", ["tb1", "step1"])
def test_equilibration_then_region_sums(sched):
    """The equilibration phase on a lattice with reservoirs and regions, then
    the propagation phase: region FIDs and populations from the restart
    against the oracle run from the equilibrated populations."""
    shape = (16, 32, 96)
    inp = lpc_inputs.random_case(shape, 361, periodic=(0, 1, 1), solid_frac=0.1, F_sd=0.8, alpha=0.9, msd_axes=1)
    inp.reservoirs = ((0.0, 1.0, 1.0), (-0.5, 0.75, 0.5j), None, None, None, None)
    lab = lpc_inputs.random_regions(shape, 362, 3)
    lat = _lattice(inp, sched, region=lab, n_regions=3)
    it, _ = lat.equilibrate(0.0, 2000, check_every=500)
    assert it == 2000 and lat.steps_done == 0
    rho = lat.density().astype(np.float64)
    steps = 60
    lat.step(steps)
    o = oracle.run(oracle.pack_input(inp, oracle.MODE_F32), rho, steps, msd_axes=1, region=lab, n_regions=3)
    assert H.rel_l2(lat.fid(), o.M) <= 1e-5
    for r in range(3):
        assert H.rel_l2(lat.fid_region(r), o.Mr[r]) <= 1e-5
        assert H.rel_l2(lat.population_region(r), o.Pr[r]) <= 1e-5
    lat.close()


# Reservoirs on z faces: the paper's supercapacitor is non-periodic in z
# (Sec. 4).  The library keeps a z reservoir as a halo plane below or above
# the own planes; results must equal the oracle's reservoir rule.
RES_Z = (None, None, None, None, (-0.25, 1.5, 0.75 + 0.5j), (0.75, 0.5, 0.25 - 0.5j))


@pytest.mark.parametrize("sched", ["auto", "step1", "tb1", "batch"])
@pytest.mark.parametrize("faces", ["z", "z_low_only", "xz"])
def test_z_face_reservoir_parity(sched, faces):
    from paper_2603_22553_b300.lattice import Lattice
    shape = (24, 30, 100)
    per = {"z": (1, 1, 0), "z_low_only": (1, 0, 0), "xz": (0, 1, 0)}[faces]
    inp = lpc_inputs.random_case(shape, 321, periodic=per, alpha=0.8, msd_axes=7)
    res = list(RES_Z)
    if faces == "z_low_only":
        res[5] = None
    if faces == "xz":
        res[0], res[1] = RES[0], RES[1]
    inp.reservoirs = tuple(res)
    lat = _lattice(inp, sched)
    info = lat.info()
    assert info["n_sites"] == inp.n_sites
    pk = oracle.pack_input(inp, oracle.MODE_F32)
    w = lat.weights().reshape(6, -1).T.astype(np.float64)
    assert np.array_equal(w == 0, pk.w == 0), "link geometry differs"
    assert _ulp_diff(w, pk.w, 24).max() <= 1.0
    assert np.array_equal(lat.solid_mask(), inp.solid)
    steps = 150
    _advance(lat, sched, steps)
    g = _read(lat, 7)
    mus = [lat.moment(a).astype(np.float64) for a in range(3)]
    o = oracle.run(pk, inp.uniform_rho0(), steps, msd_axes=7)
    _compare_fid_pop(g, o, 1e-5)
    for a in range(3):
        sl = slice(10, None)
        assert np.max(np.abs(g["msd%d" % a][sl] - o.msd(a)[sl]) / np.abs(o.msd(a)[sl])) <= 1e-5
        assert H.rel_l2(mus[a], o.mu[a]) <= 1e-4
    assert abs(g["P"][-1] / g["P"][0] - 1.0) > 1e-3      # population flows through the z faces
    # a checkpoint taken now resumes bit for bit
    blob = lat.get_state()
    lat.step(7)
    ref = lat.density()
    lat.set_state(blob)
    lat.step(7)
    assert np.array_equal(lat.density(), ref)
    lat.close()


def test_z_face_reservoirs_grand_canonical_equilibrium():
    """Reservoirs at one (F_res, rho_res) on both z faces: rho_res
    exp(-(F - F_res)) is the fixed point, reached by the equilibration phase."""
    shape = (32, 8, 16)
    inp = lpc_inputs.random_case(shape, 322, periodic=(1, 1, 0), solid_frac=0.0, F_sd=0.7, alpha=1.0,
                                 msd_axes=0)
    F_res, rho_res = -0.5, 1.5
    inp.reservoirs = (None, None, None, None, (F_res, rho_res, 0.0), (F_res, rho_res, 0.0))
    lat = _lattice(inp, "auto")
    it, diff = lat.equilibrate(0.0, 40000, check_every=2000)
    assert it == 40000 and diff < 1e-5
    rho_eq = rho_res * np.exp(-(inp.F - F_res))
    assert H.rel_l2(lat.density().astype(np.float64), rho_eq) <= 1e-4
    lat.close()


def test_z_face_reservoir_with_regions_and_boltzmann_start():
    """Region sums over the own planes only (the reservoir planes belong to
    no region), and a Boltzmann start normalised over the own planes."""
    from paper_2603_22553_b300.lattice import Lattice
    shape = (16, 20, 70)
    inp = lpc_inputs.random_case(shape, 323, periodic=(1, 1, 0), alpha=0.9, msd_axes=4)
    inp.reservoirs = RES_Z
    lab = lpc_inputs.random_regions(shape, 324, 3)
    lat = Lattice.from_input(inp, region=lab, n_regions=3, init=1)
    rho_b = oracle.boltzmann(inp.F, inp.solid)
    assert H.rel_l2(lat.density().astype(np.float64), rho_b) <= 1e-6
    steps = 60
    lat.step(steps)
    pk = oracle.pack_input(inp, oracle.MODE_F32)
    o = oracle.run(pk, rho_b, steps, msd_axes=4, region=lab, n_regions=3)
    assert H.rel_l2(lat.fid(), o.M) <= 1e-5
    for r in range(3):
        assert H.rel_l2(lat.fid_region(r), o.Mr[r]) <= 1e-5
        assert H.rel_l2(lat.population_region(r), o.Pr[r]) <= 1e-5
    lat.close()
