"""Parity at the full workload sizes.

* 512^3 monolith (the benchmark workload, in the schedule bench.py times):
  after n steps the value at a site depends only on the sites within L1
  distance n and on their hop weights, which depend on sites one further
  out.  The FP64 oracle run on a box of half-width n + 2 around a sampled
  site (walls on the box faces) therefore gives that site's exact value;
  sampled sites, including ones near the periodic faces, are compared one by
  one.  Conservation and |M| <= P(0) hold at any size.
* Precision sweep on the 64^3 corner of the same fields, 20 000 steps: FP32
  and BF16 hop weights against the FP64 oracle with exact weights and with
  its own rounding of the weights; the spectrum error equals the FID error
  (the DFT is unitary up to sqrt(N)).
"""
import numpy as np
import pytest

import lpc_inputs
import oracle
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def monolith512():
    return lpc_inputs.monolith(edge=512)


def _box(a, z, y, x, r):
    idx = [np.arange(c - r, c + r + 1) for c in (z, y, x)]
    return a.take(idx[0], axis=0, mode="wrap").take(idx[1], axis=1, mode="wrap").take(idx[2], axis=2, mode="wrap")


def test_monolith_512_sampled_sites(monolith512):
    from paper_2603_22553_b300.lattice import Lattice
    inp = monolith512
    n = 6
    lat = Lattice.from_input(inp)          # default schedule, as benchmarked
    lat.step(n)
    rho = lat.density()
    m = lat.magnetization()
    P = lat.population()
    M = lat.fid()
    assert np.max(np.abs(P / P[0] - 1.0)) <= 1e-5
    assert np.all(np.abs(M) <= P[0] * (1 + 1e-6))
    rng = np.random.default_rng(11)
    pts = [(0, 0, 0), (511, 511, 511), (0, 255, 511), (3, 508, 1), (256, 0, 300)]
    pts += [tuple(int(v) for v in rng.integers(0, 512, 3)) for _ in range(35)]
    r = n + 2
    worst = 0.0
    for (z, y, x) in pts:
        Fb = _box(inp.F, z, y, x, r)
        Ob = _box(inp.omega, z, y, x, r)
        Sb = _box(inp.solid, z, y, x, r)
        e = 2 * r + 1
        pk = oracle.pack(e, e, e, (0, 0, 0), inp.alpha, inp.dt, inp.kT, Fb, Ob, Sb, oracle.MODE_F32)
        res = oracle.run(pk, (Sb == 0).astype(np.float64), n, msd_axes=0)
        ref_r = res.rho[r, r, r]
        ref_m = res.m[r, r, r]
        scale = max(1.0, abs(ref_r))
        err = max(abs(rho[z, y, x] - ref_r), abs(m[z, y, x] - ref_m)) / scale
        worst = max(worst, err)
    assert worst <= 1e-5, worst
    lat.close()


def test_monolith_512_schedules_agree(monolith512):
    """The one-step kernels (register-pipelined and TMA-fed) give bit-identical
    states and FID within FP32 rounding at full size."""
    from paper_2603_22553_b300 import binding as B
    from paper_2603_22553_b300.lattice import Lattice
    inp = monolith512
    a = Lattice.from_input(inp)
    a.set_schedule(B.LPC_KERNEL_TB, 1)
    a.step(5)
    da, ma, Ma = a.density(), a.magnetization(), a.fid()
    a.close()
    b = Lattice.from_input(inp)
    b.set_schedule(B.LPC_KERNEL_STEP1, 1)
    b.step(5)
    assert np.array_equal(da, b.density())
    assert np.array_equal(ma, b.magnetization())
    assert np.allclose(Ma, b.fid(), rtol=1e-6, atol=1e-6 * abs(Ma[0]))
    b.close()


def test_precision_sweep_64_subvolume(monolith512):
    """FP32 state with FP32 or BF16 weights, 20 000 steps, vs the FP64 oracle."""
    sub = lpc_inputs.LatticeInput("monolith_sub64", 64, 64, 64, (1, 1, 1), monolith512.alpha,
                                  monolith512.dt, monolith512.kT,
                                  np.ascontiguousarray(monolith512.F[:64, :64, :64]),
                                  np.ascontiguousarray(monolith512.omega[:64, :64, :64]),
                                  np.ascontiguousarray(monolith512.solid[:64, :64, :64]), None, 20000,
                                  0, 0)
    steps = 20000
    exact = H.oracle_run(sub, steps, oracle.MODE_EXACT)
    report = {}
    for wdt, mode in ((0, oracle.MODE_F32), (1, oracle.MODE_BF16)):
        sub.weight_dtype = wdt
        g = H.gpu_run(sub, steps)
        matched = H.oracle_run(sub, steps, mode)
        e_matched = H.rel_l2(g["M"], matched.M)
        e_exact = H.rel_l2(g["M"], exact.M)
        _, S_g = oracle.spectrum(g["M"], sub.dt)
        _, S_o = oracle.spectrum(matched.M, sub.dt)
        e_spec = H.rel_l2(S_g, S_o)
        report[wdt] = (e_matched, e_exact, e_spec)
        assert e_matched <= 1e-4 and e_spec <= 1e-4
        assert H.rel_l2(g["rho"], matched.rho) <= 1e-4
        if wdt == 0:
            assert e_exact <= 1e-4
        g["lattice"].close()
    print("precision sweep (FID matched, FID exact, spectrum):", report)


def _box_axes(a, center, r, periodic):
    """The box of half-width r around `center` (z, y, x): wrapped on periodic
    axes, cut at the lattice faces on walled ones.  Returns the box and the
    centre's index in it."""
    out = a
    idx_c = []
    for ax, (c, per) in enumerate(zip(center, periodic)):
        n = a.shape[ax]
        if per:
            idx = np.arange(c - r, c + r + 1) % n
            idx_c.append(r)
        else:
            lo, hi = max(0, c - r), min(n, c + r + 1)
            idx = np.arange(lo, hi)
            idx_c.append(c - lo)
        out = out.take(idx, axis=ax)
    return out, tuple(idx_c)


def test_supercapacitor_full_size_sampled_sites():
    """The 2048x256x256 slab (BF16 weights, first moment along x, walls in x)
    in the schedule bench.py times: sampled sites (at the walls, at the
    electrode/bulk interfaces and at random) against the FP64 oracle on a
    box of half-width n + 2 with walls on its faces (the walls at the box
    faces are farther than n sites from the centre; where the box is cut by
    the real walls, they are the same walls)."""
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.supercapacitor()
    n = 6
    lat = Lattice.from_input(inp)
    lat.step(n)
    rho, m, mu = lat.density(), lat.magnetization(), lat.moment(0)
    P = lat.population()
    assert np.max(np.abs(P / P[0] - 1.0)) <= 1e-5
    rng = np.random.default_rng(12)
    pts = [(0, 0, 0), (255, 255, 2047), (7, 100, 895), (9, 3, 896), (200, 50, 1151), (1, 254, 1152),
           (128, 128, 1), (60, 0, 2046)]
    pts += [(int(rng.integers(0, 256)), int(rng.integers(0, 256)), int(rng.integers(0, 2048))) for _ in range(24)]
    r = n + 2
    per = (1, 1, 0)            # z, y periodic; x walls (array axes z, y, x)
    worst = 0.0
    for c in pts:
        Fb, cc = _box_axes(inp.F, c, r, per)
        Ob, _ = _box_axes(inp.omega, c, r, per)
        Sb, _ = _box_axes(inp.solid, c, r, per)
        nzb, nyb, nxb = Fb.shape
        pk = oracle.pack(nxb, nyb, nzb, (0, 0, 0), inp.alpha, inp.dt, inp.kT, Fb, Ob, Sb, oracle.MODE_BF16)
        res = oracle.run(pk, (Sb == 0).astype(np.float64), n, msd_axes=1)
        z, y, x = c
        scale = max(1.0, abs(res.rho[cc]))
        err = max(abs(rho[z, y, x] - res.rho[cc]), abs(m[z, y, x] - res.m[cc]),
                  abs(mu[z, y, x] - res.mu[0][cc])) / scale
        worst = max(worst, err)
    assert worst <= 1e-5, worst
    lat.close()


def test_particle_in_bath_256_sampled_sites():
    """The 256^3 bath (porous sphere of radius 80 in electrolyte) in the
    benchmarked schedule: sampled sites inside the sphere, at its surface, in
    the bath and at the periodic faces against the FP64 oracle on boxes."""
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.particle_in_bath()
    n = 6
    lat = Lattice.from_input(inp)
    lat.step(n)
    rho, m = lat.density(), lat.magnetization()
    P = lat.population()
    assert np.max(np.abs(P / P[0] - 1.0)) <= 1e-5
    rng = np.random.default_rng(13)
    pts = [(0, 0, 0), (255, 255, 255), (128, 128, 128), (128, 128, 48), (128, 48, 128), (40, 128, 128),
           (0, 128, 255), (200, 3, 77)]
    pts += [tuple(int(v) for v in rng.integers(0, 256, 3)) for _ in range(24)]
    r = n + 2
    worst = 0.0
    for c in pts:
        Fb, cc = _box_axes(inp.F, c, r, (1, 1, 1))
        Ob, _ = _box_axes(inp.omega, c, r, (1, 1, 1))
        Sb, _ = _box_axes(inp.solid, c, r, (1, 1, 1))
        e = 2 * r + 1
        pk = oracle.pack(e, e, e, (0, 0, 0), inp.alpha, inp.dt, inp.kT, Fb, Ob, Sb, oracle.MODE_F32)
        res = oracle.run(pk, (Sb == 0).astype(np.float64), n, msd_axes=0)
        z, y, x = c
        err = max(abs(rho[z, y, x] - res.rho[cc]), abs(m[z, y, x] - res.m[cc])) / max(1.0, abs(res.rho[cc]))
        worst = max(worst, err)
    assert worst <= 1e-5, worst
    lat.close()


def _mem_available_gb():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 2 ** 20
    except OSError:
        pass
    return 0.0


def test_near_maximum_padded_size():
    """The largest lattices the library takes: 2040 x 1020 x 1020 sites, whose
    ghost-padded arrays hold 2^31 - 8.4e6 sites (the limit of the kernels'
    32-bit plane offsets); BF16 weights.  Two steps of the default schedule:
    populations conserved, and sampled sites near the far corner (the largest
    offsets) and elsewhere against the FP64 oracle on boxes."""
    import ctypes
    import torch
    from paper_2603_22553_b300 import binding as B
    from paper_2603_22553_b300.lattice import Lattice
    nx, ny, nz = 2040, 1020, 1020
    torch.cuda.empty_cache()
    p = B.lpc_params(nx, ny, nz, (ctypes.c_int32 * 3)(1, 1, 1), 0.6, 5e-6, 1.0, 1, 0, 0, 0)
    need = ctypes.c_int64()
    B.check(B.load().lattice_footprint(ctypes.byref(p), 8, ctypes.byref(need)))
    if torch.cuda.mem_get_info()[0] < need.value * 1.1 or _mem_available_gb() < 100:
        pytest.skip("needs %.0f GB of device memory and 100 GB of host memory" % (need.value / 1e9))
    N = nx * ny * nz
    rng = np.random.default_rng(21)
    F = rng.random(N, dtype=np.float64)
    F *= -2.0
    om = np.empty(N)
    np.multiply(F, 3.0e4, out=om)
    solid = np.zeros(N, np.uint8)
    solid[rng.integers(0, N, N // 10)] = 1
    shape = (nz, ny, nx)
    lat = Lattice(nx, ny, nz, F, om, solid, alpha=0.6, weight_dtype=1)
    n = 2
    lat.step(n)
    P = lat.population()
    assert np.max(np.abs(P / P[0] - 1.0)) <= 1e-5
    rho = lat.density()
    pts = [(nz - 1, ny - 1, nx - 1), (nz - 1, ny - 1, 0), (nz - 1, 0, nx - 1), (0, 0, 0), (nz - 2, ny - 3, nx - 5),
           (nz // 2, ny // 2, nx // 2), (nz - 1, ny // 3, 1000)]
    pts += [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(12)]
    r = n + 2
    F3, om3, so3 = F.reshape(shape), om.reshape(shape), solid.reshape(shape)
    worst = 0.0
    for c in pts:
        Fb, cc = _box_axes(F3, c, r, (1, 1, 1))
        Ob, _ = _box_axes(om3, c, r, (1, 1, 1))
        Sb, _ = _box_axes(so3, c, r, (1, 1, 1))
        e = 2 * r + 1
        pk = oracle.pack(e, e, e, (0, 0, 0), 0.6, 5e-6, 1.0, Fb, Ob, Sb, oracle.MODE_BF16)
        res = oracle.run(pk, (Sb == 0).astype(np.float64), n, msd_axes=0)
        worst = max(worst, abs(rho[c] - res.rho[cc]) / max(1.0, abs(res.rho[cc])))
    assert worst <= 1e-5, worst
    lat.close()


@pytest.mark.parametrize("cfg", [
    ((320, 400, 400), (1, 1, 1), 0, 0),
    ((320, 400, 400), (0, 1, 1), 1, 0),          # x walls, first moment along x
    ((320, 397, 403), (1, 0, 0), 7, 0),          # ragged x and y, y and z walls, every moment
    ((336, 389, 392), (1, 1, 1), 3, 0),          # ragged, x and y moments
])
def test_link_form_matches_register_pipelined_kernel(cfg):
    """FP32 lattices of more than 5e7 sites keep their static data in link form
    (one signed weight per link): the one-step TMA kernel rebuilds every hop
    and stay weight exactly, so its states equal those of the register-
    pipelined kernel bit for bit; the sums agree to FP32 rounding, and
    sampled sites agree with the FP64 oracle on boxes."""
    from paper_2603_22553_b300 import binding as B
    from paper_2603_22553_b300.lattice import Lattice
    shape, per, msd, wdt = cfg
    nz, ny, nx = shape
    rng = np.random.default_rng(sum(shape) + msd)
    F = rng.normal(-1.0, 1.0, shape)
    om = rng.normal(0.0, 3.0e4, shape)
    solid = (rng.random(shape) < 0.25).astype(np.uint8)
    n = 6
    out = []
    for sched in ((B.LPC_KERNEL_AUTO, 1), (B.LPC_KERNEL_STEP1, 1)):
        lat = Lattice(nx, ny, nz, F, om, solid, periodic=per, alpha=0.7, weight_dtype=wdt, msd_axes=msd)
        lat.set_schedule(*sched)
        lat.step(n)
        if sched[0] == B.LPC_KERNEL_AUTO:
            info = lat.info()
            assert info["kernel"] == B.LPC_KERNEL_TB and info["block_steps"] == 1 and info["static_form"] == 2
        res = dict(rho=lat.density(), m=lat.magnetization(), M=lat.fid(), P=lat.population())
        for a in range(3):
            if msd >> a & 1:
                res["mu%d" % a] = lat.moment(a)
                res["msd%d" % a] = lat.msd(a)
        out.append(res)
        lat.close()
    a, b = out
    assert np.array_equal(a["rho"], b["rho"]) and np.array_equal(a["m"], b["m"])
    assert np.allclose(a["M"], b["M"], rtol=1e-6, atol=1e-6 * abs(b["M"][0]))
    assert np.allclose(a["P"], b["P"], rtol=1e-6)
    for ax in range(3):
        if msd >> ax & 1:
            assert np.array_equal(a["mu%d" % ax], b["mu%d" % ax])
            assert np.allclose(a["msd%d" % ax][1:], b["msd%d" % ax][1:], rtol=1e-5)
    r = n + 2
    pts = [(nz - 1, ny - 1, nx - 1), (0, 0, 0), (nz // 2, 0, nx - 1)] + \
          [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(8)]
    for c in pts:
        Fb, cc = _box_axes(F, c, r, per[::-1])
        Ob, _ = _box_axes(om, c, r, per[::-1])
        Sb, _ = _box_axes(solid, c, r, per[::-1])
        nzb, nyb, nxb = Fb.shape
        pk = oracle.pack(nxb, nyb, nzb, (0, 0, 0), 0.7, 5e-6, 1.0, Fb, Ob, Sb, H.MODE_OF_DTYPE[wdt])
        res = oracle.run(pk, (Sb == 0).astype(np.float64), n, msd_axes=0)
        assert abs(a["rho"][c] - res.rho[cc]) <= 1e-5 * max(1.0, abs(res.rho[cc]))
