"""Seeded synthetic inputs for the lattice-propagation workloads.

This module only prepares inputs: solid masks, site free energies F (in kT),
chemical shifts and the angular frequencies derived from them, initial
populations, and the request stream of the serving workload.  It holds none of
the method's arithmetic (no hop weights, no stencil, no reductions), so both
the FP64 oracle and the CUDA path can consume the same arrays.

Conventions
-----------
* Arrays are C-order ``[z][y][x]`` (x contiguous), shape ``(nz, ny, nx)``.
* Random draws use ``numpy.random.Generator(PCG64(seed))``.  Full arrays are
  drawn in a fixed order (mask, then F, then shift) before any masking, so the
  draws never depend on the mask.
* Correlated noise: N(0, 1) white noise, a periodic Gaussian filter of width
  sigma (in sites) applied through the FFT, rescaled to unit standard
  deviation, then mapped through the normal CDF to u in (0, 1).  A log-normal
  pore size exp(s*g) is monotone in g, so mapping u onto a range is the
  "log-normal pore-size field -> range" map of the workloads.
* Shifts are given in ppm and converted to angular frequency with the 19F
  Larmor frequency of a 300 MHz spectrometer (282 MHz, Sec. 4):
  omega = 2*pi*nu0*delta_ppm*1e-6 rad/s.
* Time step 5 us and residence time 1 ms (Sec. 4), so alpha = dt/tau = 0.005.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DT = 5.0e-6            # s, Sec. 4
NU0 = 282.0e6          # Hz, 19F at 300 MHz, Sec. 4
TAU = 1.0e-3           # s, residence time, Sec. 4
ALPHA = DT / TAU       # jump probability factor, Eq. 7 (alpha = dt / tau)
KT = 1.0


def ppm_to_omega(delta_ppm):
    """Chemical shift (ppm) -> angular frequency (rad/s) at nu0 = 282 MHz."""
    return 2.0 * math.pi * NU0 * np.asarray(delta_ppm, dtype=np.float64) * 1e-6


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def correlated_uniform(shape, sigma, rng):
    """Periodic Gaussian-filtered white noise mapped to u in (0, 1).

    Returns (u, g): g is the filtered field at unit standard deviation and
    u = Phi(g) with Phi the standard normal CDF.
    """
    import scipy.fft
    import scipy.special

    white = rng.standard_normal(shape)
    spec = scipy.fft.rfftn(white, workers=-1)
    kf = [np.fft.fftfreq(n) for n in shape[:-1]] + [np.fft.rfftfreq(shape[-1])]
    grids = np.meshgrid(*kf, indexing="ij", sparse=True)
    k2 = sum((2.0 * math.pi * g) ** 2 for g in grids)
    spec *= np.exp(-0.5 * sigma * sigma * k2)
    g = scipy.fft.irfftn(spec, s=shape, workers=-1)
    del spec
    g -= g.mean()
    sd = g.std()
    if sd > 0:
        g /= sd
    u = scipy.special.ndtr(g)
    return u, g


@dataclasses.dataclass
class LatticeInput:
    """One lattice problem: geometry, fields and run length."""
    name: str
    nx: int
    ny: int
    nz: int
    periodic: tuple            # (px, py, pz), 1 = periodic, 0 = wall
    alpha: float
    dt: float
    kT: float
    F: np.ndarray              # float64 (nz, ny, nx), kT units
    omega: np.ndarray          # float64 (nz, ny, nx), rad/s
    solid: np.ndarray          # uint8 (nz, ny, nx), 1 = solid
    rho0: np.ndarray | None    # float64 (nz, ny, nx) or None -> 1 on pore sites
    steps: int
    weight_dtype: int = 0      # 0 = FP32 weights, 1 = BF16 weights
    msd_axes: int = 0          # bitmask x=1, y=2, z=4
    regions: dict | None = None
    alpha_links: np.ndarray | None = None   # [3][nz][ny][nx]: alpha of the link to the +x/+y/+z neighbour
    # reservoir faces: 6 entries (face f = 2 a + side; side 0 below coordinate 0,
    # side 1 above n_a - 1), each None (wall) or (F_res, rho_res, m_res complex)
    reservoirs: tuple | None = None

    @property
    def n_sites(self):
        return self.nx * self.ny * self.nz

    def uniform_rho0(self):
        """rho0 = 1 on pore sites, 0 on solid sites."""
        return (self.solid == 0).astype(np.float64)


def particle(edge=32, seed=1, steps=2000, solid_frac=0.30, F_mean=-2.0, F_sd=1.0,
             shift_mean=-6.0, shift_sd=2.0, weight_dtype=0, msd_axes=7, alpha=ALPHA,
             shape=None, periodic=(1, 1, 1)):
    """Single carbon particle: Bernoulli solid mask, Gaussian F and shift.

    Default is the 32^3 particle: 30 % solid, F ~ N(-2, 1) kT and
    shift ~ N(-6, 2) ppm on pore sites, 0 on solid, rho0 = 1, 2000 steps.
    ``shape`` = (nz, ny, nx) overrides the cubic edge.
    """
    rng = _rng(seed)
    shp = tuple(shape) if shape is not None else (edge, edge, edge)
    solid = (rng.random(shp) < solid_frac).astype(np.uint8)
    F = rng.normal(F_mean, F_sd, shp)
    delta = rng.normal(shift_mean, shift_sd, shp)
    pore = solid == 0
    F = np.where(pore, F, 0.0)
    delta = np.where(pore, delta, 0.0)
    nz, ny, nx = shp
    return LatticeInput("particle", nx, ny, nz, tuple(periodic), alpha, DT, KT, F,
                        ppm_to_omega(delta), solid, None, steps, weight_dtype, msd_axes)


def particle_in_bath(edge=256, radius=80.0, seed=2, steps=10000, sigma=4.0,
                     weight_dtype=0, msd_axes=0, alpha=ALPHA):
    """Porous sphere of radius 80 in a 256^3 electrolyte bath, no solid sites.

    Inside: F = -4 (1 - u) kT, shift = -10 (1 - u) ppm with u from correlated
    noise (sigma 4 sites).  Outside (bulk): F = shift = 0.
    """
    rng = _rng(seed)
    shp = (edge, edge, edge)
    u, _ = correlated_uniform(shp, sigma, rng)
    c = (edge - 1) / 2.0
    i = np.arange(edge, dtype=np.float64) - c
    r2 = i[:, None, None] ** 2 + i[None, :, None] ** 2 + i[None, None, :] ** 2
    inside = r2 < radius * radius
    F = np.where(inside, -4.0 * (1.0 - u), 0.0)
    delta = np.where(inside, -10.0 * (1.0 - u), 0.0)
    solid = np.zeros(shp, np.uint8)
    return LatticeInput("particle_in_bath", edge, edge, edge, (1, 1, 1), alpha, DT, KT, F,
                        ppm_to_omega(delta), solid, None, steps, weight_dtype, msd_axes,
                        regions={"inside": inside})


def supercapacitor(nx=2048, ny=256, nz=256, electrode=896, bulk=256, seeds=(31, 32),
                   sigma=4.0, steps=5000, weight_dtype=1, msd_axes=1, alpha=ALPHA):
    """Electrode / bulk / electrode slab along x, walls at x = 0 and x = nx - 1.

    Each electrode has its own correlated field (its own seed) on its own
    sub-box; F = -4 (1 - u) kT and shift = -10 (1 - u) ppm there; the bulk
    separator has F = shift = 0.  No solid sites.  BF16 weights, MSD along x.
    """
    assert 2 * electrode + bulk == nx
    F = np.zeros((nz, ny, nx))
    delta = np.zeros((nz, ny, nx))
    x_lo = (0, electrode + bulk)
    for seed, x0 in zip(seeds, x_lo):
        u, _ = correlated_uniform((nz, ny, electrode), sigma, _rng(seed))
        F[:, :, x0:x0 + electrode] = -4.0 * (1.0 - u)
        delta[:, :, x0:x0 + electrode] = -10.0 * (1.0 - u)
        del u
    solid = np.zeros((nz, ny, nx), np.uint8)
    regions = {"electrode_minus": (0, electrode), "bulk": (electrode, electrode + bulk),
               "electrode_plus": (electrode + bulk, nx)}
    return LatticeInput("supercapacitor", nx, ny, nz, (0, 1, 1), alpha, DT, KT, F,
                        ppm_to_omega(delta), solid, None, steps, weight_dtype, msd_axes,
                        regions=regions)


def sphere_packing(box, radius, fraction, rng):
    """Centres of non-touching monodisperse spheres filling about ``fraction``
    of a box (nz, ny, nx): a cubic arrangement whose spacing per axis is the
    box edge over round(edge / a), a = radius (4 pi / (3 fraction))^(1/3)
    (the spacing at which the spheres take ``fraction`` of the volume), each
    centre moved by a seeded uniform jitter of at most half of the spacing's
    excess over 2 radius + 1, so that no site of one sphere is a neighbour of a
    site of another (sites belong to a sphere when their centres lie inside
    it).  Returns an array of (z, y, x) centres (floats, in sites)."""
    a = radius * (4.0 * math.pi / (3.0 * fraction)) ** (1.0 / 3.0)
    # per axis floor or ceil of edge / a (spacing >= 2 radius), the combination
    # whose sphere fraction is closest to the target
    opts = []
    for n in box:
        c = sorted({max(1, int(math.floor(n / a))), max(1, int(math.ceil(n / a)))})
        c = [k for k in c if n / k >= 2.0 * radius + 1.0] or [max(1, int(n // (2.0 * radius + 1.0)))]
        opts.append(c)
    vol = 4.0 / 3.0 * math.pi * radius ** 3
    cells = min(((i, j, k) for i in opts[0] for j in opts[1] for k in opts[2]),
                key=lambda c: abs(c[0] * c[1] * c[2] * vol / (box[0] * box[1] * box[2]) - fraction))
    spacing = [n / c for n, c in zip(box, cells)]
    gap = min(spacing) - (2.0 * radius + 1.0)
    if gap < 0:
        raise ValueError("spheres of this radius do not fit at this fraction")
    grids = np.meshgrid(*[(np.arange(c) + 0.5) * sp for c, sp in zip(cells, spacing)], indexing="ij")
    centres = np.stack([g.reshape(-1) for g in grids], axis=1)
    centres += rng.uniform(-0.5 * gap, 0.5 * gap, centres.shape) * 0.999
    return centres


def film_supercapacitor(nx=2048, ny=256, nz=256, electrode=896, bulk=256, seeds=(41, 42), radius=9.0,
                        fraction=0.38, sigma=4.0, steps=5000, weight_dtype=1, msd_axes=1, alpha=ALPHA):
    """Film electrodes (Sec. 4, Fig. 7 bottom): in each electrode slab along x,
    monodisperse porous carbon particles of radius 9 sites take 38 % of the
    volume, separated by bulk-like electrolyte; the separator is bulk.  Inside
    a particle F = -4 (1 - u) kT and shift = -10 (1 - u) ppm from the slab's
    own correlated field u (its own seed); elsewhere F = shift = 0.  No solid
    sites; x walls, y and z periodic (particles wrap across y and z).  The
    attribute ``particles`` marks the particle sites; ``regions`` are the
    three slabs, as for the monolith slab."""
    assert 2 * electrode + bulk == nx
    F = np.zeros((nz, ny, nx))
    delta = np.zeros((nz, ny, nx))
    particles = np.zeros((nz, ny, nx), bool)
    x_lo = (0, electrode + bulk)
    r2 = radius * radius
    ext = int(math.ceil(radius))
    off = np.arange(-ext, ext + 1)
    for seed, x0 in zip(seeds, x_lo):
        rng = _rng(seed)
        centres = sphere_packing((nz, ny, electrode), radius, fraction, rng)
        inside = np.zeros((nz, ny, electrode), bool)
        for cz, cy, cx in centres:
            iz, iy, ix = int(math.floor(cz)), int(math.floor(cy)), int(math.floor(cx))
            zz, yy, xx = np.meshgrid(iz + off, iy + off, ix + off, indexing="ij")
            d2 = (zz + 0.5 - cz) ** 2 + (yy + 0.5 - cy) ** 2 + (xx + 0.5 - cx) ** 2
            sel = (d2 < r2) & (xx >= 0) & (xx < electrode)
            inside[zz[sel] % nz, yy[sel] % ny, xx[sel]] = True
        u, _ = correlated_uniform((nz, ny, electrode), sigma, rng)
        F[:, :, x0:x0 + electrode] = np.where(inside, -4.0 * (1.0 - u), 0.0)
        delta[:, :, x0:x0 + electrode] = np.where(inside, -10.0 * (1.0 - u), 0.0)
        particles[:, :, x0:x0 + electrode] = inside
        del u
    solid = np.zeros((nz, ny, nx), np.uint8)
    regions = {"electrode_minus": (0, electrode), "bulk": (electrode, electrode + bulk),
               "electrode_plus": (electrode + bulk, nx)}
    inp = LatticeInput("film_supercapacitor", nx, ny, nz, (0, 1, 1), alpha, DT, KT, F,
                       ppm_to_omega(delta), solid, None, steps, weight_dtype, msd_axes, regions=regions)
    inp.particles = particles
    return inp


def monolith(edge=512, seed=5, steps=20000, sigma=4.0, solid_quantile=0.40,
             weight_dtype=0, msd_axes=0, alpha=ALPHA, sub=None):
    """Porous monolith: solid where a correlated field is below its 40 % quantile.

    A second correlated field u (drawn after the mask field) sets
    F = -5 (1 - u) kT and shift = -12 (1 - u) ppm on pore sites.
    ``sub`` = e (int) returns the periodic [0, e)^3 corner of the same fields.
    """
    rng = _rng(seed)
    shp = (edge, edge, edge)
    _, gm = correlated_uniform(shp, sigma, rng)
    thr = np.quantile(gm, solid_quantile) if edge <= 256 else _quantile_sample(gm, solid_quantile)
    solid = (gm < thr).astype(np.uint8)
    del gm
    u, _ = correlated_uniform(shp, sigma, rng)
    pore = solid == 0
    F = np.where(pore, -5.0 * (1.0 - u), 0.0)
    delta = np.where(pore, -12.0 * (1.0 - u), 0.0)
    del u
    name = "monolith"
    if sub is not None:
        F = np.ascontiguousarray(F[:sub, :sub, :sub])
        delta = np.ascontiguousarray(delta[:sub, :sub, :sub])
        solid = np.ascontiguousarray(solid[:sub, :sub, :sub])
        shp = (sub, sub, sub)
        name = "monolith_sub"
    nz, ny, nx = shp
    return LatticeInput(name, nx, ny, nz, (1, 1, 1), alpha, DT, KT, F, ppm_to_omega(delta),
                        solid, None, steps, weight_dtype, msd_axes)


def _quantile_sample(a, q):
    """Exact quantile by partition (avoids the full sort of a huge array)."""
    flat = a.reshape(-1)
    k = int(q * (flat.size - 1))
    return float(np.partition(flat, k)[k])


def random_case(shape, seed, periodic=(1, 1, 1), solid_frac=0.2, F_sd=1.0, shift_sd=5.0,
                alpha=0.5, steps=50, weight_dtype=0, msd_axes=7, dt=DT):
    """Small random lattice for tests: Bernoulli solid, Gaussian F and shift."""
    rng = _rng(seed)
    shp = tuple(shape)
    solid = (rng.random(shp) < solid_frac).astype(np.uint8)
    F = rng.normal(0.0, F_sd, shp)
    delta = rng.normal(0.0, shift_sd, shp)
    pore = solid == 0
    F = np.where(pore, F, 0.0)
    delta = np.where(pore, delta, 0.0)
    nz, ny, nx = shp
    return LatticeInput("random", nx, ny, nz, tuple(periodic), alpha, dt, KT, F,
                        ppm_to_omega(delta), solid, None, steps, weight_dtype, msd_axes)


@dataclasses.dataclass
class Request:
    """One lattice solve of the serving stream."""
    rid: int
    arrival_s: float
    edge: int
    steps: int
    seed: int

    def lattice(self, steps=None):
        return particle(edge=self.edge, seed=self.seed,
                        steps=self.steps if steps is None else steps, msd_axes=0)


def request_stream(n=1000, seed=4, edge_lo=24, edge_hi=192, steps_lo=1000, steps_hi=20000,
                   rate_per_s=50.0):
    """Serving stream: log-uniform cubic edges, uniform step counts, Poisson arrivals.

    Request i uses the particle fields of seed 1000 + i.
    """
    rng = _rng(seed)
    edges = np.rint(np.exp(rng.uniform(math.log(edge_lo), math.log(edge_hi), n))).astype(int)
    steps = rng.integers(steps_lo, steps_hi + 1, n)
    gaps = rng.exponential(1.0 / rate_per_s, n)
    t = np.cumsum(gaps) - gaps[0]
    return [Request(i, float(t[i]), int(edges[i]), int(steps[i]), 1000 + i) for i in range(n)]


CONFIGS = {
    "particle_32": lambda: particle(),
    "particle_in_bath_256": lambda: particle_in_bath(),
    "supercapacitor_2048x256x256": lambda: supercapacitor(),
    "monolith_512": lambda: monolith(),
    "monolith_512_sub64": lambda: monolith(sub=64),
    "film_supercapacitor_2048x256x256": lambda: film_supercapacitor(),
}


def symmetric_links(shape, seed, lo=0.2, hi=1.0):
    """Per-link jump factors alpha_ij = lo + (hi - lo) (u_i + u_j) / 2 from a
    seeded per-site field u ~ U(0, 1): symmetric in i and j by construction.

    Returns (u, links) with links[a][z, y, x] the factor of the link between
    the site and its +a neighbour (periodic wrap; links across a wall are never
    used)."""
    rng = _rng(seed)
    u = rng.random(tuple(shape))
    links = np.empty((3,) + tuple(shape))
    for a in range(3):
        nb = np.roll(u, -1, axis=2 - a)          # axis a of (x, y, z) is array axis 2 - a
        links[a] = lo + (hi - lo) * 0.5 * (u + nb)
    return u, links


def region_labels(inp):
    """Per-site region labels (uint8, shape (nz, ny, nx)) and their names from
    the workload's ``regions`` description: a boolean mask (label 1 where set,
    0 elsewhere, names ("outside", name)) or x ranges [x0, x1) (labels in the
    order given)."""
    shp = (inp.nz, inp.ny, inp.nx)
    lab = np.zeros(shp, np.uint8)
    if not inp.regions:
        return lab, ("all",)
    items = list(inp.regions.items())
    if len(items) == 1 and isinstance(items[0][1], np.ndarray):
        name, mask = items[0]
        lab[np.asarray(mask, dtype=bool)] = 1
        return lab, ("outside", name)
    names = []
    for r, (name, (x0, x1)) in enumerate(items):
        lab[:, :, x0:x1] = r
        names.append(name)
    return lab, tuple(names)


def random_regions(shape, seed, n_regions):
    """Random per-site labels in [0, n_regions) for tests."""
    return _rng(seed).integers(0, n_regions, tuple(shape)).astype(np.uint8)
