"""FP64 CPU oracle of the LPC3D lattice step (arXiv 2603.22553).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library ``paper_2603_22553_b300``; both consume the seeded
inputs of ``lpc_inputs``.

The arithmetic lives in ``lpc_oracle.c`` (plain triple loops, FP64); this
module marshals numpy arrays into it and adds the plain downstream formulas:

* ``pack``: hop weights w_k (Eq. 1, Sec. 2.1, alpha of Eq. 7), stay weights
  s = 1 - sum_k w_k, rotation factors R = exp(i omega dt).
* ``run``: the step recursion (Eq. 13 in 3D with the stay term) for the
  population, the complex magnetisation and the first displacement moments,
  with the per-step sums M(n) (Eq. 12), P(n) and the MSD increments (Eq. 5).
* ``msd``: MSD_a(n) = sum_{j<n} dMSD_a(j) / P(0); ``diffusion``: D = MSD/(2 n dt)
  per axis (Eq. 6-7).
* ``vacf`` / ``kohn_diffusion``: the displacement autocorrelations and the
  truncated Kohn sum of Eq. 4 from an equilibrium start; ``region_diffusion``:
  D of the particles in a region.
* ``spectrum``: the plain DFT of M (Eq. 9), numpy's e^{-2 pi i k n / N}.
* ``boltzmann``: the equilibrium densities of Eq. 2 over pore sites.
* reservoir faces (Sec. 3.2 item 1: fixed field values in the ghost layer of a
  non-periodic face) and region-resolved sums M_r, P_r, dMSD_a,r (the
  spectra and diffusion of separate parts of the system, Sec. 4).

Parity pins are in ``tests/test_oracle_pins.py``.  The physics outputs of the
paper's Sec. 4 (D/D_bulk in Table 1, spectral peaks of Fig. 9) need the
missing MD/DFT parametrisation: parity unpinned for those (out of scope).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lpc_oracle.c")
_SO = os.path.join(_HERE, "liblpc_oracle.so")
_lib = None

MODE_EXACT, MODE_F32, MODE_BF16 = 0, 1, 2


def build(force=False):
    """Compile the oracle with gcc (-O2 -fopenmp), in place."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _bind(_SO)
    return _lib


def _bind(path):
    """Load a compiled oracle library from ``path`` and declare its signatures."""
    if True:
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.or_pack.argtypes = [ctypes.c_int] * 3 + [ip, ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_double, ctypes.c_int, dp, dp, u8p,
                                                     dp, dp, dp]
        lib.or_pack.restype = ctypes.c_int
        lib.or_pack_links.argtypes = [ctypes.c_int] * 3 + [ip, ctypes.c_double, dp, ctypes.c_double,
                                                           ctypes.c_double, ctypes.c_int, dp, dp, u8p,
                                                           dp, dp, dp]
        lib.or_pack_links.restype = ctypes.c_int
        lib.or_run.argtypes = [ctypes.c_int] * 3 + [ip, dp, dp, dp, ctypes.c_int, ctypes.c_int64,
                                                    ctypes.c_int, dp, dp, dp, dp, dp, dp]
        lib.or_run.restype = ctypes.c_int
        lib.or_pack_ex.argtypes = [ctypes.c_int] * 3 + [ip, ctypes.c_double, dp, ctypes.c_double,
                                                        ctypes.c_double, ctypes.c_int, dp, dp, u8p,
                                                        dp, dp, dp, dp, dp]
        lib.or_pack_ex.restype = ctypes.c_int
        lib.or_run_ex.argtypes = [ctypes.c_int] * 3 + [ip, dp, dp, dp, dp, dp, u8p, ctypes.c_int,
                                                       ctypes.c_int, ctypes.c_int64, ctypes.c_int,
                                                       dp, dp, dp, dp, dp, dp, dp, dp, dp]
        lib.or_run_ex.restype = ctypes.c_int
        lib.or_boltzmann.argtypes = [ctypes.c_int64, dp, u8p, ctypes.c_double, ctypes.c_double, dp]
        lib.or_boltzmann.restype = ctypes.c_int
        lib.or_round_f32.argtypes = [ctypes.c_double]
        lib.or_round_f32.restype = ctypes.c_double
        lib.or_round_bf16.argtypes = [ctypes.c_double]
        lib.or_round_bf16.restype = ctypes.c_double
        lib.or_max_threads.restype = ctypes.c_int
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class Packed:
    """Weights w[N, 6] (k = +x, -x, +y, -y, +z, -z), stay s[N], rotation R[N]
    (complex); with reservoir faces also res[6, 5] and the reservoir
    in-weights wres[N, 6]."""

    def __init__(self, shape, periodic, w, s, R, res=None, wres=None):
        self.shape = shape
        self.periodic = periodic
        self.w = w
        self.s = s
        self.R = R
        self.res = res
        self.wres = wres


def reservoir_table(reservoirs):
    """[6, 5] table {enabled, F_res, rho_res, m_res re, m_res im} per face
    f = 2 a + side (side 0 below coordinate 0, side 1 above n_a - 1) from a
    sequence of 6 entries, each None or (F_res, rho_res, m_res)."""
    if reservoirs is None:
        return None
    t = np.zeros((6, 5))
    for f, e in enumerate(reservoirs):
        if e is None:
            continue
        F_res, rho_res, m_res = e
        t[f] = (1.0, F_res, rho_res, complex(m_res).real, complex(m_res).imag)
    return t


def pack(nx, ny, nz, periodic, alpha, dt, kT, F, omega, solid, mode=MODE_EXACT, alpha_links=None,
         reservoirs=None):
    """Hop weights of Eq. 1 times alpha/6 (alpha_links: optional [3][nz][ny][nx]
    per-link factors, link between a site and its +x, +y, +z neighbour;
    reservoirs: optional 6 faces, see ``reservoir_table``)."""
    lib = _load()
    N = nx * ny * nz
    F = _c64(F, (N,))
    omega = _c64(omega, (N,))
    solid = np.ascontiguousarray(solid, dtype=np.uint8).reshape(N)
    w = np.empty((N, 6))
    s = np.empty(N)
    R = np.empty((N, 2))
    per = (ctypes.c_int * 3)(*[int(p) for p in periodic])
    links = None if alpha_links is None else _c64(alpha_links, (3 * N,))
    res = reservoir_table(reservoirs)
    wres = None if res is None else np.empty((N, 6))
    rc = lib.or_pack_ex(nx, ny, nz, per, float(alpha), None if links is None else _dp(links),
                        float(dt), float(kT), int(mode), _dp(F), _dp(omega),
                        solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                        None if res is None else _dp(res), _dp(w), _dp(s), _dp(R),
                        None if wres is None else _dp(wres))
    if rc != 0:
        raise ValueError("oracle pack rejected its inputs")
    return Packed((nz, ny, nx), tuple(int(p) for p in periodic), w, s, R[:, 0] + 1j * R[:, 1], res, wres)


def pack_input(inp, mode=MODE_EXACT):
    """``pack`` on an ``lpc_inputs.LatticeInput``."""
    return pack(inp.nx, inp.ny, inp.nz, inp.periodic, inp.alpha, inp.dt, inp.kT, inp.F,
                inp.omega, inp.solid, mode, getattr(inp, "alpha_links", None),
                getattr(inp, "reservoirs", None))


class Result:
    """Final state and per-step histories of an oracle run."""

    def __init__(self, rho, m, mu, M, P, dmsd, msd_axes, Mr=None, Pr=None, Dr=None):
        self.rho = rho          # (nz, ny, nx) float64
        self.m = m              # (nz, ny, nx) complex128
        self.mu = mu            # (3, nz, ny, nx) float64
        self.M = M              # (steps+1,) complex128
        self.P = P              # (steps+1,) float64
        self.dmsd = dmsd        # (3, steps) float64
        self.msd_axes = msd_axes
        self.Mr = Mr            # (n_regions, steps+1) complex128, or None
        self.Pr = Pr            # (n_regions, steps+1) float64
        self.Dr = Dr            # (n_regions, 3, steps) float64

    def msd(self, axis):
        """MSD_a(n), n = 0..steps."""
        return msd(self.dmsd[axis], self.P[0])


def run(packed, rho0, steps, m0=None, mu0=None, msd_axes=7, nthreads=0, region=None, n_regions=0):
    """Run ``steps`` steps from rho0 (m0 = rho0 and mu0 = 0 unless given).
    region: optional [nz][ny][nx] labels < n_regions for region-resolved sums."""
    lib = _load()
    nz, ny, nx = packed.shape
    N = nx * ny * nz
    rho = _c64(rho0, (N,)).copy()
    if m0 is None:
        m = np.zeros((N, 2))
        m[:, 0] = rho
    else:
        m0 = np.asarray(m0, dtype=np.complex128).reshape(N)
        m = np.ascontiguousarray(np.stack([m0.real, m0.imag], axis=1))
    mu = np.zeros((3, N)) if mu0 is None else _c64(mu0, (3, N)).copy()
    w = np.ascontiguousarray(packed.w, dtype=np.float64)
    s = np.ascontiguousarray(packed.s, dtype=np.float64)
    R = np.ascontiguousarray(np.stack([packed.R.real, packed.R.imag], axis=1))
    M = np.zeros((steps + 1, 2))
    P = np.zeros(steps + 1)
    dmsd = np.zeros((3, max(steps, 1)))
    per = (ctypes.c_int * 3)(*packed.periodic)
    res = packed.res
    wres = None if packed.wres is None else np.ascontiguousarray(packed.wres, dtype=np.float64)
    reg = None
    nr = 0
    if region is not None:
        reg = np.ascontiguousarray(region, dtype=np.uint8).reshape(N)
        nr = int(n_regions)
    Mr = np.zeros((max(nr, 1), steps + 1, 2))
    Pr = np.zeros((max(nr, 1), steps + 1))
    Dr = np.zeros((max(nr, 1), 3, max(steps, 1)))
    rc = lib.or_run_ex(nx, ny, nz, per, _dp(w), _dp(s), _dp(R),
                       None if wres is None else _dp(wres), None if res is None else _dp(res),
                       None if reg is None else reg.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                       nr, int(msd_axes), int(steps), int(nthreads), _dp(rho), _dp(m), _dp(mu),
                       _dp(M), _dp(P), _dp(dmsd), _dp(Mr), _dp(Pr), _dp(Dr))
    if rc != 0:
        raise ValueError("oracle run rejected its inputs")
    extra = {}
    if nr:
        extra = dict(Mr=Mr[..., 0] + 1j * Mr[..., 1], Pr=Pr, Dr=Dr[:, :, :steps])
    return Result(rho.reshape(nz, ny, nx), (m[:, 0] + 1j * m[:, 1]).reshape(nz, ny, nx),
                  mu.reshape(3, nz, ny, nx), M[:, 0] + 1j * M[:, 1], P, dmsd[:, :steps],
                  msd_axes, **extra)


def boltzmann(F, solid, kT=1.0, mean_rho=1.0):
    """Eq. 2 over pore sites: rho_i = <rho> n_pore e^{-F_i/kT} / sum_j e^{-F_j/kT}."""
    lib = _load()
    shape = np.shape(F)
    F = _c64(F).reshape(-1)
    solid = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
    rho = np.empty_like(F)
    rc = lib.or_boltzmann(F.size, _dp(F), solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                          float(kT), float(mean_rho), _dp(rho))
    if rc != 0:
        raise ValueError("no pore site")
    return rho.reshape(shape)


def msd(dmsd_axis, P0):
    """MSD(n) = sum_{j<n} dMSD(j) / P(0) for n = 0..len(dmsd)."""
    out = np.zeros(len(dmsd_axis) + 1)
    np.cumsum(dmsd_axis, out=out[1:])
    return out / P0


def diffusion(msd_n, dt):
    """D(n) = MSD(n) / (2 n dt) per axis (Eq. 6-7 with d = 1 per axis), n >= 1."""
    n = np.arange(len(msd_n), dtype=np.float64)
    D = np.full(len(msd_n), np.nan)
    D[1:] = msd_n[1:] / (2.0 * n[1:] * dt)
    return D


def vacf(dmsd_axis, P0):
    """Displacement autocorrelations of Eq. 4 from the MSD increments of a run
    started in equilibrium (a stationary walk): c_0 = <dx_1^2> = dMSD(0)/P0 and,
    for m >= 1, c_m = <dx_1 dx_(m+1)> = (dMSD(m) - dMSD(m-1)) / (2 P0), since
    MSD(n) = n c_0 + 2 sum_{m=1}^{n-1} (n - m) c_m."""
    d = np.asarray(dmsd_axis, dtype=np.float64) / P0
    c = np.empty(len(d))
    c[0] = d[0]
    c[1:] = 0.5 * (d[1:] - d[:-1])
    return c


def kohn_diffusion(dmsd_axis, P0, dt):
    """Eq. 4 truncated after n + 1 displacements:
    D_n = <dx^2> / (2 dt) + (1/dt) sum_{j=2}^{n+1} <dx_1 dx_j>, n = 0 .. len - 1."""
    c = vacf(dmsd_axis, P0)
    D = np.empty(len(c))
    acc = c[0] / (2.0 * dt)
    D[0] = acc
    for n in range(1, len(c)):
        acc += c[n] / dt
        D[n] = acc
    return D


def region_diffusion(dmsd_region_axis, P_region, dt):
    """Diffusion coefficient of the particles in a region at step n:
    D_r(n) = dMSD_r(n) / (2 dt P_r(n)), the MSD increment of the particles that
    are in region r at step n per particle (one axis)."""
    d = np.asarray(dmsd_region_axis, dtype=np.float64)
    P = np.asarray(P_region, dtype=np.float64)[:len(d)]
    return d / (2.0 * dt * P)


def spectrum(M, dt):
    """Plain DFT of the FID (Eq. 9), fftshifted; returns (freq_hz, S)."""
    S = np.fft.fftshift(np.fft.fft(np.asarray(M, dtype=np.complex128)))
    f = np.fft.fftshift(np.fft.fftfreq(len(M), d=dt))
    return f, S


def round_f32(v):
    return _load().or_round_f32(float(v))


def round_bf16(v):
    return _load().or_round_bf16(float(v))


def max_threads():
    return _load().or_max_threads()
