"""Quantities computed downstream of the step (Sec. 2.2-2.3, Sec. 3.2 item 5).

* NMR spectrum: Fourier transform of the FID (Eq. 9), numpy sign convention
  e^{-2 pi i k n / N}, unnormalised, fftshifted; frequencies in Hz and in ppm
  of the Larmor frequency nu0.  Computed with torch.fft (cuFFT on the GPU).
* Diffusion coefficient per axis: D_a(n) = MSD_a(n) / (2 n dt) (Eq. 6-7,
  one dimension per axis); the isotropic D is the mean over axes.
* Kohn route (Eq. 4): from an equilibrium start the displacement
  autocorrelations are the second differences of the MSD; the truncated sum
  D_n = <dx^2>/(2 dt) + (1/dt) sum_{j=2}^{n+1} <dx_1 dx_j>.
* Diffusion of the particles in a region: D_r(n) = dMSD_r(n) / (2 dt P_r(n)).
* Density profiles (sum over the other two axes) and adsorbed amounts
  (population summed over a slab), as in Sec. 4.1.
"""
from __future__ import annotations

import numpy as np


def spectrum(M, dt, nu0=282.0e6, device=None):
    """Return (freq_hz, freq_ppm, S) with S = fftshift(FFT(M))."""
    import torch
    dev = device or ("cuda" if torch.cuda.is_available() else "cpu")
    m = torch.as_tensor(np.asarray(M, dtype=np.complex128), device=dev)
    S = torch.fft.fftshift(torch.fft.fft(m)).cpu().numpy()
    f = np.fft.fftshift(np.fft.fftfreq(len(M), d=dt))
    return f, f / nu0 * 1e6, S


def diffusion(msd, dt):
    """D(n) = MSD(n) / (2 n dt); D(0) is NaN."""
    msd = np.asarray(msd, dtype=np.float64)
    n = np.arange(len(msd), dtype=np.float64)
    D = np.full(len(msd), np.nan)
    D[1:] = msd[1:] / (2.0 * n[1:] * dt)
    return D


def density_profile(rho, axis="x"):
    """Sum of the populations over the two other axes (rho is [z][y][x])."""
    ax = {"x": (0, 1), "y": (0, 2), "z": (1, 2)}[axis]
    return np.asarray(rho, dtype=np.float64).sum(axis=ax)


def adsorbed_amount(rho, x_range):
    """Population summed over the slab x in [x0, x1) (an electrode region)."""
    x0, x1 = x_range
    return float(np.asarray(rho[:, :, x0:x1], dtype=np.float64).sum())


def _increments(msd):
    """dMSD(n) / P(0) = MSD(n + 1) - MSD(n) for n = 0 .. len(msd) - 2."""
    return np.diff(np.asarray(msd, dtype=np.float64))


def vacf(msd):
    """<dx_1 dx_(m+1)> for m = 0 .. len(msd) - 2 from an MSD history started in
    equilibrium: c_0 = MSD(1), c_m = (MSD(m+1) - 2 MSD(m) + MSD(m-1)) / 2."""
    d = _increments(msd)
    c = np.empty(len(d))
    c[0] = d[0]
    c[1:] = 0.5 * np.diff(d)
    return c


def kohn_diffusion(msd, dt):
    """Eq. 4 truncated after n + 1 displacements, n = 0 .. len(msd) - 2."""
    c = vacf(msd)
    return (np.cumsum(c) - 0.5 * c[0]) / dt


def region_diffusion(msd_region, population_region, P0, dt):
    """D of the particles in a region at step n: the region's MSD increment
    (lattice_msd_region is normalised by P(0)) per particle in the region."""
    d = _increments(msd_region) * P0
    P = np.asarray(population_region, dtype=np.float64)[:len(d)]
    return d / (2.0 * dt * P)
