"""The downstream estimators of the package (host code, fed by the GPU's
histories) against the oracle's own, on oracle histories: spectra (Eq. 9),
D from the MSD (Eq. 6-7), the Kohn route (Eq. 4) and the diffusion of the
particles in a region.  The two sides are separate implementations."""
import numpy as np

import lpc_inputs
import oracle
from paper_2603_22553_b300 import downstream


def _run():
    shape = (6, 7, 8)
    inp = lpc_inputs.random_case(shape, 401, periodic=(1, 0, 1), solid_frac=0.15, F_sd=1.0, alpha=0.7)
    lab = lpc_inputs.random_regions(shape, 402, 3)
    rho_eq = oracle.boltzmann(inp.F, inp.solid)
    r = oracle.run(oracle.pack_input(inp), rho_eq, 120, msd_axes=7, region=lab, n_regions=3)
    return inp, r


def test_kohn_vacf_and_region_diffusion_agree_with_the_oracle():
    inp, r = _run()
    for a in range(3):
        msd = r.msd(a)
        assert np.allclose(downstream.vacf(msd), oracle.vacf(r.dmsd[a], r.P[0]), rtol=1e-9, atol=1e-14)
        assert np.allclose(downstream.kohn_diffusion(msd, inp.dt), oracle.kohn_diffusion(r.dmsd[a], r.P[0], inp.dt),
                           rtol=1e-9)
        D = downstream.diffusion(msd, inp.dt)
        assert np.allclose(D[1:], oracle.diffusion(msd, inp.dt)[1:], rtol=1e-12)
        for g in range(3):
            msd_r = np.concatenate([[0.0], np.cumsum(r.Dr[g, a])]) / r.P[0]
            assert np.allclose(downstream.region_diffusion(msd_r, r.Pr[g], r.P[0], inp.dt),
                               oracle.region_diffusion(r.Dr[g, a], r.Pr[g], inp.dt), rtol=1e-9)


def test_spectrum_agrees_with_the_oracle():
    inp, r = _run()
    f, ppm, S = downstream.spectrum(r.M, inp.dt, device="cpu")
    fo, So = oracle.spectrum(r.M, inp.dt)
    assert np.allclose(f, fo) and np.allclose(S, So, rtol=1e-12, atol=1e-12 * np.abs(So).max())
    assert np.allclose(ppm, f / 282.0e6 * 1e6)
