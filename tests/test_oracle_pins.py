"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here checks the oracle against something other than itself:
closed forms, invariants (conservation, detailed balance, the Boltzmann
steady state of Eq. 2), the Kohn identity of Eq. 4, brute-force dense matrix
powers and brute-force (site, displacement) distributions on tiny lattices,
and library routines (numpy FFT, numpy's binary32 cast).
"""
import math

import numpy as np
import pytest

import lpc_inputs
import oracle
from tests import bruteforce as bf


def _uniform_rho(inp):
    return inp.uniform_rho0()


# --------------------------------------------------------------------------
# rounding helpers used by the matched-input oracle mode
# --------------------------------------------------------------------------

def test_round_f32_matches_numpy_cast():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.random(2000) * 0.2, rng.random(200) * 1e-4, [1.0, 0.5, 1 / 3]])
    got = np.array([oracle.round_f32(x) for x in v])
    assert np.array_equal(got, v.astype(np.float32).astype(np.float64))


def test_round_bf16_matches_bit_rounding():
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.random(2000) * 0.2, rng.random(200) * 1e-3, [1.0, 1 / 3]])
    # exact ties: significand ...1|1000... and ...0|1000...
    ties = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 0.25 * (1.0 + 2.0 ** -8)])
    v = np.concatenate([v, ties])
    got = np.array([oracle.round_bf16(x) for x in v])
    assert np.array_equal(got, bf.bits_round(v, 45))
    assert np.array_equal(np.array([oracle.round_f32(x) for x in v]), bf.bits_round(v, 29))
    # ties go to the even neighbour
    assert oracle.round_bf16(1.0 + 2.0 ** -8) == 1.0
    assert oracle.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


# --------------------------------------------------------------------------
# weights: Eq. 1 detailed balance, walls, solids
# --------------------------------------------------------------------------

@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 1, 1), (1, 0, 0)])
def test_weights_detailed_balance_and_walls(periodic):
    inp = lpc_inputs.random_case((5, 6, 7), 11, periodic=periodic, solid_frac=0.25)
    pk = oracle.pack_input(inp)
    nz, ny, nx = inp.F.shape
    pi = np.exp(-inp.F.reshape(-1))
    w = pk.w
    solid = inp.solid.reshape(-1)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = (z * ny + y) * nx + x
                for k, off in enumerate(bf.OFFSETS):
                    j = bf._target(x, y, z, off, inp.F.shape, periodic)
                    if j is None or solid[i] or solid[j]:
                        assert w[i, k] == 0.0
                        continue
                    # detailed balance: pi_i w_k(i) = pi_j w_{-k}(j)
                    assert pi[i] * w[i, k] == pytest.approx(pi[j] * w[j, k ^ 1], rel=1e-14)
                    assert 0.0 < w[i, k] <= inp.alpha / 6.0
    assert np.allclose(pk.s, 1.0 - w.sum(axis=1), rtol=0, atol=1e-15)
    assert np.all(pk.s >= 1.0 - inp.alpha - 1e-15)


def test_pack_rounded_modes():
    inp = lpc_inputs.random_case((4, 5, 6), 12)
    ex = oracle.pack_input(inp, oracle.MODE_EXACT)
    f32 = oracle.pack_input(inp, oracle.MODE_F32)
    b16 = oracle.pack_input(inp, oracle.MODE_BF16)
    assert np.array_equal(f32.w, ex.w.astype(np.float32).astype(np.float64))
    pos = ex.w > 0
    assert np.array_equal(b16.w[pos], bf.bits_round(ex.w[pos], 45))
    assert np.allclose(b16.s, 1.0 - b16.w.sum(axis=1), atol=1e-15)
    assert np.array_equal(f32.R.real, ex.R.real.astype(np.float32).astype(np.float64))
    assert np.array_equal(b16.R.imag, ex.R.imag.astype(np.float32).astype(np.float64))


# --------------------------------------------------------------------------
# population: conservation, Boltzmann stationarity and convergence (Eq. 2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 1, 0)])
def test_conservation(periodic):
    inp = lpc_inputs.random_case((6, 5, 7), 21, periodic=periodic, alpha=0.8)
    pk = oracle.pack_input(inp)
    rng = np.random.default_rng(2)
    rho0 = rng.random(inp.F.shape) * (inp.solid == 0)
    r = oracle.run(pk, rho0, 300, msd_axes=0)
    assert np.max(np.abs(r.P / r.P[0] - 1.0)) <= 1e-12
    assert abs(r.rho.sum() / rho0.sum() - 1.0) <= 1e-12


@pytest.mark.parametrize("periodic", [(1, 1, 1), (1, 0, 1)])
def test_boltzmann_start_is_stationary(periodic):
    inp = lpc_inputs.random_case((6, 7, 5), 22, periodic=periodic, F_sd=1.5, alpha=1.0)
    pk = oracle.pack_input(inp)
    rho_eq = oracle.boltzmann(inp.F, inp.solid)
    r = oracle.run(pk, rho_eq, 1, msd_axes=0)
    assert np.max(np.abs(r.rho - rho_eq)) <= 1e-14 * rho_eq.max()
    # Eq. 2 normalisation: the mean over pore sites is <rho> = 1
    assert rho_eq[inp.solid == 0].mean() == pytest.approx(1.0, rel=1e-13)


@pytest.mark.parametrize("kT", [0.7, 2.5])
def test_boltzmann_stationary_at_temperature(kT):
    """Eq. 1-2 with kT != 1: rho ∝ exp(-F/kT) is stationary, exp(-F) is not."""
    inp = lpc_inputs.random_case((5, 6, 7), 25, periodic=(1, 1, 0), F_sd=1.0, alpha=0.9)
    inp.kT = kT
    pk = oracle.pack_input(inp)
    rho_eq = oracle.boltzmann(inp.F, inp.solid, kT=kT)
    r = oracle.run(pk, rho_eq, 1, msd_axes=0)
    assert np.max(np.abs(r.rho - rho_eq)) <= 1e-14 * rho_eq.max()
    wrong = oracle.boltzmann(inp.F, inp.solid, kT=1.0)
    r2 = oracle.run(pk, wrong, 1, msd_axes=0)
    assert np.max(np.abs(r2.rho - wrong)) > 1e-6 * wrong.max()


def test_boltzmann_eq2_against_direct_formula():
    inp = lpc_inputs.random_case((3, 4, 5), 23)
    rho = oracle.boltzmann(inp.F, inp.solid, kT=1.0, mean_rho=2.0)
    pore = inp.solid == 0
    e = np.exp(-inp.F[pore])
    assert np.allclose(rho[pore], 2.0 * pore.sum() * e / e.sum(), rtol=1e-14)
    assert np.all(rho[~pore] == 0.0)


def test_convergence_to_boltzmann_per_cluster():
    """8^3, 20 % solid, alpha = 0.5, 2e4 steps: rho / e^{-F} is constant on each
    connected pore cluster, and each cluster keeps its initial population."""
    inp = lpc_inputs.random_case((8, 8, 8), 24, solid_frac=0.2, F_sd=1.0, alpha=0.5)
    pk = oracle.pack_input(inp)
    rho0 = inp.uniform_rho0()
    r = oracle.run(pk, rho0, 20000, msd_axes=0)
    label, ncl = bf.pore_clusters(inp.solid, inp.periodic)
    ratio = r.rho / np.exp(-inp.F)
    assert ncl >= 1
    for c in range(ncl):
        sel = label == c
        v = ratio[sel]
        assert np.max(np.abs(v / v.mean() - 1.0)) <= 1e-10
        assert r.rho[sel].sum() == pytest.approx(rho0[sel].sum(), rel=1e-11)


# --------------------------------------------------------------------------
# uniform lattice: the lazy random walk in closed form, MSD and D (Eq. 6-7)
# --------------------------------------------------------------------------

def _uniform_case(shape, alpha, omega0=0.0):
    nz, ny, nx = shape
    F = np.zeros(shape)
    solid = np.zeros(shape, np.uint8)
    om = np.full(shape, omega0)
    return nx, ny, nz, F, om, solid


@pytest.mark.parametrize("alpha", [0.3, 1.0])
def test_uniform_closed_form(alpha):
    shape = (5, 6, 7)
    nx, ny, nz, F, om, solid = _uniform_case(shape, alpha, omega0=1234.5)
    dt = lpc_inputs.DT
    pk = oracle.pack(nx, ny, nz, (1, 1, 1), alpha, dt, 1.0, F, om, solid)
    rng = np.random.default_rng(3)
    rho0 = rng.random(shape)
    n = 37
    r = oracle.run(pk, rho0, n, msd_axes=7)
    q = np.meshgrid(*[2 * np.pi * np.fft.fftfreq(s) for s in shape], indexing="ij")
    lam = 1.0 - alpha + alpha / 3.0 * (np.cos(q[0]) + np.cos(q[1]) + np.cos(q[2]))
    expect = np.fft.ifftn(np.fft.fftn(rho0) * lam ** n).real
    assert np.max(np.abs(r.rho - expect)) <= 1e-12 * rho0.max()
    phase = np.exp(1j * 1234.5 * dt * n)
    assert np.max(np.abs(r.m - phase * expect)) <= 1e-12 * rho0.max()
    # MSD_a(n) = alpha n / 3 per axis for any start, D_a = alpha a^2 / (6 dt)
    for a in range(3):
        msd = r.msd(a)
        assert np.allclose(msd, alpha * np.arange(n + 1) / 3.0, rtol=1e-12, atol=1e-14)
        D = oracle.diffusion(msd, dt)
        assert np.allclose(D[1:], alpha / (6.0 * dt), rtol=1e-12)


# --------------------------------------------------------------------------
# magnetisation: omega = 0, uniform omega (single spectral line), |M| <= P
# --------------------------------------------------------------------------

def test_zero_omega_gives_m_equal_rho():
    inp = lpc_inputs.random_case((5, 4, 6), 31, periodic=(1, 0, 1))
    inp.omega[:] = 0.0
    pk = oracle.pack_input(inp)
    r = oracle.run(pk, _uniform_rho(inp), 60, msd_axes=0)
    assert np.array_equal(r.m.real, r.rho)
    assert np.all(r.m.imag == 0.0)


def test_uniform_omega_single_spectral_line():
    nfft = 256
    j = 7
    dt = lpc_inputs.DT
    inp = lpc_inputs.random_case((5, 6, 4), 32, periodic=(1, 1, 0))
    omega0 = 2 * np.pi * j / (nfft * dt)
    inp.omega[:] = omega0
    pk = oracle.pack_input(inp)
    r = oracle.run(pk, _uniform_rho(inp), nfft - 1, msd_axes=0)
    n = np.arange(nfft)
    assert np.allclose(r.M, np.exp(1j * omega0 * dt * n) * r.P[0], rtol=0, atol=1e-12 * r.P[0])
    f, S = oracle.spectrum(r.M, dt)
    peak = np.argmax(np.abs(S))
    assert f[peak] == pytest.approx(omega0 / (2 * np.pi))
    others = np.delete(np.abs(S), peak)
    assert others.max() <= 1e-12 * nfft * r.P[0]
    assert abs(S[peak]) == pytest.approx(nfft * r.P[0], rel=1e-12)


def test_fid_modulus_bounded_by_population():
    inp = lpc_inputs.random_case((6, 6, 6), 33, shift_sd=20.0)
    pk = oracle.pack_input(inp)
    r = oracle.run(pk, _uniform_rho(inp), 200, msd_axes=0)
    assert np.all(np.abs(r.M) <= r.P[0] * (1 + 1e-13))
    assert abs(r.M[0] - r.P[0]) == 0.0


# --------------------------------------------------------------------------
# whole operator: dense matrix powers on 4^3 lattices
# --------------------------------------------------------------------------

@pytest.mark.parametrize("periodic,seed", [((1, 1, 1), 41), ((0, 1, 1), 42), ((1, 1, 0), 43)])
def test_dense_matrix_power(periodic, seed):
    inp = lpc_inputs.random_case((4, 4, 4), seed, periodic=periodic, solid_frac=0.2,
                                 F_sd=1.2, shift_sd=30.0, alpha=0.7)
    pk = oracle.pack_input(inp)
    T = bf.transition_matrix(inp.F, inp.solid, periodic, inp.alpha)
    R = np.exp(1j * inp.omega.reshape(-1) * inp.dt)
    A = R[:, None] * T
    rng = np.random.default_rng(seed)
    rho0 = rng.random(64) * (inp.solid.reshape(-1) == 0)
    r = oracle.run(pk, rho0.reshape(4, 4, 4), 200, msd_axes=0)
    one = np.ones(64)
    for n in (1, 7, 50, 200):
        An = np.linalg.matrix_power(A, n)
        Mn = one @ (An @ rho0)
        assert abs(r.M[n] - Mn) <= 1e-12 * rho0.sum()
    Tn = np.linalg.matrix_power(T, 200)
    assert np.max(np.abs(r.rho.reshape(-1) - Tn @ rho0)) <= 1e-12 * rho0.max()
    assert np.max(np.abs(r.m.reshape(-1) - np.linalg.matrix_power(A, 200) @ rho0)) <= 1e-12


# --------------------------------------------------------------------------
# MSD: brute-force displacement distributions, one-step MSD (Eq. 5), Kohn (Eq. 4)
# --------------------------------------------------------------------------

def test_msd_chain_with_walls_bruteforce():
    """A 1D chain n x 1 x 1 with walls on every axis, up to 10 steps."""
    nx = 6
    shape = (1, 1, nx)
    rng = np.random.default_rng(5)
    F = rng.normal(0, 1, shape)
    solid = np.zeros(shape, np.uint8)
    om = np.zeros(shape)
    periodic = (0, 0, 0)
    pk = oracle.pack(nx, 1, 1, periodic, 0.9, lpc_inputs.DT, 1.0, F, om, solid)
    rho0 = rng.random(shape)
    steps = 10
    r = oracle.run(pk, rho0, steps, msd_axes=7)
    msd_bf, rhos = bf.distribution_msd(F, solid, periodic, 0.9, rho0, steps)
    assert np.allclose(r.msd(0), msd_bf[0], rtol=1e-12, atol=1e-15)
    assert np.allclose(r.msd(1), 0.0, atol=0) and np.allclose(r.msd(2), 0.0, atol=0)
    assert np.allclose(r.rho.reshape(-1), rhos[-1], rtol=1e-12)


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 1, 0)])
def test_msd_3d_bruteforce(periodic):
    """3 x 4 x 3 lattice with solids: unwrapped displacement distribution, 5 steps."""
    inp = lpc_inputs.random_case((3, 4, 3), 51, periodic=periodic, solid_frac=0.2, alpha=0.8)
    pk = oracle.pack_input(inp)
    rho0 = np.random.default_rng(6).random(inp.F.shape) * (inp.solid == 0)
    steps = 5
    r = oracle.run(pk, rho0, steps, msd_axes=7)
    msd_bf, _ = bf.distribution_msd(inp.F, inp.solid, periodic, inp.alpha, rho0, steps)
    for a in range(3):
        assert np.allclose(r.msd(a), msd_bf[a], rtol=1e-12, atol=1e-15)


def test_one_step_msd_eq5():
    """Eq. 5: the one-step MSD along x is sum_j p_acc(i->j) a_x(j)^2 / z averaged
    with weight rho, i.e. the accepted-move probability to the two x
    neighbours, summed over sites with weight rho / sum(rho)."""
    inp = lpc_inputs.random_case((5, 5, 5), 52, periodic=(0, 1, 1), alpha=1.0)
    pk = oracle.pack_input(inp)
    rho0 = np.random.default_rng(7).random(inp.F.shape) * (inp.solid == 0)
    r = oracle.run(pk, rho0, 1, msd_axes=1)
    acc = 0.0
    for i, j, p, off in bf.moves(inp.F, inp.solid, inp.periodic, inp.alpha):
        acc += rho0.reshape(-1)[i] * p * off[0] ** 2
    assert r.msd(0)[1] == pytest.approx(acc / rho0.sum(), rel=1e-13)


@pytest.mark.parametrize("axis", [0, 2])
def test_kohn_identity_eq4(axis):
    """Eq. 4 from an equilibrium start: MSD(n) = n c0 + 2 sum_{m=1}^{n-1} (n-m) c_m,
    with the displacement autocorrelations c_m from dense matrices."""
    inp = lpc_inputs.random_case((4, 5, 3), 53, periodic=(1, 0, 1), solid_frac=0.15,
                                 F_sd=1.0, alpha=0.6)
    pk = oracle.pack_input(inp)
    rho_eq = oracle.boltzmann(inp.F, inp.solid).reshape(-1)
    n = 25
    r = oracle.run(pk, rho_eq.reshape(inp.F.shape), n, msd_axes=1 << axis)
    T = bf.transition_matrix(inp.F, inp.solid, inp.periodic, inp.alpha)
    D = bf.displacement_operator(inp.F, inp.solid, inp.periodic, inp.alpha, axis)
    Dsq = np.abs(bf.displacement_operator(inp.F, inp.solid, inp.periodic, inp.alpha, axis))
    P0 = rho_eq.sum()
    c0 = Dsq.sum(axis=0) @ rho_eq / P0           # <dx^2>: |d| = d^2 for unit hops
    u = D.sum(axis=0)                            # expected displacement from each site
    g = D @ rho_eq
    c = [c0]
    h = g.copy()
    for m in range(1, n):
        c.append(u @ h / P0)
        h = T @ h
    msd_kohn = np.array([k * c0 + 2.0 * sum((k - m) * c[m] for m in range(1, k))
                         for k in range(n + 1)])
    assert np.allclose(r.msd(axis), msd_kohn, rtol=1e-11, atol=1e-14)


# --------------------------------------------------------------------------
# Position-dependent diffusivity: per-link alpha_ij = alpha_ji (Sec. 2.1, after Eq. 7)
# --------------------------------------------------------------------------

def _links_case(shape, seed, periodic):
    inp = lpc_inputs.random_case(shape, seed, periodic=periodic, solid_frac=0.2, F_sd=1.2,
                                 shift_sd=30.0, alpha=1.0)
    u, links = lpc_inputs.symmetric_links(shape, seed + 1000)
    uf = u.reshape(-1)

    def link_alpha(i, j):
        return 0.2 + 0.8 * 0.5 * (uf[i] + uf[j])
    return inp, links, link_alpha


def test_links_uniform_reduce_to_scalar_alpha():
    inp = lpc_inputs.random_case((4, 5, 6), 61, periodic=(1, 0, 1), alpha=0.37)
    a = oracle.pack_input(inp)
    b = oracle.pack(inp.nx, inp.ny, inp.nz, inp.periodic, inp.alpha, inp.dt, inp.kT, inp.F, inp.omega,
                    inp.solid, alpha_links=np.full((3,) + inp.F.shape, inp.alpha))
    assert np.array_equal(a.w, b.w) and np.array_equal(a.s, b.s)


@pytest.mark.parametrize("periodic", [(1, 1, 1), (0, 1, 1), (1, 0, 0)])
def test_links_detailed_balance_and_boltzmann(periodic):
    inp, links, link_alpha = _links_case((5, 6, 7), 62, periodic)
    pk = oracle.pack(inp.nx, inp.ny, inp.nz, periodic, inp.alpha, inp.dt, inp.kT, inp.F, inp.omega,
                     inp.solid, alpha_links=links)
    nz, ny, nx = inp.F.shape
    pi = np.exp(-inp.F.reshape(-1))
    solid = inp.solid.reshape(-1)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = (z * ny + y) * nx + x
                for k, off in enumerate(bf.OFFSETS):
                    j = bf._target(x, y, z, off, inp.F.shape, periodic)
                    if j is None or solid[i] or solid[j]:
                        assert pk.w[i, k] == 0.0
                        continue
                    assert pi[i] * pk.w[i, k] == pytest.approx(pi[j] * pk.w[j, k ^ 1], rel=1e-14)
                    assert 0.0 < pk.w[i, k] <= link_alpha(i, j) / 6.0 * (1 + 1e-15)
    rho_eq = oracle.boltzmann(inp.F, inp.solid)
    r = oracle.run(pk, rho_eq, 1, msd_axes=0)
    assert np.max(np.abs(r.rho - rho_eq)) <= 1e-14 * rho_eq.max()


@pytest.mark.parametrize("periodic", [(1, 1, 1), (1, 0, 1)])
def test_links_dense_matrix_power(periodic):
    """Brute force with alpha_ij evaluated from the two sites (no storage convention)."""
    inp, links, link_alpha = _links_case((4, 3, 5), 63, periodic)
    pk = oracle.pack(inp.nx, inp.ny, inp.nz, periodic, inp.alpha, inp.dt, inp.kT, inp.F, inp.omega,
                     inp.solid, alpha_links=links)
    T = bf.transition_matrix(inp.F, inp.solid, periodic, inp.alpha, link_alpha=link_alpha)
    N = inp.F.size
    R = np.exp(1j * inp.omega.reshape(-1) * inp.dt)
    A = R[:, None] * T
    rng = np.random.default_rng(64)
    rho0 = rng.random(N) * (inp.solid.reshape(-1) == 0)
    r = oracle.run(pk, rho0.reshape(inp.F.shape), 120, msd_axes=0)
    assert np.max(np.abs(r.rho.reshape(-1) - np.linalg.matrix_power(T, 120) @ rho0)) <= 1e-12 * rho0.max()
    for n in (1, 9, 120):
        assert abs(r.M[n] - np.ones(N) @ (np.linalg.matrix_power(A, n) @ rho0)) <= 1e-12 * rho0.sum()


# --------------------------------------------------------------------------
# Reservoir faces (Sec. 3.2 item 1: field values fixed in the ghost layer of
# a non-periodic face)
# --------------------------------------------------------------------------

def _with_reservoirs(inp, reservoirs):
    inp.reservoirs = tuple(reservoirs)
    return inp


@pytest.mark.parametrize("periodic,faces", [((0, 1, 1), (0, 1)), ((0, 0, 1), (0, 3)),
                                            ((0, 0, 0), (1, 2, 4))])
def test_reservoir_boltzmann_is_stationary(periodic, faces):
    """Every reservoir at the same (F_res, rho_res): the grand-canonical state
    rho = rho_res exp(-(F - F_res)/kT) on pore sites is a fixed point (detailed
    balance holds on the reservoir links too); with omega = 0 and
    m_res = rho_res the magnetisation stays equal to rho."""
    kT, F_res, rho_res = 0.8, -0.7, 1.3
    inp = lpc_inputs.random_case((5, 6, 7), 71, periodic=periodic, F_sd=1.2, alpha=0.9)
    inp.kT = kT
    inp.omega[:] = 0.0
    res = [None] * 6
    for f in faces:
        res[f] = (F_res, rho_res, rho_res)
    _with_reservoirs(inp, res)
    pk = oracle.pack_input(inp)
    rho_eq = rho_res * np.exp(-(inp.F - F_res) / kT) * (inp.solid == 0)
    r = oracle.run(pk, rho_eq, 3, msd_axes=0)
    assert np.max(np.abs(r.rho - rho_eq)) <= 1e-14 * rho_eq.max()
    assert np.max(np.abs(r.m - rho_eq)) <= 1e-14 * rho_eq.max()
    # the canonical Boltzmann state of Eq. 2 with another mean is not stationary
    other = oracle.boltzmann(inp.F, inp.solid, kT=kT, mean_rho=0.5)
    r2 = oracle.run(pk, other, 1, msd_axes=0)
    assert np.max(np.abs(r2.rho - other)) > 1e-6 * other.max()


@pytest.mark.parametrize("alpha", [1.0, 0.4])
def test_reservoir_chain_linear_profile(alpha):
    """A uniform chain between two reservoirs (F = F_res = 0): the stationary
    profile of the discrete diffusion equation is linear, with the reservoir
    values at the virtual sites x = -1 and x = n; from an empty chain the
    iteration converges to it."""
    nx, rho_lo, rho_hi = 9, 2.0, 0.5
    shape = (1, 1, nx)
    F = np.zeros(shape)
    om = np.zeros(shape)
    solid = np.zeros(shape, np.uint8)
    res = [(0.0, rho_lo, 0.0), (0.0, rho_hi, 0.0), None, None, None, None]
    pk = oracle.pack(nx, 1, 1, (0, 0, 0), alpha, lpc_inputs.DT, 1.0, F, om, solid, reservoirs=res)
    x = np.arange(nx)
    lin = (rho_lo + (rho_hi - rho_lo) * (x + 1) / (nx + 1)).reshape(shape)
    r = oracle.run(pk, lin, 1, msd_axes=0)
    assert np.max(np.abs(r.rho - lin)) <= 1e-15 * rho_lo
    # steady flux: alpha/6 (rho_lo - rho_hi)/(n + 1) per step through every link
    r = oracle.run(pk, np.zeros(shape), int(60 / alpha * (nx + 1) ** 2 / 10) * 10, msd_axes=0)
    assert np.max(np.abs(r.rho - lin)) <= 1e-12


@pytest.mark.parametrize("periodic,seed", [((0, 1, 1), 81), ((0, 0, 1), 82)])
def test_reservoir_dense_affine(periodic, seed):
    """Brute force: the augmented dense operator [[T, Win rho_res], [0, 1]]
    (and its complex and first-moment forms) raised to n, against the
    oracle's populations, FID and MSD increments."""
    inp = lpc_inputs.random_case((4, 3, 4), seed, periodic=periodic, solid_frac=0.2, F_sd=1.2,
                                 shift_sd=30.0, alpha=0.8)
    rng = np.random.default_rng(seed)
    res = [None] * 6
    for f in range(4):
        if periodic[f // 2] == 0:
            res[f] = (float(rng.normal(0, 1)), float(rng.uniform(0.3, 2.0)),
                      complex(rng.normal(0, 1), rng.normal(0, 1)))
    _with_reservoirs(inp, res)
    pk = oracle.pack_input(inp)
    op = bf.reservoir_operators(inp.F, inp.solid, periodic, inp.alpha, res)
    T, Win = op["T"], op["Win"]
    N = inp.F.size
    rho_res = np.array([0.0 if e is None else e[1] for e in res])
    m_res = np.array([0.0 if e is None else e[2] for e in res], dtype=np.complex128)
    R = np.exp(1j * inp.omega.reshape(-1) * inp.dt)
    rho0 = rng.random(N) * (inp.solid.reshape(-1) == 0)
    steps = 60
    r = oracle.run(pk, rho0.reshape(inp.F.shape), steps, msd_axes=7)
    # augmented matrices
    Aug = np.zeros((N + 1, N + 1))
    Aug[:N, :N] = T
    Aug[:N, N] = Win @ rho_res
    Aug[N, N] = 1.0
    Am = np.zeros((N + 1, N + 1), dtype=np.complex128)
    Am[:N, :N] = R[:, None] * T
    Am[:N, N] = R * (Win @ m_res)
    Am[N, N] = 1.0
    x0 = np.append(rho0, 1.0)
    for n in (1, 5, 60):
        xn = np.linalg.matrix_power(Aug, n) @ x0
        mn = np.linalg.matrix_power(Am, n) @ x0.astype(np.complex128)
        assert abs(r.P[n] - xn[:N].sum()) <= 1e-12 * max(1.0, xn[:N].sum())
        assert abs(r.M[n] - mn[:N].sum()) <= 1e-12 * max(1.0, np.abs(mn[:N]).sum())
    assert np.max(np.abs(r.rho.reshape(-1) - (np.linalg.matrix_power(Aug, steps) @ x0)[:N])) <= 1e-12
    # first moments: mu' = T mu + D rho + Win (d rho_res); dMSD = sum 2 u mu + q rho
    for a in range(3):
        rho = rho0.copy()
        mu = np.zeros(N)
        for n in range(steps):
            d = 2.0 * op["u"][a] @ mu + op["q"][a] @ rho
            assert d == pytest.approx(r.dmsd[a, n], rel=1e-11, abs=1e-13)
            mu, rho = T @ mu + op["Dax"][a] @ rho + Win @ (op["dface"][:, a] * rho_res), \
                T @ rho + Win @ rho_res
        assert np.max(np.abs(r.mu[a].reshape(-1) - mu)) <= 1e-11


# --------------------------------------------------------------------------
# Region-resolved sums (spectra and diffusion of separate parts, Sec. 4)
# --------------------------------------------------------------------------

def test_regions_partition_the_totals_and_match_bruteforce():
    inp = lpc_inputs.random_case((4, 4, 4), 91, periodic=(1, 0, 1), solid_frac=0.2, F_sd=1.0,
                                 shift_sd=30.0, alpha=0.7)
    pk = oracle.pack_input(inp)
    lab = lpc_inputs.random_regions(inp.F.shape, 92, 3)
    N = inp.F.size
    rho0 = np.random.default_rng(93).random(N) * (inp.solid.reshape(-1) == 0)
    steps = 40
    r = oracle.run(pk, rho0.reshape(inp.F.shape), steps, msd_axes=5, region=lab, n_regions=3)
    assert np.max(np.abs(r.Mr.sum(axis=0) - r.M)) <= 1e-13 * r.P[0]
    assert np.max(np.abs(r.Pr.sum(axis=0) - r.P)) <= 1e-13 * r.P[0]
    assert np.max(np.abs(r.Dr.sum(axis=0) - r.dmsd)) <= 1e-13
    T = bf.transition_matrix(inp.F, inp.solid, inp.periodic, inp.alpha)
    R = np.exp(1j * inp.omega.reshape(-1) * inp.dt)
    A = R[:, None] * T
    lf = lab.reshape(-1)
    for n in (0, 1, 13, 40):
        mn = np.linalg.matrix_power(A, n) @ rho0
        pn = np.linalg.matrix_power(T, n) @ rho0
        for g in range(3):
            assert abs(r.Mr[g, n] - mn[lf == g].sum()) <= 1e-12 * rho0.sum()
            assert abs(r.Pr[g, n] - pn[lf == g].sum()) <= 1e-12 * rho0.sum()
    # region MSD increments against dense first moments
    D = bf.displacement_operator(inp.F, inp.solid, inp.periodic, inp.alpha, 2)
    u = D.sum(axis=0)
    q = np.abs(D).sum(axis=0)
    rho, mu = rho0.copy(), np.zeros(N)
    for n in range(steps):
        for g in range(3):
            sel = lf == g
            assert r.Dr[g, 2, n] == pytest.approx(2 * u[sel] @ mu[sel] + q[sel] @ rho[sel],
                                                  rel=1e-11, abs=1e-13)
        mu, rho = T @ mu + D @ rho, T @ rho


def test_single_region_equals_the_totals_bitwise():
    inp = lpc_inputs.random_case((5, 4, 6), 94, periodic=(0, 1, 1), alpha=0.6)
    pk = oracle.pack_input(inp)
    lab = np.zeros(inp.F.shape, np.uint8)
    r = oracle.run(pk, inp.uniform_rho0(), 30, msd_axes=1, region=lab, n_regions=1)
    assert np.array_equal(r.Mr[0], r.M) and np.array_equal(r.Pr[0], r.P)
    assert np.array_equal(r.Dr[0, 0], r.dmsd[0])


# --------------------------------------------------------------------------
# Kohn / VACF diffusion estimator (Eq. 4) and the diffusion of a region
# --------------------------------------------------------------------------

@pytest.mark.parametrize("axis", [0, 1])
def test_vacf_against_dense_autocorrelations(axis):
    """c_m of the oracle's run equal the autocorrelations computed with dense
    matrices (c_0 from the squared displacements, c_m = u T^(m-1) D rho / P)."""
    inp = lpc_inputs.random_case((4, 5, 3), 101, periodic=(1, 0, 1), solid_frac=0.15, F_sd=1.0, alpha=0.6)
    pk = oracle.pack_input(inp)
    rho_eq = oracle.boltzmann(inp.F, inp.solid).reshape(-1)
    n = 30
    r = oracle.run(pk, rho_eq.reshape(inp.F.shape), n, msd_axes=1 << axis)
    T = bf.transition_matrix(inp.F, inp.solid, inp.periodic, inp.alpha)
    D = bf.displacement_operator(inp.F, inp.solid, inp.periodic, inp.alpha, axis)
    P0 = rho_eq.sum()
    c = [np.abs(D).sum(axis=0) @ rho_eq / P0]
    h = D @ rho_eq
    u = D.sum(axis=0)
    for m in range(1, n):
        c.append(u @ h / P0)
        h = T @ h
    got = oracle.vacf(r.dmsd[axis], r.P[0])
    assert np.allclose(got, c, rtol=1e-9, atol=1e-13 * c[0])
    # the truncated Kohn sum is the running sum of the autocorrelations
    Dk = oracle.kohn_diffusion(r.dmsd[axis], r.P[0], inp.dt)
    for k in (0, 1, 7, n - 1):
        assert Dk[k] == pytest.approx((c[0] / 2 + sum(c[1:k + 1])) / inp.dt, rel=1e-9)


def test_kohn_and_region_diffusion_on_a_uniform_lattice():
    """Uniform lattice in equilibrium: uncorrelated jumps, c_0 = alpha/3 and
    c_m = 0, so D = alpha a^2 / (2 d dt) with d = 3 (Eq. 7) at every n, and the
    same D for the particles of any region."""
    shape = (5, 6, 7)
    nz, ny, nx = shape
    alpha, dt = 0.45, lpc_inputs.DT
    pk = oracle.pack(nx, ny, nz, (1, 1, 1), alpha, dt, 1.0, np.zeros(shape), np.zeros(shape),
                     np.zeros(shape, np.uint8))
    lab = lpc_inputs.random_regions(shape, 102, 3)
    r = oracle.run(pk, np.full(shape, 2.0), 25, msd_axes=7, region=lab, n_regions=3)
    for a in range(3):
        assert np.allclose(oracle.kohn_diffusion(r.dmsd[a], r.P[0], dt), alpha / (6 * dt), rtol=1e-12)
        c = oracle.vacf(r.dmsd[a], r.P[0])
        assert c[0] == pytest.approx(alpha / 3, rel=1e-12) and np.max(np.abs(c[1:])) <= 1e-14
        for g in range(3):
            Dr = oracle.region_diffusion(r.Dr[g, a], r.Pr[g], dt)
            assert np.allclose(Dr, alpha / (6 * dt), rtol=1e-12)


def test_region_diffusion_against_dense_moments_off_equilibrium():
    """D of the particles in a region at step n (Table 1's D per region):
    dMSD_r(n) / (2 dt P_r(n)), both taken at step n.  A non-uniform lattice
    (solids, random F, three regions) started far from equilibrium, so that
    P_r(n) changes from step to step: the oracle's estimator must equal the
    one built from dense powers of the transition operator, T^n rho0 for the
    populations and the dense first moments for the MSD increments.  Reading
    P_r at step n + 1 or at step 0 instead fails here (on a uniform lattice
    started uniform both readings pass)."""
    inp = lpc_inputs.random_case((5, 4, 3), 95, periodic=(1, 1, 0), solid_frac=0.2, F_sd=1.2,
                                 alpha=0.8)
    pk = oracle.pack_input(inp)
    lab = lpc_inputs.random_regions(inp.F.shape, 96, 3)
    N = inp.F.size
    pore = inp.solid.reshape(-1) == 0
    lf = lab.reshape(-1)
    rho0 = np.zeros(N)
    for g in range(3):                              # all particles start in two sites per region
        rho0[np.flatnonzero(pore & (lf == g))[:2]] = 5.0 + g
    steps, dt = 30, inp.dt
    r = oracle.run(pk, rho0.reshape(inp.F.shape), steps, msd_axes=3, region=lab, n_regions=3)
    T = bf.transition_matrix(inp.F, inp.solid, inp.periodic, inp.alpha)
    for axis in (0, 1):
        Dop = bf.displacement_operator(inp.F, inp.solid, inp.periodic, inp.alpha, axis)
        u, q = Dop.sum(axis=0), np.abs(Dop).sum(axis=0)
        rho, mu = rho0.copy(), np.zeros(N)
        dense = np.zeros((3, steps))
        for n in range(steps):
            for g in range(3):
                sel = lf == g
                dense[g, n] = (2 * u[sel] @ mu[sel] + q[sel] @ rho[sel]) / (2.0 * dt * rho[sel].sum())
            mu, rho = T @ mu + Dop @ rho, T @ rho
        for g in range(3):
            got = oracle.region_diffusion(r.Dr[g, axis], r.Pr[g], dt)
            assert got.shape == (steps,) and np.all(np.isfinite(dense[g]))
            assert np.allclose(got, dense[g], rtol=1e-10, atol=1e-12 * np.max(np.abs(dense[g])))
    # the populations of the regions do change over the run, so the reading of n matters
    assert np.max(np.abs(np.diff(r.Pr, axis=1))) > 1e-3 * r.P[0]
