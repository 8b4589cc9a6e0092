"""GPU parity against the FP64 oracle (through the C ABI, same seeded inputs).

Tolerances: geometry (solid mask, zero pattern of the weights) bit-exact;
stored FP32 / BF16 weights and FP32 rotation factors within one unit in the
last place of the oracle's own rounding of its FP64 values; FID, densities,
magnetisation relative L2 <= 1e-4 and MSD max relative error <= 1e-4 (for
n >= 10), both against the matched-input oracle (the oracle run on its own
FP32 / BF16 roundings) and, for FP32 weights, against the exact oracle.
"""
import numpy as np
import pytest

import lpc_inputs
import oracle
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _ulp_diff(a, b, bits):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = np.where(b != 0, 2.0 ** (np.floor(np.log2(np.abs(np.where(b != 0, b, 1.0)))) - (bits - 1)), 1.0)
    return np.abs(a - b) / scale


@pytest.mark.parametrize("wdt", [0, 1])
@pytest.mark.parametrize("case", range(4))
def test_geometry_and_weights(case, wdt):
    inp = H.small_cases()[case]
    inp.weight_dtype = wdt
    g = H.gpu_run(inp, 0)
    lat = g["lattice"]
    assert np.array_equal(lat.solid_mask(), inp.solid)
    pk = oracle.pack_input(inp, H.MODE_OF_DTYPE[wdt])
    w_or = pk.w.T.reshape((6,) + inp.F.shape)
    w_gpu = lat.weights().astype(np.float64)
    assert np.array_equal(w_gpu == 0, w_or == 0), "link geometry differs"
    bits = 24 if wdt == 0 else 8
    d = _ulp_diff(w_gpu, w_or, bits)
    assert d.max() <= 1.0
    assert np.mean(d > 0) < 1e-3
    R = lat.rotation()
    assert _ulp_diff(R[..., 0], pk.R.real.reshape(inp.F.shape), 24).max() <= 1.0
    assert _ulp_diff(R[..., 1], pk.R.imag.reshape(inp.F.shape), 24).max() <= 1.0
    lat.close()


@pytest.mark.parametrize("shift_sd", [5.0, 150.0])
def test_rotation_factors_small_and_large_phases(shift_sd):
    """R = exp(i omega dt) (Eq. 7-8) as the pack stores it, for the method's
    small phases (shifts of a few ppm) and for phases of several radians: the
    FP32 value of the FP64 oracle's phase factor in all but a handful of
    sites, never more than one unit in the last place from it."""
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.random_case((24, 40, 70), 390, solid_frac=0.1, shift_sd=shift_sd, msd_axes=0)
    theta = np.abs(inp.omega * inp.dt)
    if shift_sd > 100:
        assert np.mean(theta > 0.25) > 0.5 and theta.max() > 3.0     # both paths, and the wrap of large phases
    else:
        assert theta.max() < 0.25
    lat = Lattice.from_input(inp)
    R = lat.rotation().astype(np.float64)
    lat.close()
    pk = oracle.pack_input(inp, oracle.MODE_F32)
    Ro = pk.R.reshape(inp.F.shape)
    for part, ref in ((R[..., 0], Ro.real), (R[..., 1], Ro.imag)):
        d = _ulp_diff(part, ref, 24)
        assert d.max() <= 1.0
        assert np.mean(part != ref) < 1e-4


@pytest.mark.parametrize("case", range(4))
def test_parity_small_fp32(case):
    inp = H.small_cases()[case]
    steps = 300
    g = H.gpu_run(inp, steps)
    o = H.oracle_run(inp, steps, oracle.MODE_F32)
    errs = H.compare(g, o, inp.msd_axes, tol=1e-5)
    oe = H.oracle_run(inp, steps, oracle.MODE_EXACT)
    H.compare(g, oe, inp.msd_axes, tol=1e-4)
    assert np.max(np.abs(g["P"] / g["P"][0] - 1)) < 1e-5
    for a in range(3):
        if inp.msd_axes >> a & 1:
            assert H.rel_l2(g["mu%d" % a], o.mu[a]) <= 1e-4
    g["lattice"].close()
    print(errs)


@pytest.mark.parametrize("case", [0, 1])
def test_parity_small_bf16(case):
    inp = H.small_cases()[case]
    inp.weight_dtype = 1
    steps = 300
    g = H.gpu_run(inp, steps)
    o = H.oracle_run(inp, steps, oracle.MODE_BF16)
    H.compare(g, o, inp.msd_axes, tol=1e-5)
    g["lattice"].close()


def test_particle_32_full_run():
    """The 32^3 particle workload, 2000 steps, FP32 weights, MSD on x, y, z."""
    inp = lpc_inputs.particle()
    g = H.gpu_run(inp, inp.steps)
    o = H.oracle_run(inp, inp.steps, oracle.MODE_EXACT)
    errs = H.compare(g, o, inp.msd_axes, tol=1e-4)
    om = H.oracle_run(inp, inp.steps, oracle.MODE_F32)
    H.compare(g, om, inp.msd_axes, tol=1e-4)
    assert np.max(np.abs(g["P"] / g["P"][0] - 1)) <= 1e-5
    assert np.all(np.abs(g["M"]) <= g["P"][0] * (1 + 1e-5))
    g["lattice"].close()
    print(errs)


def test_uniform_lattice_closed_form():
    shape = (12, 10, 40)
    alpha = 0.6
    inp = lpc_inputs.random_case(shape, 7, solid_frac=0.0, F_sd=0.0, shift_sd=0.0, alpha=alpha)
    inp.F[:] = 0.0
    omega0 = 2 * np.pi * 3 / (64 * inp.dt)
    inp.omega[:] = omega0
    rho0 = np.random.default_rng(9).random(shape)
    n = 63
    g = H.gpu_run(inp, n, rho0=rho0)
    q = np.meshgrid(*[2 * np.pi * np.fft.fftfreq(s) for s in shape], indexing="ij")
    lam = 1 - alpha + alpha / 3 * (np.cos(q[0]) + np.cos(q[1]) + np.cos(q[2]))
    expect = np.fft.ifftn(np.fft.fftn(rho0) * lam ** n).real
    assert H.rel_l2(g["rho"], expect) <= 1e-5
    # single spectral line of the 64-sample FID at bin 3
    S = np.fft.fft(g["M"])
    assert np.argmax(np.abs(S)) == 3
    assert np.max(np.abs(np.delete(S, 3))) <= 1e-4 * np.abs(S[3])
    for a in range(3):
        assert np.allclose(g["msd%d" % a], alpha * np.arange(n + 1) / 3, rtol=1e-5, atol=1e-6)
    g["lattice"].close()


def test_boltzmann_init_is_stationary():
    inp = lpc_inputs.random_case((16, 20, 36), 8, periodic=(1, 0, 1), alpha=1.0)
    from paper_2603_22553_b300.lattice import Lattice
    lat = Lattice.from_input(inp, init=1)
    rho_eq = oracle.boltzmann(inp.F, inp.solid)
    r0 = lat.density().astype(np.float64)
    assert H.rel_l2(r0, rho_eq) <= 1e-6
    lat.step(50)
    assert H.rel_l2(lat.density(), rho_eq) <= 1e-5
    lat.close()


def test_graph_replay_matches_single_launches():
    inp = H.small_cases()[0]
    a = H.gpu_run(inp, 70)                       # graphs of 32 steps + remainder
    b = H.gpu_run(inp, 70, chunks=[1] * 70)      # one launch per call
    assert np.array_equal(a["rho"], b["rho"])
    assert np.array_equal(a["M"], b["M"])
    assert np.array_equal(a["msd0"], b["msd0"])
    a["lattice"].close()
    b["lattice"].close()


def test_checkpoint_resume_bit_identical():
    inp = H.small_cases()[1]
    from paper_2603_22553_b300.lattice import Lattice
    ref = Lattice.from_input(inp)
    ref.step(90)
    a = Lattice.from_input(inp)
    a.step(40)
    blob = a.get_state()
    b = Lattice.from_input(inp)
    b.set_state(blob)
    assert b.steps_done == 40
    b.step(50)
    assert np.array_equal(b.density(), ref.density())
    assert np.array_equal(b.fid(), ref.fid())
    assert np.array_equal(b.msd(0), ref.msd(0))
    for l in (ref, a, b):
        l.close()


@pytest.mark.parametrize("shape,periodic", [((1, 1, 1), (1, 1, 1)), ((1, 1, 7), (0, 0, 0)),
                                            ((3, 1, 2), (1, 1, 1)), ((2, 9, 1), (1, 0, 1)),
                                            ((4, 4, 4), (0, 0, 0))])
def test_degenerate_shapes(shape, periodic):
    frac = 0.1 if np.prod(shape) >= 20 else 0.0
    inp = lpc_inputs.random_case(shape, 5, periodic=periodic, solid_frac=frac, alpha=0.8, msd_axes=7)
    g = H.gpu_run(inp, 25)
    o = H.oracle_run(inp, 25, oracle.MODE_F32)
    H.compare(g, o, 7, tol=1e-5)
    g["lattice"].close()


def test_all_solid_and_zero_steps():
    inp = lpc_inputs.random_case((4, 5, 6), 6, solid_frac=1.0)
    g = H.gpu_run(inp, 0)
    assert g["M"].shape == (1,) and g["M"][0] == 0 and g["P"][0] == 0
    g["lattice"].step(10)
    assert np.all(g["lattice"].population() == 0)
    g["lattice"].close()


def test_query_range_errors():
    from paper_2603_22553_b300 import binding as B
    from paper_2603_22553_b300.lattice import Lattice
    inp = H.small_cases()[3]
    lat = Lattice.from_input(inp)
    lat.step(5)
    with pytest.raises(B.LPCError):
        lat.fid(0, 7)
    with pytest.raises(B.LPCError):
        lat.msd(0)            # MSD not enabled for this case
    with pytest.raises(B.LPCError):
        lat.step(-1)
    lat.close()


def test_raw_cuda_allocator_path():
    inp = H.small_cases()[0]
    a = H.gpu_run(inp, 40, allocator=None)
    b = H.gpu_run(inp, 40)
    assert np.array_equal(a["M"], b["M"])
    a["lattice"].close()
    b["lattice"].close()


def test_equilibration_rho_only_tma_step_matches_full_step():
    """With the one-step TMA schedule the equilibration phase propagates rho
    alone; its populations are bit-identical to full steps of the
    register-pipelined kernel, and it stops after the same number of steps."""
    from paper_2603_22553_b300 import binding as B
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.random_case((40, 70, 130), 13, solid_frac=0.2, alpha=0.5, msd_axes=2)
    out = []
    for sched in ((B.LPC_KERNEL_TB, 1), (B.LPC_KERNEL_STEP1, 1)):
        lat = Lattice.from_input(inp)
        lat.set_schedule(*sched)
        it, diff = lat.equilibrate(1e-5, 3000, check_every=150)
        out.append((it, diff, lat.density(), lat.magnetization(), lat.fid(), lat.population()))
        lat.step(5)
        out[-1] += (lat.density(),)
        lat.close()
    a, b = out
    assert a[0] == b[0] and a[1] == b[1]
    for x, y in zip(a[2:], b[2:]):
        assert np.array_equal(x, y)


def test_equilibration_phase():
    inp = lpc_inputs.random_case((8, 12, 40), 12, solid_frac=0.2, alpha=0.5, msd_axes=1)
    from paper_2603_22553_b300.lattice import Lattice
    lat = Lattice.from_input(inp)
    iters, diff = lat.equilibrate(1e-6, 20000, check_every=200)
    assert diff < 1e-6 and iters < 20000 and iters % 200 == 0
    o = H.oracle_run(inp, iters, oracle.MODE_F32, msd_axes=0)
    assert H.rel_l2(lat.density(), o.rho) <= 1e-4
    # the propagation phase restarts from the equilibrated populations
    assert lat.steps_done == 0
    assert np.allclose(lat.fid(), lat.population(), rtol=1e-7)
    lat.step(10)
    assert lat.msd(0)[-1] > 0
    lat.close()


@pytest.mark.parametrize("sched", ["auto", "step1", "tb1", "batch"])
def test_per_link_alpha_parity(sched):
    """Position-dependent diffusivity (per-link alpha_ij = alpha_ji): GPU
    weights equal the oracle's rounded weights; every schedule matches the
    FP64 oracle and the Boltzmann state stays stationary."""
    from paper_2603_22553_b300 import binding as B
    from paper_2603_22553_b300.lattice import Lattice, step_many
    shape = (20, 36, 130)
    inp = lpc_inputs.random_case(shape, 71, periodic=(1, 0, 1), alpha=1.0, msd_axes=5)
    _, inp.alpha_links = lpc_inputs.symmetric_links(shape, 72, lo=0.05, hi=0.9)
    lat = Lattice.from_input(inp)
    if sched == "step1":
        lat.set_schedule(B.LPC_KERNEL_STEP1, 1)
    elif sched == "tb1":
        lat.set_schedule(B.LPC_KERNEL_TB, 1)
    steps = 60
    if sched == "batch":
        step_many([lat], [steps])
    else:
        lat.step(steps)
    pk = oracle.pack_input(inp, oracle.MODE_F32)
    w = lat.weights().reshape(6, -1).T.astype(np.float64)      # (N, 6) like the oracle
    assert np.array_equal(w, pk.w)
    g = dict(M=lat.fid(), P=lat.population(), rho=lat.density().astype(np.float64), m=lat.magnetization())
    for a in (0, 2):
        g["msd%d" % a] = lat.msd(a)
    o = oracle.run(pk, inp.uniform_rho0(), steps, msd_axes=5)
    H.compare(g, o, 5, tol=1e-5)
    lat.close()
