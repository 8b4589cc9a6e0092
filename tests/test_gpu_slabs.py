"""Slab decomposition along z on one GPU: several slab handles of one lattice,
with device-to-device copies standing in for the transfers between GPUs
(``LocalTransport``, the same exchange interface as the multi-rank
``DistTransport``).

After n steps the slabs' own planes, put together, must equal the whole
lattice stepped by ``lattice_step_n`` bit for bit (the per-site arithmetic
is the same; a slab's halos hold exactly the neighbours' planes), in every
one-step kernel and static-data form; the FID, population and MSD
histories added over the slabs agree with the whole lattice's to FP32
summation order, and with the FP64 oracle.
"""
import numpy as np
import pytest

import lpc_inputs
import oracle
from paper_2603_22553_b300 import binding as B
from paper_2603_22553_b300 import slabs as S
from tests import helpers as H

pytestmark = pytest.mark.gpu

STEP1 = (B.LPC_KERNEL_STEP1, 1)
TMA1 = (B.LPC_KERNEL_TB, 1)

# (nz, ny, nx), periodic (x, y, z), MSD axes, weight type, parts, schedule, static form, seed
CASES = [
    ((24, 20, 33), (1, 1, 1), 7, 0, 2, STEP1, None, 501),
    ((25, 17, 40), (1, 0, 0), 5, 0, 3, STEP1, None, 502),        # z walls: all-solid outer halos
    ((12, 20, 70), (1, 1, 1), 1, 0, 1, STEP1, None, 503),        # one slab, its own neighbour
    ((36, 40, 130), (0, 1, 1), 1, 0, 2, TMA1, B.LPC_STATIC_GATHER, 504),
    ((36, 40, 130), (1, 1, 1), 6, 0, 3, TMA1, B.LPC_STATIC_LINK, 505),
    ((31, 33, 96), (1, 0, 0), 3, 1, 2, TMA1, B.LPC_STATIC_LINK, 506),   # BF16, walls in y and z
    ((40, 64, 200), (1, 1, 1), 0, 0, 4, None, None, 507),        # the automatic schedule of each slab
]


def _whole(inp, steps, schedule, form):
    from paper_2603_22553_b300.lattice import Lattice
    lat = Lattice.from_input(inp)
    lat.set_schedule(*schedule)
    if form is not None and schedule == TMA1:
        lat.set_static_form(form)
    lat.step(steps)
    out = dict(rho=lat.density(), m=lat.magnetization(), M=lat.fid(), P=lat.population())
    for a in range(3):
        if inp.msd_axes >> a & 1:
            out["mu%d" % a] = lat.moment(a)
            out["msd%d" % a] = lat.msd(a)
    lat.close()
    return out


@pytest.mark.parametrize("shape,periodic,msd,wdt,parts,schedule,form,seed", CASES)
def test_slabs_equal_the_whole_lattice(shape, periodic, msd, wdt, parts, schedule, form, seed):
    inp = lpc_inputs.random_case(shape, seed, periodic=periodic, solid_frac=0.2, alpha=0.7, msd_axes=msd,
                                 weight_dtype=wdt)
    steps = 41
    sl = S.SlabLattice(inp, parts, schedule=schedule, static_form=form)
    used = sl.slabs[0].lattice.info()
    assert all(s.lattice.info()["kernel"] == used["kernel"] for s in sl.slabs)
    sl.step(steps)
    if form is not None:
        assert all(s.lattice.info()["static_form"] == {B.LPC_STATIC_GATHER: 1, B.LPC_STATIC_LINK: 2}[form]
                   for s in sl.slabs)
    M, P, D = sl.histories()
    rho, m = sl.density(), sl.magnetization()
    mus = {a: sl.moment(a) for a in range(3) if msd >> a & 1}
    sl.close()
    ref = _whole(inp, steps, (used["kernel"], 1), form)
    assert np.array_equal(rho, ref["rho"])
    assert np.array_equal(m, ref["m"])
    for a, mu in mus.items():
        assert np.array_equal(mu, ref["mu%d" % a])
    assert np.allclose(M, ref["M"], rtol=1e-6, atol=1e-6 * ref["P"][0])
    assert np.allclose(P, ref["P"], rtol=1e-6)
    msd_s = S.msd_from(D, P[0])
    for a in mus:
        assert np.allclose(msd_s[a][1:], ref["msd%d" % a][1:], rtol=1e-5, atol=1e-9)


def test_slabs_against_the_oracle_300_steps():
    """Three slabs of a lattice large enough for the TMA-fed kernel, 300 steps,
    against the FP64 oracle on the matched FP32 weights."""
    inp = lpc_inputs.random_case((48, 64, 128), 508, periodic=(1, 1, 1), solid_frac=0.25, alpha=0.5, msd_axes=4)
    steps = 300
    sl = S.SlabLattice(inp, 3, schedule=TMA1)
    sl.step(steps)
    M, P, D = sl.histories()
    g = dict(M=M, P=P, rho=sl.density().astype(np.float64), m=sl.magnetization(),
             msd2=S.msd_from(D, P[0])[2])
    sl.close()
    o = H.oracle_run(inp, steps, oracle.MODE_F32)
    errs = H.compare(g, o, 4, tol=1e-5)
    print("3 slabs, 300 steps:", errs)


def test_slab_queries_and_rejections():
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.random_case((10, 12, 70), 509, periodic=(1, 1, 1), alpha=0.6, msd_axes=1)
    plan = S.SlabPlan(10, 2, True)
    s = S.Slab(inp, plan, 1)
    lat = s.lattice
    info = lat.info()
    z0, z1 = plan.bounds[1]
    assert info["n_sites"] == 70 * 12 * (z1 - z0)
    assert lat.density().shape == (z1 - z0, 12, 70)
    assert np.array_equal(lat.solid_mask(), inp.solid[z0:z1])
    w = lat.weights()
    assert w.shape == (6, z1 - z0, 12, 70)
    planes = lat.slab_planes(S.FIRST)
    assert len(planes) == 3 and planes[0][1] == info["pitch_x"] * info["pitch_y"] * 4
    with pytest.raises(B.LPCError):
        lat.set_schedule(B.LPC_KERNEL_TB, 2)         # a slab steps once between exchanges
    with pytest.raises(B.LPCError) as ei:
        lat.equilibrate(1e-6, 10)
    assert ei.value.status == B.LPC_ERR_STATE
    s.close()
    whole = Lattice.from_input(inp)
    with pytest.raises(B.LPCError):
        whole.slab_planes(S.FIRST)                   # not a slab
    whole.close()
