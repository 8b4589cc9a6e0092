"""GPU tests of the temporally blocked (TMA) schedule.

The TB kernel computes K steps per launch with the same per-site arithmetic
as the one-step kernel, so its states must be bit-identical to K one-step
launches for every block depth, ghost width, weight type and MSD mask; its
sums (FP32 row partials over a different tiling) agree to FP32 rounding.
Parity with the FP64 oracle is checked as for the one-step kernel.
"""
import numpy as np
import pytest

import lpc_inputs
import oracle
from paper_2603_22553_b300 import binding as B
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _run(inp, steps, schedule, ghost, **kw):
    return H.gpu_run(inp, steps, schedule=schedule, ghost=ghost, **kw)


CASES = [
    # shape (nz, ny, nx), periodic, msd mask, weight dtype, K, ghost
    ((12, 30, 61), (1, 1, 1), 0, 0, 2, 2),
    ((9, 41, 50), (0, 1, 1), 1, 0, 2, 2),
    ((10, 26, 33), (1, 0, 1), 7, 0, 3, 4),
    ((7, 35, 70), (1, 1, 0), 2, 1, 4, 4),
    ((16, 20, 24), (1, 1, 1), 5, 1, 2, 4),
    ((5, 9, 13), (1, 1, 1), 0, 0, 1, 2),
    ((3, 50, 100), (0, 0, 1), 6, 1, 3, 4),
    ((6, 7, 45), (1, 1, 1), 1, 0, 1, 2),          # depth 1, small tile shape
    ((9, 70, 40), (1, 0, 1), 7, 1, 1, 4),         # depth 1, big tile, all moments
    ((20, 37, 130), (1, 1, 1), 3, 0, 1, 2),       # depth 1, three x tiles, ragged x and y
    ((33, 19, 200), (0, 1, 0), 4, 1, 1, 6),       # depth 1, x and z walls, BF16, wide ghost
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_tb_bit_identical_to_one_step(case):
    shape, per, msd, wdt, K, G = CASES[case]
    inp = lpc_inputs.random_case(shape, 300 + case, periodic=per, alpha=0.7, msd_axes=msd,
                                 weight_dtype=wdt)
    steps = 11 * K + (1 if K > 1 else 0)          # TB launches plus a one-step remainder
    a = _run(inp, steps, (B.LPC_KERNEL_TB, K), G)
    b = _run(inp, steps, (B.LPC_KERNEL_STEP1, 1), G)
    assert np.array_equal(a["rho"], b["rho"])
    assert np.array_equal(a["m"], b["m"])
    for ax in range(3):
        if msd >> ax & 1:
            assert np.array_equal(a["mu%d" % ax], b["mu%d" % ax])
            assert np.allclose(a["msd%d" % ax][1:], b["msd%d" % ax][1:], rtol=1e-5)
    assert np.allclose(a["M"], b["M"], rtol=1e-6, atol=1e-6 * abs(b["M"][0]))
    assert np.allclose(a["P"], b["P"], rtol=1e-6)
    o = H.oracle_run(inp, steps, H.MODE_OF_DTYPE[wdt])
    H.compare(a, o, msd, tol=1e-5)
    a["lattice"].close()
    b["lattice"].close()


@pytest.mark.parametrize("K", [1, 2, 4])
def test_tb_graph_replay_long_run(K):
    """More than 32 launches: the captured graph of TB launches is replayed."""
    inp = lpc_inputs.random_case((20, 40, 57), 310 + K, periodic=(1, 0, 1), alpha=0.5, msd_axes=1)
    steps = 70 * K + 1
    G = max(2, K)
    a = _run(inp, steps, (B.LPC_KERNEL_TB, K), G)
    b = _run(inp, steps, (B.LPC_KERNEL_STEP1, 1), G)
    assert np.array_equal(a["rho"], b["rho"])
    assert np.array_equal(a["m"], b["m"])
    o = H.oracle_run(inp, steps, oracle.MODE_F32)
    H.compare(a, o, 1, tol=1e-5)
    a["lattice"].close()
    b["lattice"].close()


def test_tb_particle_32_full_run():
    inp = lpc_inputs.particle()
    g = _run(inp, inp.steps, (B.LPC_KERNEL_TB, 2), 2)
    o = H.oracle_run(inp, inp.steps, oracle.MODE_EXACT)
    H.compare(g, o, inp.msd_axes, tol=1e-4)
    g["lattice"].close()


def test_tb_rejects_impossible_depth():
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.random_case((4, 8, 8), 1)
    lat = Lattice.from_input(inp, ghost=2)
    with pytest.raises(B.LPCError):
        lat.set_schedule(B.LPC_KERNEL_TB, 3)     # deeper than the ghost layer
    with pytest.raises(B.LPCError):
        lat.set_schedule(B.LPC_KERNEL_TB, 0)
    lat.close()


def test_stale_allocator_memory_with_walls():
    """Lattices with walls must not read uninitialised ghost memory: fill the
    caching allocator's pool with NaN first, then create and step."""
    import torch
    junk = torch.full((64 << 20,), float("nan"), device="cuda")
    del junk
    inp = lpc_inputs.random_case((9, 40, 70), 102, periodic=(0, 1, 0), alpha=0.5, msd_axes=1)
    for sched, G in (((B.LPC_KERNEL_STEP1, 1), 2), ((B.LPC_KERNEL_TB, 1), 2), ((B.LPC_KERNEL_TB, 2), 2)):
        junk = torch.full((64 << 20,), float("nan"), device="cuda")
        del junk
        g = _run(inp, 40, sched, G)
        assert np.all(np.isfinite(g["M"])) and np.all(np.isfinite(g["m"]))
        o = H.oracle_run(inp, 40, oracle.MODE_F32)
        H.compare(g, o, 1, tol=1e-5)
        g["lattice"].close()


def test_autotune_restores_state_and_caches(tmp_path):
    """Autotuning mid-run leaves the results as if no trial had run, and the
    JSON cache replays the same choice."""
    from paper_2603_22553_b300 import autotune
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.random_case((24, 40, 70), 321, periodic=(1, 0, 1), alpha=0.6, msd_axes=1)
    ref = Lattice.from_input(inp, ghost=4)
    ref.step(30)
    lat = Lattice.from_input(inp, ghost=4)
    lat.step(10)
    path = str(tmp_path / "tune.json")
    c1 = autotune.choose(lat, trial_launches=3, path=path)
    assert not c1["cached"] and c1["kernel"] in (B.LPC_KERNEL_STEP1, B.LPC_KERNEL_TB)
    assert lat.steps_done == 10
    lat.step(20)
    assert np.array_equal(lat.density(), ref.density())
    assert np.allclose(lat.fid(), ref.fid(), rtol=1e-6, atol=1e-6 * abs(ref.fid()[0]))
    assert np.allclose(lat.msd(0)[1:], ref.msd(0)[1:], rtol=1e-5)
    other = Lattice.from_input(inp, ghost=4)
    c2 = autotune.choose(other, path=path)
    assert c2["cached"] and c2["kernel"] == c1["kernel"] and c2["block_steps"] == c1["block_steps"]
    assert c2["tile_rows"] == c1["tile_rows"] and c2["items_per_cta"] == c1["items_per_cta"]
    info = other.info()
    if c1["kernel"] == B.LPC_KERNEL_TB and c1["block_steps"] == 1:
        assert (info["tile_rows"], info["items_per_cta"]) == (c1["tile_rows"], c1["items_per_cta"])
    for l in (ref, lat, other):
        l.close()


@pytest.mark.parametrize("tiling", [(16, 0), (12, 5), (8, 200), (16, 1024)])
def test_tma_tiling_keeps_states_bit_identical(tiling):
    """Tile rows and work items per CTA of the TMA-fed one-step kernel (the
    autotuner's knobs) change the work split, not the states; sums agree to
    FP32 summation order."""
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.random_case((48, 70, 150), 331, periodic=(1, 0, 1), alpha=0.6, msd_axes=3)
    out = []
    for t in ((0, 0), tiling):
        lat = Lattice.from_input(inp)
        lat.set_schedule(B.LPC_KERNEL_TB, 1)
        lat.set_tiling(*t)
        lat.step(25)
        info = lat.info()
        if t[0]:
            assert info["tile_rows"] == t[0]
        if t[1]:
            assert info["items_per_cta"] == t[1]
        out.append((lat.density(), lat.magnetization(), lat.moment(0), lat.fid(), lat.msd(1)))
        lat.close()
    a, b = out
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    assert np.allclose(a[3], b[3], rtol=1e-6, atol=1e-6 * abs(a[3][0]))
    assert np.allclose(a[4][1:], b[4][1:], rtol=1e-5)


def test_one_step_tma_sums_bit_reproducible():
    """The work-queue kernel hands items to whichever CTA is free, but its
    sums are per item and added in item order: FID, P and MSD histories are
    identical from run to run."""
    inp = lpc_inputs.random_case((40, 70, 192), 7, periodic=(1, 1, 1), alpha=0.6, msd_axes=7)
    runs = []
    for _ in range(3):
        g = _run(inp, 30, (B.LPC_KERNEL_TB, 1), 2)
        runs.append([g["M"], g["P"], g["msd0"], g["msd1"], g["msd2"], g["rho"]])
        g["lattice"].close()
    for r in runs[1:]:
        for a, b in zip(runs[0], r):
            assert np.array_equal(a, b)
