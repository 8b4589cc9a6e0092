"""Host logic of the slab decomposition (no GPU).

* The plan: slabs partition the planes, neighbours and halo planes follow
  the boundary along z, every halo that is not at a wall receives exactly
  one plane per step, from the right slab.
* The field slicing: a slab's fields are the global planes it owns plus the
  planes just outside it (an all-solid plane at a z wall).
* Two ranks over gloo (world_size 2): each rank advances its slab with a CPU
  stand-in for the library's step (the FP64 oracle on the slab's planes) and
  exchanges halos through ``DistTransport``, the transport the multi-GPU run
  uses; the histories are gathered and added in rank order.  The gathered
  state must equal the oracle's run of the whole lattice bit for bit (the
  per-site arithmetic of an own plane is the same as in the whole lattice),
  and the sums agree to FP64 rounding.
"""
import os
import socket

import numpy as np
import pytest

import lpc_inputs
import oracle
from paper_2603_22553_b300 import slabs as S


@pytest.mark.parametrize("nz,parts,periodic", [(10, 1, True), (10, 1, False), (10, 3, True), (11, 4, False),
                                               (7, 7, True), (2, 2, False)])
def test_plan_partitions_and_pairs_every_halo(nz, parts, periodic):
    plan = S.SlabPlan(nz, parts, periodic)
    owned = [z for z0, z1 in plan.bounds for z in range(z0, z1)]
    assert owned == list(range(nz))
    assert all(z1 - z0 >= 1 for z0, z1 in plan.bounds)
    received = {}
    for src, sp, dst, dp in plan.exchanges():
        assert (dst, dp) not in received
        received[(dst, dp)] = (src, sp)
    for r in range(parts):
        z0, z1 = plan.bounds[r]
        lo, hi = plan.halo_planes(r)
        if periodic or r > 0:
            assert lo == (z0 - 1) % nz
            src, sp = received[(r, S.HALO_BELOW)]
            assert sp == S.LAST and plan.bounds[src][1] - 1 == lo
        else:
            assert lo is None and (r, S.HALO_BELOW) not in received
        if periodic or r < parts - 1:
            assert hi == z1 % nz
            src, sp = received[(r, S.HALO_ABOVE)]
            assert sp == S.FIRST and plan.bounds[src][0] == hi
        else:
            assert hi is None and (r, S.HALO_ABOVE) not in received


def test_plan_rejects_more_slabs_than_planes():
    with pytest.raises(ValueError):
        S.SlabPlan(3, 4, True)


def test_slab_fields_take_the_neighbouring_planes_and_solid_walls():
    inp = lpc_inputs.random_case((9, 4, 5), 11, periodic=(1, 1, 0))
    plan = S.SlabPlan(9, 3, False)
    for r in range(3):
        f = S.slab_fields(inp, plan, r)
        z0, z1 = plan.bounds[r]
        assert f["F"].shape == (z1 - z0 + 2, 4, 5)
        assert np.array_equal(f["F"][1:-1], inp.F[z0:z1])
        assert np.array_equal(f["solid"][1:-1], inp.solid[z0:z1])
        if r == 0:
            assert np.all(f["solid"][0] == 1)
        else:
            assert np.array_equal(f["omega"][0], inp.omega[z0 - 1])
        if r == 2:
            assert np.all(f["solid"][-1] == 1)
        else:
            assert np.array_equal(f["F"][-1], inp.F[z1])


def test_reduce_histories_adds_in_slab_order():
    rng = np.random.default_rng(3)
    hs = [(rng.normal(size=5) + 1j * rng.normal(size=5), rng.random(5), rng.normal(size=(3, 4))) for _ in range(3)]
    M, P, D = S.reduce_histories(hs)
    assert np.array_equal(M, (hs[0][0] + hs[1][0]) + hs[2][0])
    assert np.array_equal(P, (hs[0][1] + hs[1][1]) + hs[2][1])
    assert np.array_equal(D, (hs[0][2] + hs[1][2]) + hs[2][2])


class OracleSlab:
    """CPU stand-in for a slab handle: the FP64 oracle steps the slab's nz + 2
    planes (walls in z: the halos bound it) one step at a time; the own planes
    carry region label 1, so the oracle's region sums are the own planes'
    sums.  ``planes`` returns tensors sharing the state's memory."""

    def __init__(self, inp, plan, r):
        import torch
        self.torch = torch
        f = S.slab_fields(inp, plan, r)
        z0, z1 = plan.bounds[r]
        self.nzl = z1 - z0
        shape = (self.nzl + 2, inp.ny, inp.nx)
        self.pk = oracle.pack(inp.nx, inp.ny, self.nzl + 2, (inp.periodic[0], inp.periodic[1], 0), inp.alpha,
                              inp.dt, inp.kT, f["F"], f["omega"], f["solid"])
        self.lab = np.zeros(shape, np.uint8)
        self.lab[1:-1] = 1
        self.msd_axes = inp.msd_axes
        self.rho = (f["solid"] == 0).astype(np.float64)
        self.m = np.zeros(shape + (2,))
        self.m[..., 0] = self.rho
        self.mu = np.zeros((3,) + shape)
        self.M, self.P, self.D = [self._sum_m()], [self.rho[1:-1].sum()], []

    def _sum_m(self):
        return self.m[1:-1, :, :, 0].sum() + 1j * self.m[1:-1, :, :, 1].sum()

    def step(self):
        res = oracle.run(self.pk, self.rho, 1, m0=self.m[..., 0] + 1j * self.m[..., 1], mu0=self.mu,
                         msd_axes=self.msd_axes, region=self.lab, n_regions=2, nthreads=1)
        self.rho[...] = res.rho
        self.m[..., 0] = res.m.real
        self.m[..., 1] = res.m.imag
        self.mu[...] = res.mu
        self.M.append(res.Mr[1, 1])
        self.P.append(res.Pr[1, 1])
        self.D.append(res.Dr[1, :, 0])

    def planes(self, which):
        z = {S.FIRST: 1, S.LAST: self.nzl, S.HALO_BELOW: 0, S.HALO_ABOVE: self.nzl + 1}[which]
        out = [self.torch.from_numpy(self.rho[z]), self.torch.from_numpy(self.m[z])]
        for a in range(3):
            if self.msd_axes >> a & 1:
                out.append(self.torch.from_numpy(self.mu[a, z]))
        return out

    def history(self):
        return np.array(self.M), np.array(self.P), np.array(self.D).T.reshape(3, -1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, case, steps, outdir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        shape, periodic, msd = case
        inp = lpc_inputs.random_case(shape, 41, periodic=periodic, solid_frac=0.2, alpha=0.7, msd_axes=msd)
        plan = S.SlabPlan(inp.nz, ws, periodic[2])
        slab = OracleSlab(inp, plan, rank)
        tr = S.DistTransport()
        mine = {rank: slab}
        for _ in range(steps):
            slab.step()
            tr.exchange(plan, mine)
        M, P, D = S.gather_histories(slab.history())
        np.savez(os.path.join(outdir, "rank%d.npz" % rank), rho=slab.rho[1:-1], m=slab.m[1:-1],
                 mu=slab.mu[:, 1:-1], M=M, P=P, D=D)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", [((6, 5, 7), (1, 0, 1), 7), ((7, 6, 5), (0, 1, 0), 5)])
def test_two_ranks_over_gloo_equal_the_whole_lattice(case, tmp_path):
    import torch.multiprocessing as mp
    steps = 9
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), case, steps, str(tmp_path)), nprocs=ws,
                       start_method="spawn")
    shape, periodic, msd = case
    inp = lpc_inputs.random_case(shape, 41, periodic=periodic, solid_frac=0.2, alpha=0.7, msd_axes=msd)
    ref = oracle.run(oracle.pack_input(inp), inp.uniform_rho0(), steps, msd_axes=msd)
    parts = [np.load(os.path.join(tmp_path, "rank%d.npz" % r)) for r in range(ws)]
    rho = np.concatenate([p["rho"] for p in parts])
    m = np.concatenate([p["m"] for p in parts])
    mu = np.concatenate([p["mu"] for p in parts], axis=1)
    assert np.array_equal(rho, ref.rho)
    assert np.array_equal(m[..., 0] + 1j * m[..., 1], ref.m)
    for a in range(3):
        if msd >> a & 1:
            assert np.array_equal(mu[a], ref.mu[a])
    for p in parts:           # every rank holds the same reduced histories
        assert np.array_equal(p["M"], parts[0]["M"]) and np.array_equal(p["P"], parts[0]["P"])
    M, P, D = parts[0]["M"], parts[0]["P"], parts[0]["D"]
    assert np.allclose(M, ref.M, rtol=0, atol=1e-12 * ref.P[0])
    assert np.allclose(P, ref.P, rtol=1e-13)
    for a in range(3):
        if msd >> a & 1:
            assert np.allclose(D[a], ref.dmsd[a], rtol=1e-12, atol=1e-13)
            assert np.allclose(S.msd_from(D, P[0])[a], ref.msd(a), rtol=1e-12, atol=1e-13)
