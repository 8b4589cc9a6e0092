"""One lattice decomposed along z into slabs, with halo exchange.

The paper runs large systems as several processes, each owning a part of
the lattice with ghost layers that neighbours refresh between steps (Sec.
3.2-3.3).  Here a lattice of nz planes is cut along z (the slowest axis)
into ``parts`` slabs of near-equal thickness.  Each slab is a library
handle (``lattice_create_slab``) holding its own planes plus one halo plane
on each side.  Every step is:

1. each slab advances its own planes one step (``lattice_step_n(h, 1)``);
2. the halo exchange: every slab's first own plane goes into the upper halo
   of the slab below it and its last own plane into the lower halo of the
   slab above it (``lattice_slab_planes`` gives the device addresses);
   with a periodic z the first and last slabs are neighbours, and a single
   slab is its own neighbour; at a z wall the halo is an all-solid plane
   that is never exchanged.

The per-step sums M, P and dMSD of the slabs add up to the whole lattice's:
each slab sums over its own planes.  ``reduce_histories`` adds them in slab
order in FP64, so the result does not depend on timing.

Two transports move the planes, behind one interface (``exchange(plan,
slabs)``):

* ``LocalTransport``: all slabs are handles in this process (on one device):
  device-to-device copies on the current stream.
* ``DistTransport``: one slab per rank of a ``torch.distributed`` process
  group (NCCL between GPUs, or gloo for host tensors): point-to-point sends
  and receives, matched by the plan's fixed order of exchanges.

The plan, the field slicing, the exchange order and the reduction order are
host logic; the stepping runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import binding as B

FIRST, LAST, HALO_BELOW, HALO_ABOVE = (B.LPC_PLANE_FIRST, B.LPC_PLANE_LAST, B.LPC_PLANE_HALO_BELOW,
                                       B.LPC_PLANE_HALO_ABOVE)


class SlabPlan:
    """Cut of ``nz`` planes into ``parts`` slabs along z.

    Slab r owns the planes [bounds[r][0], bounds[r][1]).  ``periodic_z``:
    the lattice wraps in z (the first and last slabs are neighbours)."""

    def __init__(self, nz, parts, periodic_z):
        if parts < 1 or parts > nz:
            raise ValueError("need 1 <= parts <= nz")
        self.nz = int(nz)
        self.parts = int(parts)
        self.periodic_z = bool(periodic_z)
        self.bounds = [(self.nz * r // self.parts, self.nz * (r + 1) // self.parts) for r in range(self.parts)]

    def below(self, r):
        """The slab whose last plane is the lower halo of slab r (None at a wall)."""
        if r > 0:
            return r - 1
        return self.parts - 1 if self.periodic_z else None

    def above(self, r):
        """The slab whose first plane is the upper halo of slab r (None at a wall)."""
        if r < self.parts - 1:
            return r + 1
        return 0 if self.periodic_z else None

    def halo_planes(self, r):
        """Global plane indices of slab r's lower and upper halos (None at a wall)."""
        z0, z1 = self.bounds[r]
        lo = (z0 - 1) % self.nz if self.below(r) is not None else None
        hi = z1 % self.nz if self.above(r) is not None else None
        return lo, hi

    def exchanges(self):
        """Every copy of one step's exchange as (src slab, src plane, dst slab,
        dst plane), in a fixed order that both ends of a transfer share."""
        out = []
        for r in range(self.parts):
            a = self.above(r)
            if a is not None:
                out.append((r, LAST, a, HALO_BELOW))
            b = self.below(r)
            if b is not None:
                out.append((r, FIRST, b, HALO_ABOVE))
        return out


def slab_field(field, plan, r, wall_value):
    """Planes of a [nz][ny][nx] global field for slab r: the lower halo, the
    own planes, the upper halo ([nz_r + 2][ny][nx]); a halo at a z wall is
    filled with ``wall_value``."""
    field = np.asarray(field)
    z0, z1 = plan.bounds[r]
    lo, hi = plan.halo_planes(r)
    wall = np.full((1,) + field.shape[1:], wall_value, dtype=field.dtype)
    parts = [field[lo:lo + 1] if lo is not None else wall, field[z0:z1],
             field[hi:hi + 1] if hi is not None else wall]
    return np.ascontiguousarray(np.concatenate(parts, axis=0))


def slab_fields(inp, plan, r, rho0=None):
    """Keyword arguments of slab r's fields from an ``lpc_inputs.LatticeInput``
    (F, omega, solid, rho0, alpha_links): halo planes at a z wall are solid."""
    kw = dict(F=slab_field(inp.F, plan, r, 0.0), omega=slab_field(inp.omega, plan, r, 0.0),
              solid=slab_field(inp.solid, plan, r, 1))
    r0 = rho0 if rho0 is not None else inp.rho0
    if r0 is not None:
        kw["rho0"] = slab_field(np.asarray(r0, dtype=np.float64).reshape(inp.F.shape), plan, r, 0.0)
    links = getattr(inp, "alpha_links", None)
    if links is not None:
        la = np.asarray(links, dtype=np.float64).reshape((3,) + inp.F.shape)
        kw["alpha_links"] = np.stack([slab_field(la[a], plan, r, 0.0) for a in range(3)])
    return kw


class _DeviceBytes:
    """A device buffer described by address and size (the CUDA array
    interface), so that torch can view it without copying."""

    def __init__(self, addr, nbytes):
        self.__cuda_array_interface__ = {"shape": (int(nbytes),), "typestr": "|u1", "data": (int(addr), False),
                                         "version": 3, "strides": None}


def device_view(addr, nbytes):
    """A uint8 torch CUDA tensor over ``nbytes`` bytes at device address ``addr``."""
    import torch
    return torch.as_tensor(_DeviceBytes(addr, nbytes), device="cuda")


class Slab:
    """One slab on the GPU: a ``Lattice`` created with ``slab=True``."""

    def __init__(self, inp, plan, r, rho0=None, **kw):
        from .lattice import Lattice
        z0, z1 = plan.bounds[r]
        self.rank = r
        f = slab_fields(inp, plan, r, rho0)
        args = dict(periodic=inp.periodic, alpha=inp.alpha, dt=inp.dt, kT=inp.kT, weight_dtype=inp.weight_dtype,
                    msd_axes=inp.msd_axes, reservoirs=getattr(inp, "reservoirs", None))
        args.update(kw)
        self.lattice = Lattice(inp.nx, inp.ny, z1 - z0, f["F"], f["omega"], f["solid"], rho0=f.get("rho0"),
                               alpha_links=f.get("alpha_links"), slab=True, **args)
        self._views = {}

    def step(self):
        self.lattice.step(1)

    def planes(self, which):
        """Byte views (torch CUDA tensors) of the state planes named by ``which``
        (the views of the two state buffers are made once and kept)."""
        out = []
        for a, n in self.lattice.slab_planes(which):
            t = self._views.get(a)
            if t is None:
                t = self._views[a] = device_view(a, n)
            out.append(t)
        return out

    def history(self):
        """(M complex, P, dMSD [3][steps]) of this slab's own planes."""
        lat = self.lattice
        M, P = lat.fid(), lat.population()
        steps = len(P) - 1
        d = np.zeros((3, steps))
        for a in range(3):
            if lat.msd_axes >> a & 1 and steps > 0:
                d[a] = lat.dmsd(a)
        return M, P, d

    def close(self):
        self._views = {}
        self.lattice.close()


class LocalTransport:
    """Halo exchange between slabs of this process: device-to-device copies
    on the current stream (ordered after the slabs' steps, which return on
    that stream, and before their next steps)."""

    def exchange(self, plan, slabs):
        for src, sp, dst, dp in plan.exchanges():
            for s, d in zip(slabs[src].planes(sp), slabs[dst].planes(dp)):
                d.copy_(s)


class DistTransport:
    """Halo exchange between ranks of a torch.distributed group, one slab per
    rank (``slabs`` maps the rank to its slab): every transfer of the plan's
    list is one send on its source rank and one receive on its destination
    rank, posted in the list's order with the transfer's index as tag."""

    def __init__(self, group=None):
        self.group = group

    def exchange(self, plan, slabs):
        import torch.distributed as dist
        me = dist.get_rank(self.group)
        ops = []
        for t, (src, sp, dst, dp) in enumerate(plan.exchanges()):
            if src == me and dst == me:
                for s, d in zip(slabs[me].planes(sp), slabs[me].planes(dp)):
                    d.copy_(s)
            elif src == me:
                for q, s in enumerate(slabs[me].planes(sp)):
                    ops.append(dist.P2POp(dist.isend, s.contiguous(), dst, self.group, tag=8 * t + q))
            elif dst == me:
                for q, d in enumerate(slabs[me].planes(dp)):
                    ops.append(dist.P2POp(dist.irecv, d, src, self.group, tag=8 * t + q))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()


def common_schedule(kernels):
    """One schedule for every slab of a lattice.  The one-step kernels give
    the same states, but they attribute a link's MSD increment to different
    ends (the TMA-fed kernel to the destination, the register-pipelined one to
    the source), so slabs of one lattice must use the same kernel for their
    increments to add up: the register-pipelined kernel if any slab's
    automatic choice is it, else the TMA-fed one."""
    if any(k == B.LPC_KERNEL_STEP1 for k in kernels):
        return (B.LPC_KERNEL_STEP1, 1)
    return (B.LPC_KERNEL_TB, 1)


def reduce_histories(histories):
    """Whole-lattice M, P and dMSD from per-slab histories, added in slab order
    (FP64).  ``histories``: a list of (M, P, dMSD) in slab order."""
    M = np.zeros_like(histories[0][0])
    P = np.zeros_like(histories[0][1])
    D = np.zeros_like(histories[0][2])
    for m, p, d in histories:
        M = M + m
        P = P + p
        D = D + d
    return M, P, D


def gather_histories(local, group=None):
    """Every rank's (M, P, dMSD) history, gathered to every rank and added in
    rank order (``reduce_histories``); the FP64 values travel as they are."""
    import torch
    import torch.distributed as dist
    M, P, D = local
    flat = np.concatenate([M.real, M.imag, P, D.reshape(-1)]).astype(np.float64)
    backend = dist.get_backend(group)
    dev = "cuda" if backend == "nccl" else "cpu"
    t = torch.from_numpy(flat).to(dev)
    ws = dist.get_world_size(group)
    outs = [torch.empty_like(t) for _ in range(ws)]
    dist.all_gather(outs, t, group=group)
    n = len(P)
    hist = []
    for o in outs:
        a = o.cpu().numpy()
        hist.append((a[:n] + 1j * a[n:2 * n], a[2 * n:3 * n], a[3 * n:].reshape(D.shape)))
    return reduce_histories(hist)


def msd_from(D, P0):
    """MSD(n) = sum_{j<n} dMSD(j) / P(0) along each axis, n = 0 .. steps."""
    out = np.zeros((D.shape[0], D.shape[1] + 1))
    np.cumsum(D, axis=1, out=out[:, 1:])
    return out / P0


class SlabLattice:
    """A lattice run as ``parts`` slabs in this process (one device), with the
    local transport: the single-GPU form of the decomposition, and the
    reference for the multi-rank one."""

    def __init__(self, inp, parts, rho0=None, transport=None, schedule=None, static_form=None, **kw):
        self.plan = SlabPlan(inp.nz, parts, inp.periodic[2])
        self.slabs = [Slab(inp, self.plan, r, rho0=rho0, **kw) for r in range(parts)]
        self.transport = transport or LocalTransport()
        self.shape = inp.F.shape
        if schedule is None:
            schedule = common_schedule([s.lattice.info()["kernel"] for s in self.slabs])
        for s in self.slabs:
            s.lattice.set_schedule(*schedule)
            if static_form is not None:
                s.lattice.set_static_form(static_form)

    def step(self, n):
        for _ in range(int(n)):
            for s in self.slabs:
                s.step()
            self.transport.exchange(self.plan, self.slabs)

    def histories(self):
        """Whole-lattice (M, P, dMSD) in slab order."""
        return reduce_histories([s.history() for s in self.slabs])

    def _gather(self, fn):
        return np.concatenate([fn(s.lattice) for s in self.slabs], axis=0)

    def density(self):
        return self._gather(lambda l: l.density())

    def magnetization(self):
        return self._gather(lambda l: l.magnetization())

    def moment(self, axis):
        return self._gather(lambda l: l.moment(axis))

    def close(self):
        for s in self.slabs:
            s.close()
