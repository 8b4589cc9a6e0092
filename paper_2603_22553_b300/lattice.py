"""Python handle around one device-resident lattice (C ABI ``lattice_*``).

PyTorch supplies device memory (its caching allocator, through the
``lpc_allocator`` hooks) and the CUDA stream; all lattice arithmetic runs in
the CUDA library.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding as B


class TorchAllocator:
    """``lpc_allocator`` backed by PyTorch's CUDA caching allocator."""

    def __init__(self, device=None):
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device() if device is None else device

        def _alloc(nbytes, stream, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                              int(stream or 0)))
            except Exception:
                return None

        def _free(ptr, stream, ctx):
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))

        self._alloc_cb = B.ALLOC_FN(_alloc)
        self._free_cb = B.FREE_FN(_free)
        self.struct = B.lpc_allocator(self._alloc_cb, self._free_cb, None)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def step_many(lattices, steps):
    """Advance lattice i by steps[i] in batched launches (``lattice_step_many``)."""
    lats = list(lattices)
    if not lats:
        return
    lib = lats[0].lib
    hs = (ctypes.c_void_p * len(lats))(*[l.h.value for l in lats])
    ns = (ctypes.c_int64 * len(lats))(*[int(s) for s in steps])
    B.check(lib.lattice_step_many(hs, ns, len(lats)), lib)


class Lattice:
    """A lattice on the GPU: create, step, query, checkpoint, destroy."""

    def __init__(self, nx, ny, nz, F, omega, solid, *, periodic=(1, 1, 1), alpha=0.005,
                 dt=5e-6, kT=1.0, rho0=None, weight_dtype=0, msd_axes=0, init=0, ghost=0,
                 stream=None, allocator="torch", alpha_links=None, reservoirs=None, region=None,
                 n_regions=0, slab=False):
        """reservoirs: None or 6 faces (f = 2 a + side), each None (wall) or
        (F_res, rho_res, m_res complex); region: None or per-site labels
        < n_regions for region-resolved sums.  slab: a slab of a lattice
        decomposed along z (``lattice_create_slab``): nz is the slab's own
        planes and the fields hold nz + 2 planes (a halo plane on each side);
        queries return the own planes."""
        self.lib = B.load()
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.slab = bool(slab)
        nfield = nx * ny * (nz + 2) if slab else self.N
        self.msd_axes = msd_axes
        self.weight_dtype = int(weight_dtype)
        self.dt = dt
        p = B.lpc_params(nx, ny, nz, (ctypes.c_int32 * 3)(*[int(v) for v in periodic]),
                         float(alpha), float(dt), float(kT), int(weight_dtype), int(msd_axes),
                         int(init), int(ghost))
        F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1)
        om = np.ascontiguousarray(omega, dtype=np.float64).reshape(-1)
        sol = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
        if F.size != nfield or om.size != nfield or sol.size != nfield:
            raise ValueError("field sizes do not match the lattice")
        r0 = None
        if rho0 is not None:
            r0 = np.ascontiguousarray(rho0, dtype=np.float64).reshape(-1)
            if r0.size != nfield:
                raise ValueError("rho0 size does not match the lattice")
        links = None
        if alpha_links is not None:
            links = np.ascontiguousarray(alpha_links, dtype=np.float64).reshape(-1)
            if links.size != 3 * nfield:
                raise ValueError("alpha_links must hold 3 values per site")
        opts = None
        self.n_regions = 0
        if reservoirs is not None or region is not None or (slab and links is not None):
            opts = B.lpc_options()
            if links is not None:
                opts.alpha_links = links.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            for f, e in enumerate(reservoirs or ()):
                if e is None:
                    continue
                F_res, rho_res, m_res = e
                opts.reservoir[f] = B.lpc_reservoir(1, 0, float(F_res), float(rho_res),
                                                    complex(m_res).real, complex(m_res).imag)
            if region is not None:
                reg = np.ascontiguousarray(region, dtype=np.uint8).reshape(-1)
                if reg.size != self.N:
                    raise ValueError("region labels must hold one value per site")
                self._region = reg
                opts.region = reg.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
                opts.n_regions = int(n_regions)
                self.n_regions = int(n_regions)
        self._alloc = None
        aptr = None
        if allocator == "torch":
            self._alloc = TorchAllocator()
            aptr = ctypes.byref(self._alloc.struct)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = int(stream)
        h = ctypes.c_void_p()
        if slab:
            st = self.lib.lattice_create_slab(ctypes.byref(p), 1, ctypes.byref(opts) if opts is not None else None,
                                              _dp(F), _dp(om), sol.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                              _dp(r0) if r0 is not None else None, aptr,
                                              ctypes.c_void_p(self.stream), ctypes.byref(h))
        elif opts is not None:
            st = self.lib.lattice_create_ex(ctypes.byref(p), ctypes.byref(opts), _dp(F), _dp(om),
                                            sol.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                            _dp(r0) if r0 is not None else None, aptr,
                                            ctypes.c_void_p(self.stream), ctypes.byref(h))
        elif links is None:
            st = self.lib.lattice_create(ctypes.byref(p), _dp(F), _dp(om),
                                         sol.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                         _dp(r0) if r0 is not None else None, aptr,
                                         ctypes.c_void_p(self.stream), ctypes.byref(h))
        else:
            st = self.lib.lattice_create_links(ctypes.byref(p), _dp(F), _dp(om),
                                               sol.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                               _dp(r0) if r0 is not None else None, _dp(links), aptr,
                                               ctypes.c_void_p(self.stream), ctypes.byref(h))
        B.check(st, self.lib)
        self.h = h

    @classmethod
    def from_input(cls, inp, **kw):
        """Create from an ``lpc_inputs.LatticeInput``."""
        args = dict(periodic=inp.periodic, alpha=inp.alpha, dt=inp.dt, kT=inp.kT,
                    rho0=inp.rho0, weight_dtype=inp.weight_dtype, msd_axes=inp.msd_axes,
                    alpha_links=getattr(inp, "alpha_links", None),
                    reservoirs=getattr(inp, "reservoirs", None))
        args.update(kw)
        return cls(inp.nx, inp.ny, inp.nz, inp.F, inp.omega, inp.solid, **args)

    # -- lifetime --------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.lattice_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- stepping --------------------------------------------------------------
    def step(self, n):
        B.check(self.lib.lattice_step_n(self.h, int(n)), self.lib)

    def set_schedule(self, kernel, block_steps=1):
        B.check(self.lib.lattice_set_schedule(self.h, int(kernel), int(block_steps)), self.lib)

    def set_tiling(self, tile_rows=0, items_per_cta=0):
        """Tile rows (8, 12, 16) and work items per CTA of the TMA-fed one-step
        kernel; 0 = its heuristic (``lattice_set_tiling``)."""
        B.check(self.lib.lattice_set_tiling(self.h, int(tile_rows), int(items_per_cta)), self.lib)

    def set_static_form(self, form):
        """Static data form of the TMA-fed one-step kernel: B.LPC_STATIC_AUTO,
        _GATHER or _LINK (``lattice_set_static_form``)."""
        B.check(self.lib.lattice_set_static_form(self.h, int(form)), self.lib)

    def sync(self):
        B.check(self.lib.lattice_sync(self.h), self.lib)

    def slab_planes(self, which):
        """Device addresses and sizes of one plane of a slab's current state
        (``lattice_slab_planes``): a list of (address, bytes) for rho, m and
        the enabled moments, in the order rho, m, mu_x, mu_y, mu_z."""
        ps = B.lpc_plane_set()
        B.check(self.lib.lattice_slab_planes(self.h, int(which), ctypes.byref(ps)), self.lib)
        return [(ps.plane[q], ps.bytes[q]) for q in range(5) if ps.plane[q]]

    def autotune(self, trial_launches=6):
        """Time every schedule the ghost width allows and keep the fastest
        (``lattice_autotune``; the lattice's state is restored)."""
        k = ctypes.c_int32()
        d = ctypes.c_int32()
        r = ctypes.c_double()
        B.check(self.lib.lattice_autotune(self.h, int(trial_launches), ctypes.byref(k), ctypes.byref(d),
                                          ctypes.byref(r)), self.lib)
        return {"kernel": k.value, "block_steps": d.value, "rate": r.value}

    @property
    def steps_done(self):
        n = ctypes.c_int64()
        B.check(self.lib.lattice_steps_done(self.h, ctypes.byref(n)), self.lib)
        return n.value

    def info(self):
        i = B.lpc_info()
        B.check(self.lib.lattice_info(self.h, ctypes.byref(i)), self.lib)
        return {f: getattr(i, f) for f, _ in B.lpc_info._fields_}

    def equilibrate(self, threshold, max_iter, check_every=100):
        it = ctypes.c_int64()
        d = ctypes.c_double()
        B.check(self.lib.lattice_equilibrate(self.h, float(threshold), int(max_iter),
                                             int(check_every), ctypes.byref(it), ctypes.byref(d)),
                self.lib)
        return it.value, d.value

    # -- histories -------------------------------------------------------------
    def fid(self, first=0, count=None):
        """M(n) for n in [first, first+count) as complex128."""
        if count is None:
            count = self.steps_done + 1 - first
        out = np.empty(2 * count)
        B.check(self.lib.lattice_fid(self.h, int(first), int(count), _dp(out)), self.lib)
        return out[0::2] + 1j * out[1::2]

    def population(self, first=0, count=None):
        if count is None:
            count = self.steps_done + 1 - first
        out = np.empty(count)
        B.check(self.lib.lattice_population(self.h, int(first), int(count), _dp(out)), self.lib)
        return out

    def msd(self, axis, first=0, count=None):
        if count is None:
            count = self.steps_done + 1 - first
        out = np.empty(count)
        B.check(self.lib.lattice_msd(self.h, int(axis), int(first), int(count), _dp(out)), self.lib)
        return out

    def dmsd(self, axis, first=0, count=None):
        """Per-step MSD increments dMSD_axis(n), n in [first, first+count) (unnormalised)."""
        if count is None:
            count = self.steps_done - first
        out = np.empty(count)
        B.check(self.lib.lattice_dmsd(self.h, int(axis), int(first), int(count), _dp(out)), self.lib)
        return out

    def fid_region(self, region, first=0, count=None):
        """M_r(n): the FID summed over the sites labelled ``region``."""
        if count is None:
            count = self.steps_done + 1 - first
        out = np.empty(2 * count)
        B.check(self.lib.lattice_fid_region(self.h, int(region), int(first), int(count), _dp(out)), self.lib)
        return out[0::2] + 1j * out[1::2]

    def population_region(self, region, first=0, count=None):
        if count is None:
            count = self.steps_done + 1 - first
        out = np.empty(count)
        B.check(self.lib.lattice_population_region(self.h, int(region), int(first), int(count), _dp(out)),
                self.lib)
        return out

    def msd_region(self, region, axis, first=0, count=None):
        """The part of MSD_axis(n) accrued while particles were in ``region``."""
        if count is None:
            count = self.steps_done + 1 - first
        out = np.empty(count)
        B.check(self.lib.lattice_msd_region(self.h, int(region), int(axis), int(first), int(count), _dp(out)),
                self.lib)
        return out

    # -- fields ----------------------------------------------------------------
    def _host_out(self, out, count):
        """A caller-provided float32 host buffer of ``count`` values (e.g. a
        reused or pinned one: a fresh buffer's page faults cost more than the
        copy), or a new one."""
        if out is None:
            return np.empty(count, np.float32)
        out = np.asarray(out)
        if out.dtype != np.float32 or out.size != count or not out.flags["C_CONTIGUOUS"]:
            raise ValueError("out must be a C-contiguous float32 array of %d values" % count)
        return out.reshape(-1)

    def density(self, out=None):
        """Populations rho(x, n) as float32 (nz, ny, nx); ``out``: optional host buffer."""
        buf = self._host_out(out, self.N)
        B.check(self.lib.lattice_density(self.h, buf.ctypes.data_as(ctypes.c_void_p), 0), self.lib)
        return buf.reshape(self.shape)

    def density_device(self):
        """Densities as a torch CUDA tensor (copied on the lattice's stream)."""
        import torch
        t = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        B.check(self.lib.lattice_density(self.h, ctypes.c_void_p(t.data_ptr()), 1), self.lib)
        return t

    def magnetization(self):
        out = np.empty(2 * self.N, np.float32)
        B.check(self.lib.lattice_magnetization(self.h, out.ctypes.data_as(ctypes.c_void_p), 0),
                self.lib)
        return (out[0::2].astype(np.float64) + 1j * out[1::2]).reshape(self.shape)

    def moment(self, axis):
        out = np.empty(self.N, np.float32)
        B.check(self.lib.lattice_moment(self.h, int(axis), out.ctypes.data_as(ctypes.c_void_p), 0),
                self.lib)
        return out.reshape(self.shape)

    def weights(self):
        """Stored hop weights widened to float: shape (6, nz, ny, nx)."""
        out = np.empty(6 * self.N, np.float32)
        B.check(self.lib.lattice_weights(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
                self.lib)
        return out.reshape((6,) + self.shape)

    def rotation(self):
        out = np.empty(2 * self.N, np.float32)
        B.check(self.lib.lattice_rotation(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
                self.lib)
        return out.reshape(self.shape + (2,))

    def solid_mask(self):
        out = np.empty(self.N, np.uint8)
        B.check(self.lib.lattice_solid(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))),
                self.lib)
        return out.reshape(self.shape)

    # -- checkpoint ------------------------------------------------------------
    def get_state(self):
        n = ctypes.c_size_t()
        B.check(self.lib.lattice_state_size(self.h, ctypes.byref(n)), self.lib)
        buf = ctypes.create_string_buffer(n.value)
        B.check(self.lib.lattice_get_state(self.h, buf, n.value), self.lib)
        return bytes(buf.raw)

    def set_state(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        B.check(self.lib.lattice_set_state(self.h, buf, len(blob)), self.lib)
