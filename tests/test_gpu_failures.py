"""GPU tests of failure detection, with no GPU fault, trap or hang.

* Device allocations that fail (injected through the caller's allocator
  hooks: the k-th allocation returns NULL) make lattice_create,
  lattice_step_n (history growth) and queries that need a temporary buffer
  return LPC_ERR_OOM; every block taken is handed back and the device stays
  usable.
* A bounded device wait that runs out (an mbarrier that never completes, a
  flag that nothing sets; a budget of about a millisecond) makes the kernel
  return LPC_ERR_TIMEOUT instead of hanging, and the context stays usable.
"""
import ctypes

import numpy as np
import pytest

import lpc_inputs
from paper_2603_22553_b300 import binding as B

pytestmark = pytest.mark.gpu


class InjectingAllocator:
    """lpc_allocator over PyTorch's caching allocator whose allocation number
    ``fail_at`` (and every later one if ``fail_after``) returns NULL."""

    def __init__(self, fail_at=None, fail_after=False):
        import torch
        self.torch = torch
        self.fail_at = fail_at
        self.fail_after = fail_after
        self.count = 0
        self.live = {}
        self.bad_frees = 0
        dev = torch.cuda.current_device()

        def _alloc(nbytes, stream, ctx):
            i = self.count
            self.count += 1
            if self.fail_at is not None and (i == self.fail_at or (self.fail_after and i > self.fail_at)):
                return None
            p = int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0)))
            self.live[p] = int(nbytes)
            return p

        def _free(ptr, stream, ctx):
            if ptr not in self.live:
                self.bad_frees += 1
                return
            del self.live[ptr]
            torch.cuda.caching_allocator_delete(int(ptr))

        self._a = B.ALLOC_FN(_alloc)
        self._f = B.FREE_FN(_free)
        self.struct = B.lpc_allocator(self._a, self._f, None)


def _create(lib, inp, alloc):
    p = B.lpc_params(inp.nx, inp.ny, inp.nz, (ctypes.c_int32 * 3)(*inp.periodic), inp.alpha, inp.dt, inp.kT,
                     inp.weight_dtype, inp.msd_axes, 0, 0)
    h = ctypes.c_void_p()
    dp = lambda a: np.ascontiguousarray(a, dtype=np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    F = np.ascontiguousarray(inp.F, dtype=np.float64)
    om = np.ascontiguousarray(inp.omega, dtype=np.float64)
    so = np.ascontiguousarray(inp.solid, dtype=np.uint8)
    st = lib.lattice_create(ctypes.byref(p), dp(F), dp(om), so.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                            None, ctypes.byref(alloc.struct), None, ctypes.byref(h))
    return st, h


def test_injected_allocation_failures_return_oom():
    import torch
    lib = B.load()
    inp = lpc_inputs.random_case((8, 9, 10), 901, periodic=(1, 1, 0), alpha=0.6, msd_axes=1)
    clean = InjectingAllocator()
    st, h = _create(lib, inp, clean)
    B.check(st, lib)
    n_create = clean.count
    assert n_create >= 8
    B.check(lib.lattice_destroy(h), lib)
    assert not clean.live and clean.bad_frees == 0

    # every allocation of create fails once in turn
    for k in range(n_create):
        a = InjectingAllocator(fail_at=k)
        st, h = _create(lib, inp, a)
        assert st == B.LPC_ERR_OOM, (k, st)
        assert not h.value
        assert b"alloc" in lib.lpc_last_error()
        assert not a.live and a.bad_frees == 0, k

    # after create every allocation fails: history growth and temporaries
    a = InjectingAllocator(fail_at=n_create, fail_after=True)
    st, h = _create(lib, inp, a)
    B.check(st, lib)
    B.check(lib.lattice_step_n(h, 1000), lib)            # within the initial history
    assert lib.lattice_step_n(h, 100) == B.LPC_ERR_OOM    # needs a larger history
    done = ctypes.c_int64()
    B.check(lib.lattice_steps_done(h, ctypes.byref(done)), lib)
    assert done.value == 1000
    w = np.zeros(6 * inp.n_sites, np.float32)
    assert lib.lattice_weights(h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))) == B.LPC_ERR_OOM
    # the lattice is still usable: its history up to the last completed step reads back
    M = np.zeros(2 * 1001)
    B.check(lib.lattice_fid(h, 0, 1001, M.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), lib)
    assert np.all(np.isfinite(M)) and M[0] > 0
    B.check(lib.lattice_destroy(h), lib)
    assert not a.live and a.bad_frees == 0
    torch.cuda.synchronize()


@pytest.mark.parametrize("mode,expect", [(0, B.LPC_ERR_TIMEOUT), (1, B.LPC_ERR_TIMEOUT), (2, B.LPC_OK)])
def test_bounded_wait_that_runs_out_reports_timeout(mode, expect):
    import torch
    from paper_2603_22553_b300.lattice import Lattice
    lib = B.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.lpc_wait_selftest(mode, 2_000_000, stream)       # about a millisecond
    assert st == expect, lib.lpc_last_error()
    if expect == B.LPC_ERR_TIMEOUT:
        assert b"ran out" in lib.lpc_last_error()
    # the context is still usable: a lattice steps and matches itself
    inp = lpc_inputs.random_case((6, 7, 8), 902, periodic=(1, 1, 1), alpha=0.5, msd_axes=0)
    lat = Lattice.from_input(inp)
    lat.step(20)
    P = lat.population()
    lat.close()
    assert np.allclose(P, P[0], rtol=1e-5)
    assert lib.lpc_wait_selftest(3, 100, stream) == B.LPC_ERR_INVALID
    assert lib.lpc_wait_selftest(0, 0, stream) == B.LPC_ERR_INVALID
    assert lib.lpc_wait_selftest(0, 5_000_000_000, stream) == B.LPC_ERR_INVALID


@pytest.mark.parametrize("field", ["F", "omega", "rho0", "links"])
def test_large_lattice_input_checks_on_the_device(field):
    """Lattices of 2^22 sites or more check their values on the device, in the
    uploaded copies (a host scan of gigabytes costs as much as the upload): a
    bad value still returns LPC_ERR_INVALID, no handle, and the device memory
    taken meanwhile is given back."""
    import torch
    from paper_2603_22553_b300.lattice import Lattice
    inp = lpc_inputs.random_case((64, 256, 260), 61, periodic=(1, 1, 1), alpha=0.6, msd_axes=0)
    assert inp.n_sites >= 1 << 22
    kw = {}
    pore = np.flatnonzero(inp.solid.reshape(-1) == 0)
    F, om = inp.F.copy(), inp.omega.copy()
    if field == "F":
        F.reshape(-1)[pore[-3]] = np.nan
    elif field == "omega":
        om.reshape(-1)[7] = np.inf
    elif field == "rho0":
        r0 = np.ones(inp.n_sites)
        r0[pore[1000]] = np.nan
        kw["rho0"] = r0
    else:
        links = np.full((3,) + inp.F.shape, 0.5)
        links.reshape(-1)[12345] = 1.5
        kw["alpha_links"] = links
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    with pytest.raises(B.LPCError) as ei:
        Lattice(inp.nx, inp.ny, inp.nz, F, om, inp.solid, periodic=inp.periodic, alpha=inp.alpha, **kw)
    assert ei.value.status == B.LPC_ERR_INVALID
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
    ok = Lattice.from_input(inp)
    ok.step(3)
    assert ok.steps_done == 3
    ok.close()
