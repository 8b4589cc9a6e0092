"""The no-allocation step entry point, lpc_step_noalloc.

It serves callers that cannot allocate device memory where they advance the
lattice (their device memory is reserved once through their own pool, or
they are plain C hosts without allocator hooks): they pass their own device
buffers, and the call uses only a fixed scratch array inside the library.
Two calls in a row through the C ABI must reproduce two steps of the
library's own entry point (lattice_step_n): the states bit for bit (the same
per-site arithmetic), the FID and population sums within FP32 summation
order.  The shapes cover several 32-site x segments per row with the
periodic wrap between them, walls, and 1-thick periodic axes.  This file
sorts last so that a run that stops at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

import lpc_inputs
from paper_2603_22553_b300 import binding as B

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


# (nz, ny, nx), periodic flags per axis (x, y, z), seed
SHAPES = [
    ((10, 23, 45), (1, 0, 1), 77),
    ((3, 5, 70), (1, 1, 1), 78),      # three x segments per row, periodic wrap between them
    ((1, 1, 33), (1, 1, 1), 79),      # 1-thick periodic y and z: a site is its own neighbour
    ((1, 7, 1), (1, 0, 1), 80),       # 1-thick periodic x and z, walls in y
]


@pytest.mark.parametrize("shape,periodic,seed", SHAPES)
def test_noalloc_two_calls_match_lattice_step(shape, periodic, seed):
    import torch
    from paper_2603_22553_b300.lattice import Lattice

    lib = B.load()
    inp = lpc_inputs.random_case(shape, seed, periodic=periodic, alpha=0.7, msd_axes=0)
    lat = Lattice.from_input(inp)
    w = lat.weights().reshape(-1)
    R = lat.rotation().reshape(-1)
    rho0 = lat.density().reshape(-1)
    m0c = lat.magnetization().reshape(-1)
    m0 = np.stack([m0c.real, m0c.imag], axis=1).astype(np.float32).reshape(-1)

    dev = torch.device("cuda")
    tw = torch.from_numpy(w).to(dev)
    tR = torch.from_numpy(R).to(dev)
    r = [torch.from_numpy(rho0).to(dev), torch.empty(rho0.size, dtype=torch.float32, device=dev)]
    m = [torch.from_numpy(m0).to(dev), torch.empty(m0.size, dtype=torch.float32, device=dev)]
    sums = [torch.zeros(3, dtype=torch.float64, device=dev) for _ in range(2)]
    per = (ctypes.c_int32 * 3)(*inp.periodic)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    dens, mags, fid, pop = [], [], [], []
    for call in range(2):
        src, dst = call % 2, (call + 1) % 2
        st = lib.lpc_step_noalloc(inp.nx, inp.ny, inp.nz, per, _ptr(tw), _ptr(tR), _ptr(r[src]),
                                  _ptr(m[src]), _ptr(r[dst]), _ptr(m[dst]), _ptr(sums[call]), stream)
        B.check(st, lib)
        torch.cuda.synchronize()
        dens.append(r[dst].cpu().numpy().copy())
        mm = m[dst].cpu().numpy().reshape(-1, 2)
        mags.append(mm[:, 0].astype(np.float64) + 1j * mm[:, 1])
        s = sums[call].cpu().numpy()
        fid.append(s[0] + 1j * s[1])
        pop.append(s[2])

    # the library's own entry point, one step at a time
    ref_d, ref_m = [], []
    for _ in range(2):
        lat.step(1)
        ref_d.append(lat.density().reshape(-1))
        ref_m.append(lat.magnetization().reshape(-1))
    ref_M = lat.fid()
    ref_P = lat.population()
    lat.close()

    for n in range(2):
        assert np.array_equal(dens[n], ref_d[n]), "density after call %d differs" % (n + 1)
        assert np.array_equal(mags[n], ref_m[n]), "magnetisation after call %d differs" % (n + 1)
        # M and P: FP64 sums of FP32 partials, in another order than the library's
        assert abs(fid[n] - ref_M[n + 1]) <= 1e-6 * abs(ref_P[0])
        assert abs(pop[n] - ref_P[n + 1]) <= 1e-6 * ref_P[0]


def test_noalloc_rejects_more_planes_than_its_scratch():
    """Host-side checks: they return before any device work."""
    lib = B.load()
    per = (ctypes.c_int32 * 3)(1, 1, 1)
    dummy = ctypes.c_void_p(256)
    st = lib.lpc_step_noalloc(4, 4, 5000, per, dummy, dummy, dummy, dummy, ctypes.c_void_p(512),
                              ctypes.c_void_p(768), dummy, None)
    assert st == B.LPC_ERR_INVALID
    assert b"4096" in lib.lpc_last_error()
    # a view one float into a buffer: m and R must be 8-byte aligned, w 4-byte
    a = [ctypes.c_void_p(1024 * (i + 1)) for i in range(7)]
    for bad, off in ((1, 4), (3, 4), (5, 4), (6, 4), (0, 2), (2, 2), (4, 2)):
        args = list(a)
        args[bad] = ctypes.c_void_p(args[bad].value + off)
        st = lib.lpc_step_noalloc(4, 4, 4, per, *args, None)
        assert st == B.LPC_ERR_INVALID, (bad, off)
        assert b"aligned" in lib.lpc_last_error()
