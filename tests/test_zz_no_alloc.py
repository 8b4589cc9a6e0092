"""The no-allocation step entry point, lpc_step_noalloc.

It serves callers that cannot allocate device memory where they advance the
lattice (their device memory is reserved once through their own pool, or
they are plain C hosts without allocator hooks): they pass their own device
buffers, and the call uses only a fixed scratch array inside the library.
Two calls in a row through the C ABI must reproduce two steps of the
library's own entry point (lattice_step_n) within the parity tolerance of
the other GPU tests.  This file sorts last so that a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import lpc_inputs
from paper_2603_22553_b300 import binding as B
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_two_calls_match_lattice_step():
    import torch
    from paper_2603_22553_b300.lattice import Lattice

    lib = B.load()
    inp = lpc_inputs.random_case((10, 23, 45), 77, periodic=(1, 0, 1), alpha=0.7, msd_axes=0)
    lat = Lattice.from_input(inp)
    w = lat.weights().reshape(-1)
    R = lat.rotation().reshape(-1)
    rho0 = lat.density().reshape(-1)
    m0c = lat.magnetization().reshape(-1)
    m0 = np.stack([m0c.real, m0c.imag], axis=1).astype(np.float32).reshape(-1)

    dev = torch.device("cuda")
    tw = torch.from_numpy(w).to(dev)
    tR = torch.from_numpy(R).to(dev)
    r = [torch.from_numpy(rho0).to(dev), torch.empty_like(torch.from_numpy(rho0), device=dev)]
    m = [torch.from_numpy(m0).to(dev), torch.empty_like(torch.from_numpy(m0), device=dev)]
    sums = [torch.zeros(3, dtype=torch.float64, device=dev) for _ in range(2)]
    per = (ctypes.c_int32 * 3)(*inp.periodic)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    dens, fid, pop = [], [], []
    for call in range(2):
        src, dst = call % 2, (call + 1) % 2
        st = lib.lpc_step_noalloc(inp.nx, inp.ny, inp.nz, per, _ptr(tw), _ptr(tR), _ptr(r[src]),
                                  _ptr(m[src]), _ptr(r[dst]), _ptr(m[dst]), _ptr(sums[call]), stream)
        B.check(st, lib)
        torch.cuda.synchronize()
        dens.append(r[dst].cpu().numpy().astype(np.float64))
        s = sums[call].cpu().numpy()
        fid.append(s[0] + 1j * s[1])
        pop.append(s[2])

    lat.step(2)
    ref_M = lat.fid()
    ref_P = lat.population()
    ref = Lattice.from_input(inp)
    ref.step(1)
    ref_d1 = ref.density().reshape(-1).astype(np.float64)
    ref.close()
    ref_d2 = lat.density().reshape(-1).astype(np.float64)
    lat.close()

    assert H.rel_l2(dens[0], ref_d1) <= 1e-5
    assert H.rel_l2(dens[1], ref_d2) <= 1e-5
    for n in (1, 2):
        assert abs(fid[n - 1] - ref_M[n]) <= 1e-6 * abs(ref_M[n])
        assert abs(pop[n - 1] - ref_P[n]) <= 1e-6 * ref_P[n]


def test_noalloc_rejects_more_planes_than_its_scratch():
    lib = B.load()
    per = (ctypes.c_int32 * 3)(1, 1, 1)
    dummy = ctypes.c_void_p(256)
    st = lib.lpc_step_noalloc(4, 4, 5000, per, dummy, dummy, dummy, dummy, ctypes.c_void_p(512),
                              ctypes.c_void_p(768), dummy, None)
    assert st == B.LPC_ERR_INVALID
    assert b"4096" in lib.lpc_last_error()
