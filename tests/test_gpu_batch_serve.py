"""GPU tests of batched stepping (lattice_step_many) and of the serving loop.

* Batched launches give states bit-identical to lattice_step_n, sums within
  FP32 rounding of it, and results bit-identical whether a lattice is
  advanced alone or in a batch with other lattices of other sizes, weight
  types and MSD masks.
* A served stream returns, for every request, the FID it gets when served
  alone, bit for bit, and matches the FP64 oracle.
"""
import numpy as np
import pytest

import lpc_inputs
import oracle
from paper_2603_22553_b300.lattice import Lattice, step_many
from tests import helpers as H

pytestmark = pytest.mark.gpu


def _cases():
    return [
        lpc_inputs.random_case((7, 20, 33), 501, periodic=(1, 1, 1), alpha=0.6, msd_axes=0),
        lpc_inputs.random_case((17, 9, 40), 502, periodic=(0, 1, 1), alpha=0.8, msd_axes=0),
        lpc_inputs.random_case((24, 24, 24), 503, periodic=(1, 1, 1), alpha=0.5, msd_axes=1),
        lpc_inputs.random_case((5, 30, 70), 504, periodic=(1, 0, 1), alpha=0.7, msd_axes=0,
                               weight_dtype=1),
        lpc_inputs.random_case((33, 16, 16), 505, periodic=(1, 1, 0), alpha=0.4, msd_axes=0),
    ]


def _read(lat, msd):
    out = {"rho": lat.density(), "m": lat.magnetization(), "M": lat.fid(), "P": lat.population()}
    for a in range(3):
        if msd >> a & 1:
            out["msd%d" % a] = lat.msd(a)
    return out


def test_step_many_alone_vs_mixed_and_vs_step_n():
    cases = _cases()
    steps = [40, 25, 31, 40, 12]
    mixed = [Lattice.from_input(c) for c in cases]
    step_many(mixed, steps)
    res_mixed = [_read(l, c.msd_axes) for l, c in zip(mixed, cases)]
    for i, c in enumerate(cases):
        alone = Lattice.from_input(c)
        step_many([alone], [steps[i]])
        ra = _read(alone, c.msd_axes)
        for k in ra:
            assert np.array_equal(ra[k], res_mixed[i][k]), (i, k)
        ref = Lattice.from_input(c)
        ref.step(steps[i])
        rr = _read(ref, c.msd_axes)
        assert np.array_equal(rr["rho"], ra["rho"])
        assert np.array_equal(rr["m"], ra["m"])
        assert np.allclose(rr["M"], ra["M"], rtol=1e-6, atol=1e-6 * abs(rr["M"][0]))
        o = H.oracle_run(c, steps[i], H.MODE_OF_DTYPE[c.weight_dtype])
        g = dict(ra)
        g["rho"] = ra["rho"].astype(np.float64)
        H.compare(g, o, c.msd_axes, tol=1e-5)
        for l in (alone, ref):
            l.close()
    for l in mixed:
        l.close()


def test_step_many_interleaved_with_step_n():
    cases = _cases()[:3]
    a = [Lattice.from_input(c) for c in cases]
    b = [Lattice.from_input(c) for c in cases]
    step_many(a, [10, 10, 10])
    a[1].step(7)                      # one-step kernel in between
    step_many(a, [5, 0, 9])
    for l, n in zip(b, [15, 17, 19]):
        l.step(n)
    for la, lb in zip(a, b):
        assert la.steps_done == lb.steps_done
        assert np.array_equal(la.density(), lb.density())
        assert np.allclose(la.fid(), lb.fid(), rtol=1e-6, atol=1e-6 * abs(lb.fid()[0]))
    for l in a + b:
        l.close()


def test_served_results_equal_alone_and_oracle():
    import torch
    from paper_2603_22553_b300.serve import GpuEngine, Server, summary

    reqs = lpc_inputs.request_stream(n=14, seed=44, edge_lo=24, edge_hi=48, steps_lo=60,
                                     steps_hi=400, rate_per_s=400.0)
    eng = GpuEngine()
    srv = Server(eng, 8 << 30, max_active=6, quantum=64, prefetch=2)
    recs = srv.run(reqs, realtime=True)
    s = summary(recs)
    assert s["requests"] == len(reqs)
    for r, rec in zip(sorted(reqs, key=lambda q: q.arrival_s), recs):
        alone = Server(eng, 8 << 30, max_active=1, quantum=64, prefetch=1).run([r], realtime=False)[0]
        assert np.array_equal(alone.fid, rec.fid), r.rid
    for r in reqs[:2]:
        inp = r.lattice()
        o = H.oracle_run(inp, r.steps, oracle.MODE_F32, msd_axes=0)
        rec = next(x for x in recs if x.rid == r.rid)
        assert H.rel_l2(rec.fid, o.M) <= 1e-5
    torch.cuda.synchronize()


@pytest.mark.parametrize("mode", ["streams", "batched"])
def test_served_tma_lattices_equal_alone(mode):
    """Requests large enough for the one-step TMA kernel are served side by
    side, each on its own stream or together in multi-lattice launches; every
    FID is bit-identical to the request served alone."""
    import torch
    from paper_2603_22553_b300.serve import GpuEngine, Server

    reqs = lpc_inputs.request_stream(n=6, seed=45, edge_lo=102, edge_hi=124, steps_lo=40,
                                     steps_hi=150, rate_per_s=1000.0)
    eng = GpuEngine(mode=mode)
    recs = Server(eng, 16 << 30, max_active=4, quantum=32, prefetch=2).run(reqs, realtime=True)
    for r, rec in zip(sorted(reqs, key=lambda q: q.arrival_s), recs):
        alone = Server(eng, 16 << 30, max_active=1, quantum=32, prefetch=1).run([r], realtime=False)[0]
        assert np.array_equal(alone.fid, rec.fid), r.rid
    torch.cuda.synchronize()


def test_step_many_multi_lattice_tma_launch_equals_own_launches():
    """Lattices on the TMA-fed one-step kernel (mid-size, gather form) advance
    together in one multi-lattice launch per step: each lattice's states and
    FID / population histories are bit-identical to its own lattice_step_n
    run (the same work items and the same fixed-order reductions), whatever
    lattices share the launch; and they match the FP64 oracle."""
    from paper_2603_22553_b300 import binding as B
    shapes = [((64, 96, 110), (1, 1, 1), 0), ((70, 70, 128), (1, 0, 1), 0), ((40, 100, 96), (0, 1, 0), 0),
              ((30, 64, 200), (1, 1, 1), 1), ((36, 70, 130), (1, 1, 0), 1)]
    cases = [lpc_inputs.random_case(sh, 610 + i, periodic=per, alpha=0.6, msd_axes=0, weight_dtype=wd)
             for i, (sh, per, wd) in enumerate(shapes)]
    steps = [23, 40, 17, 40, 9]

    def make(c):
        lat = Lattice.from_input(c)
        lat.set_schedule(B.LPC_KERNEL_TB, 1)
        lat.set_static_form(B.LPC_STATIC_GATHER)
        return lat

    mixed = [make(c) for c in cases]
    step_many(mixed, steps)
    res_mixed = [_read(l, 0) for l in mixed]
    for l in mixed:
        l.close()
    # two other mixes: every lattice with one other, and in reverse order
    for i, c in enumerate(cases):
        ref = make(c)
        ref.step(steps[i])
        rr = _read(ref, 0)
        ref.close()
        for k in rr:
            assert np.array_equal(rr[k], res_mixed[i][k]), (i, k)
        j = (i + 1) % len(cases)
        pair = [make(cases[j]), make(c)]
        step_many(pair, [steps[j], steps[i]])
        rp = _read(pair[1], 0)
        for l in pair:
            l.close()
        for k in rr:
            assert np.array_equal(rr[k], rp[k]), (i, k)
        if i < 2:
            o = H.oracle_run(c, steps[i], H.MODE_OF_DTYPE[c.weight_dtype], msd_axes=0)
            g = dict(rr)
            g["rho"] = rr["rho"].astype(np.float64)
            H.compare(g, o, 0, tol=1e-5)
