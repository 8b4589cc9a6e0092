"""Shared helpers of the GPU tests: run a case through the C ABI and through
the FP64 oracle on the same seeded inputs, and compare."""
import numpy as np

import lpc_inputs
import oracle

MODE_OF_DTYPE = {0: oracle.MODE_F32, 1: oracle.MODE_BF16}


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def gpu_run(inp, steps, rho0=None, schedule=None, chunks=None, **kw):
    from paper_2603_22553_b300.lattice import Lattice
    args = dict(rho0=rho0 if rho0 is not None else inp.rho0)
    args.update(kw)
    lat = Lattice.from_input(inp, **args)
    if schedule is not None:
        lat.set_schedule(*schedule)
    if chunks:
        for c in chunks:
            lat.step(c)
    else:
        lat.step(steps)
    out = dict(M=lat.fid(), P=lat.population(), rho=lat.density().astype(np.float64),
               m=lat.magnetization())
    axes = args.get("msd_axes", inp.msd_axes)
    for a in range(3):
        if axes >> a & 1:
            out["msd%d" % a] = lat.msd(a)
            out["mu%d" % a] = lat.moment(a).astype(np.float64)
    out["lattice"] = lat
    return out


def oracle_run(inp, steps, mode=oracle.MODE_EXACT, rho0=None, msd_axes=None):
    pk = oracle.pack_input(inp, mode)
    r0 = rho0 if rho0 is not None else (inp.rho0 if inp.rho0 is not None else inp.uniform_rho0())
    axes = inp.msd_axes if msd_axes is None else msd_axes
    return oracle.run(pk, r0, steps, msd_axes=axes)


def compare(g, o, axes, tol=1e-4, msd_from=10):
    """Parity of FID, population, densities, magnetisation and MSD."""
    errs = {
        "fid": rel_l2(g["M"], o.M),
        "pop": float(np.max(np.abs(g["P"] / o.P - 1.0))),
        "rho": rel_l2(g["rho"], o.rho),
        "m": rel_l2(g["m"], o.m),
    }
    for a in range(3):
        if axes >> a & 1:
            ref = o.msd(a)
            got = g["msd%d" % a]
            sl = slice(msd_from, None)
            if len(ref) > msd_from:
                r, gg = ref[sl], got[sl]
                nz = np.abs(r) > 1e-30
                e = float(np.max(np.abs(gg[nz] - r[nz]) / np.abs(r[nz]))) if nz.any() else 0.0
                if (~nz).any():
                    e = max(e, float(np.max(np.abs(gg[~nz]))))
                errs["msd%d" % a] = e
    for k, v in errs.items():
        assert v <= tol, "%s error %.3e > %.1e (all: %s)" % (k, v, tol, errs)
    return errs


def small_cases():
    """Ragged shapes spanning several 32 x 8 tiles, walls and periodic axes."""
    return [
        lpc_inputs.random_case((11, 29, 37), 101, periodic=(1, 1, 1), alpha=0.7, msd_axes=7),
        lpc_inputs.random_case((9, 40, 70), 102, periodic=(0, 1, 1), alpha=0.5, msd_axes=1),
        lpc_inputs.random_case((13, 17, 33), 103, periodic=(1, 0, 0), alpha=1.0, msd_axes=6),
        lpc_inputs.random_case((5, 3, 65), 104, periodic=(1, 1, 0), alpha=0.9, msd_axes=0),
    ]
