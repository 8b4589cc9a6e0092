"""CPU checks of the C ABI: the in-tree library loads, exports every function
that include/*.h declares, and rejects invalid arguments on the host before
any device work (no GPU needed for these calls)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2603_22553_b300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b([a-z][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            name = m.group(1)
            if name.startswith(("lattice_", "lpc_")):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_22553_b300 import build
    build.build_library()
    return B.load()


def test_header_declares_the_core_calls():
    names = declared_functions()
    for n in ("lattice_create", "lattice_step_n", "lattice_fid", "lattice_density",
              "lattice_msd", "lattice_destroy", "lpc_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    raw = ctypes.CDLL(B.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), "missing export: " + n
        assert n in B.SIGNATURES, "binding lacks " + n


def test_version_and_error_string(lib):
    assert b"sm_103a" in lib.lpc_version()
    assert isinstance(lib.lpc_last_error(), bytes)


def _params(**kw):
    d = dict(nx=4, ny=4, nz=4, periodic=(1, 1, 1), alpha=0.5, dt=5e-6, kT=1.0, weight_dtype=0,
             msd_axes=0, init=0, ghost=0)
    d.update(kw)
    per = (ctypes.c_int32 * 3)(*d.pop("periodic"))
    return B.lpc_params(d["nx"], d["ny"], d["nz"], per, d["alpha"], d["dt"], d["kT"],
                        d["weight_dtype"], d["msd_axes"], d["init"], d["ghost"])


def _create(lib, p, F=None, om=None, solid=None, rho0=None):
    N = p.nx * p.ny * p.nz if p.nx > 0 and p.ny > 0 and p.nz > 0 else 1
    F = np.zeros(N) if F is None else F
    om = np.zeros(N) if om is None else om
    solid = np.zeros(N, np.uint8) if solid is None else solid
    h = ctypes.c_void_p()
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = lib.lattice_create(ctypes.byref(p), dp(F), dp(om),
                            solid.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                            dp(rho0) if rho0 is not None else None, None, None, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("kw,msg", [
    (dict(nx=0), "edges"), (dict(alpha=0.0), "alpha"), (dict(alpha=1.5), "alpha"),
    (dict(kT=0.0), "kT"), (dict(weight_dtype=3), "weight_dtype"), (dict(msd_axes=9), "msd_axes"),
    (dict(init=7), "init"), (dict(ghost=9), "ghost"), (dict(ghost=3), "ghost"),
    (dict(periodic=(2, 1, 1)), "periodic"),
])
def test_invalid_parameters_rejected_on_host(lib, kw, msg):
    st, h = _create(lib, _params(**kw))
    assert st == B.LPC_ERR_INVALID
    assert not h.value
    assert msg in lib.lpc_last_error().decode()


def test_non_finite_inputs_rejected(lib):
    p = _params()
    F = np.zeros(64)
    F[5] = np.nan
    st, _ = _create(lib, p, F=F)
    assert st == B.LPC_ERR_INVALID and b"F" in lib.lpc_last_error()
    # a NaN free energy on a solid site is ignored by validation (solid sites have no F)
    om = np.zeros(64)
    om[3] = np.inf
    st, _ = _create(lib, p, om=om)
    assert st == B.LPC_ERR_INVALID and b"omega" in lib.lpc_last_error()


def test_null_handle_calls(lib):
    assert lib.lattice_step_n(None, 1) == B.LPC_ERR_INVALID
    assert lib.lattice_destroy(None) == B.LPC_OK
    out = np.zeros(2)
    assert lib.lattice_fid(None, 0, 1, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == B.LPC_ERR_INVALID
    assert lib.lattice_step_many(None, None, -1) == B.LPC_ERR_INVALID
    assert lib.lattice_set_static_form(None, B.LPC_STATIC_LINK) == B.LPC_ERR_INVALID


@pytest.mark.parametrize("bad", [1.5, -0.1, float("nan")])
def test_link_factors_outside_unit_interval_rejected(lib, bad):
    p = _params()
    z = np.zeros(64)
    links = np.full(3 * 64, 0.5)
    links[70] = bad
    h = ctypes.c_void_p()
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = lib.lattice_create_links(ctypes.byref(p), dp(z), dp(z),
                                  np.zeros(64, np.uint8).ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                  None, dp(links), None, None, ctypes.byref(h))
    assert st == B.LPC_ERR_INVALID and not h.value
    assert b"link" in lib.lpc_last_error()


def _create_ex(lib, p, opts):
    N = p.nx * p.ny * p.nz
    z = np.zeros(N)
    h = ctypes.c_void_p()
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = lib.lattice_create_ex(ctypes.byref(p), ctypes.byref(opts), dp(z), dp(z),
                               np.zeros(N, np.uint8).ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                               None, None, None, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("face,periodic,vals,msg", [
    (0, (1, 1, 1), (0.0, 1.0, 1.0), "non-periodic"),       # reservoir on a periodic axis
    (4, (0, 0, 1), (0.0, 1.0, 1.0), "non-periodic"),       # a z reservoir on a periodic z
    (2, (1, 0, 1), (float("nan"), 1.0, 1.0), "non-finite"),
    (3, (1, 0, 1), (0.0, float("inf"), 1.0), "non-finite"),
])
def test_invalid_reservoirs_rejected_on_host(lib, face, periodic, vals, msg):
    opts = B.lpc_options()
    opts.reservoir[face] = B.lpc_reservoir(1, 0, vals[0], vals[1], vals[2], 0.0)
    st, h = _create_ex(lib, _params(periodic=periodic), opts)
    assert st == B.LPC_ERR_INVALID and not h.value
    assert msg in lib.lpc_last_error().decode()


@pytest.mark.parametrize("labels_max,n_regions", [(3, 3), (0, 0), (0, 5), (1, -1)])
def test_invalid_regions_rejected_on_host(lib, labels_max, n_regions):
    p = _params()
    opts = B.lpc_options()
    lab = np.zeros(64, np.uint8)
    lab[17] = labels_max
    opts.region = lab.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    opts.n_regions = n_regions
    st, h = _create_ex(lib, p, opts)
    assert st == B.LPC_ERR_INVALID and not h.value
    assert b"region" in lib.lpc_last_error()


def test_region_queries_reject_null_handle(lib):
    out = np.zeros(4)
    dp = out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.lattice_fid_region(None, 0, 0, 1, dp) == B.LPC_ERR_INVALID
    assert lib.lattice_population_region(None, 0, 0, 1, dp) == B.LPC_ERR_INVALID
    assert lib.lattice_msd_region(None, 0, 0, 0, 1, dp) == B.LPC_ERR_INVALID


def test_padded_size_limit_rejected_on_host(lib):
    """The ghost-padded arrays must hold fewer than 2^31 sites (32-bit plane
    offsets in the kernels): 2048 x 1020 x 1020 pads to 2080 x 1024 x 1020."""
    N = 2048 * 1020 * 1020
    p = _params(nx=2048, ny=1020, nz=1020)
    z = np.zeros(1)
    h = ctypes.c_void_p()
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    # valid pointers are never read: the size check comes first
    F = np.zeros(16)
    st = lib.lattice_create(ctypes.byref(p), dp(F), dp(F), np.zeros(16, np.uint8).ctypes.data_as(
        ctypes.POINTER(ctypes.c_uint8)), None, None, None, ctypes.byref(h))
    assert st == B.LPC_ERR_INVALID and not h.value
    assert b"2^31" in lib.lpc_last_error()
    assert N < 2 ** 31 - 1       # the interior alone would fit


def test_wait_selftest_rejects_bad_arguments_on_host(lib):
    assert lib.lpc_wait_selftest(3, 100, None) == B.LPC_ERR_INVALID
    assert b"mode" in lib.lpc_last_error()
    assert lib.lpc_wait_selftest(0, 0, None) == B.LPC_ERR_INVALID
    assert lib.lpc_wait_selftest(1, 4_000_000_001, None) == B.LPC_ERR_INVALID
    assert b"budget" in lib.lpc_last_error()


def _create_slab(lib, p, halo=1, opts=None, rho0=None):
    N = p.nx * p.ny * (p.nz + 2)
    z = np.zeros(N)
    h = ctypes.c_void_p()
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st = lib.lattice_create_slab(ctypes.byref(p), halo, ctypes.byref(opts) if opts is not None else None, dp(z),
                                 dp(z), np.zeros(N, np.uint8).ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                 dp(rho0) if rho0 is not None else None, None, None, ctypes.byref(h))
    return st, h


def test_slab_arguments_rejected_on_host(lib):
    """Slab misuse is rejected before any device work: a halo other than one
    plane, region labels, a Boltzmann start without rho0, a z reservoir, and
    plane queries on a NULL handle."""
    st, h = _create_slab(lib, _params(), halo=2)
    assert st == B.LPC_ERR_INVALID and not h.value and b"halo" in lib.lpc_last_error()
    opts = B.lpc_options()
    lab = np.zeros(4 * 4 * 6, np.uint8)
    opts.region = lab.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    opts.n_regions = 1
    st, h = _create_slab(lib, _params(), opts=opts)
    assert st == B.LPC_ERR_INVALID and b"region" in lib.lpc_last_error()
    st, h = _create_slab(lib, _params(init=1))
    assert st == B.LPC_ERR_INVALID and b"rho0" in lib.lpc_last_error()
    opts = B.lpc_options()
    opts.reservoir[4] = B.lpc_reservoir(1, 0, 0.0, 1.0, 1.0, 0.0)
    st, h = _create_slab(lib, _params(periodic=(1, 1, 0)), opts=opts)
    assert st == B.LPC_ERR_INVALID and b"halo planes" in lib.lpc_last_error()
    ps = B.lpc_plane_set()
    assert lib.lattice_slab_planes(None, 0, ctypes.byref(ps)) == B.LPC_ERR_INVALID
    assert lib.lattice_set_tiling(None, 16, 40) == B.LPC_ERR_INVALID
    out = np.zeros(4)
    assert lib.lattice_dmsd(None, 0, 0, 1, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == B.LPC_ERR_INVALID
