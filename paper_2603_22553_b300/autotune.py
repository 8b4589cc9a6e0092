"""Schedule autotuning with a persistent JSON cache.

``choose(lattice)`` returns the fastest step schedule (the register-pipelined
one-step kernel; the TMA-fed one-step kernel with its tile rows and work
items per CTA; or the temporally blocked kernel with depth K) for the
lattice's shape, boundary,
weight type, MSD mask, ghost width and GPU.  A cache miss runs
``lattice_autotune`` (which times every candidate on the lattice itself and
restores its state); a hit applies the cached choice with
``lattice_set_schedule`` and ``lattice_set_tiling``.  The cache file is ``$LPC3D_AUTOTUNE_CACHE`` or
``~/.cache/lpc3d_autotune.json``.
"""
from __future__ import annotations

import json
import os
import threading

_LOCK = threading.Lock()


def cache_path():
    return os.environ.get("LPC3D_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "lpc3d_autotune.json"))


def _device_name():
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "unknown"


def key(lat):
    info = lat.info()
    nz, ny, nx = lat.shape
    return "%dx%dx%d|w%d|msd%d|g%d|%s" % (nx, ny, nz, getattr(lat, "weight_dtype", 0), lat.msd_axes,
                                           info["ghost"], _device_name())


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def choose(lat, trial_launches=6, path=None, refresh=False):
    """Apply (and return) the cached or freshly measured best schedule."""
    path = path or cache_path()
    k = key(lat)
    with _LOCK:
        table = _load(path)
    if not refresh and k in table:
        c = table[k]
        lat.set_schedule(c["kernel"], c["block_steps"])
        lat.set_tiling(c.get("tile_rows", 0), c.get("items_per_cta", 0))
        return dict(c, cached=True)
    c = lat.autotune(trial_launches)
    info = lat.info()
    c.update(tile_rows=info["tile_rows"], items_per_cta=info["items_per_cta"])
    with _LOCK:
        table = _load(path)
        table[k] = c
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return dict(c, cached=False)
