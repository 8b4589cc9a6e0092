"""Throughput of the lattice-propagation step on B300.

One bench step = one call of ``lattice_step_n(h, block)`` (``block`` lattice
time steps, each a full pass of the hot path: population hop, magnetisation
hop and rotation, FID / population sums) over the workload's lattice.  The
default workload is the 512^3 porous monolith (40 % solid, FP32 state and
FP32 hop weights); its state and weights (7.8 GB) are far larger than L2, so
no L2 flush is needed between steps.

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent
replica of the workload on its own GPU (no data-path collective); ``value``
is the site updates of all ranks divided by the slowest rank's time.

``--impl reference`` times the FP64 CPU oracle instead (the only other place
this script runs it), on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lpc_inputs  # noqa: E402

WORKLOADS = {
    "monolith_512": dict(make=lambda: lpc_inputs.monolith(edge=512, msd_axes=0),
                         desc="512^3 porous monolith, 40% solid (correlated noise sigma 4), "
                              "F in [-5,0] kT, shift in [-12,0] ppm, periodic, FP32 state, "
                              "FP32 hop weights", sub=64),
    "monolith_384": dict(make=lambda: lpc_inputs.monolith(edge=384, msd_axes=0),
                         desc="384^3 porous monolith (the 512^3 recipe at 0.42 of the sites, for "
                              "profiling), FP32 state and hop weights", sub=64),
    "monolith_320": dict(make=lambda: lpc_inputs.monolith(edge=320, msd_axes=0),
                         desc="320^3 porous monolith (the 512^3 recipe at a quarter of the sites, 4 GB on the "
                              "device with the link form: the small case of the full ncu captures), FP32",
                         sub=64),
    "monolith_512_bf16": dict(make=lambda: lpc_inputs.monolith(edge=512, msd_axes=0, weight_dtype=1),
                              desc="512^3 porous monolith, FP32 state, BF16 hop weights", sub=64),
    "particle_in_bath_256": dict(make=lambda: lpc_inputs.particle_in_bath(),
                                 desc="256^3 bath with a porous sphere of radius 80, FP32", sub=64),
    "supercapacitor_2048x256x256": dict(make=lambda: lpc_inputs.supercapacitor(),
                                        desc="2048x256x256 electrode/bulk/electrode slab, x walls, "
                                             "BF16 weights, MSD along x", sub=64),
    "supercapacitor_regions_2048x256x256": dict(
        make=lambda: _with_bulk_reservoirs(lpc_inputs.supercapacitor()),
        desc="2048x256x256 electrode/bulk/electrode slab, BF16 weights, MSD along x, bulk-electrolyte "
             "reservoirs (F = 0, rho = m = 1) on both x faces, FID/population/MSD per region "
             "(electrode-, bulk, electrode+)", sub=64, regions=True),
    "film_supercapacitor_regions_2048x256x256": dict(
        make=lambda: _with_bulk_reservoirs(lpc_inputs.film_supercapacitor()),
        desc="2048x256x256 film-electrode slab (monodisperse porous particles of radius 9 taking 38% of each "
             "electrode, bulk electrolyte between them), BF16 weights, MSD along x, bulk reservoirs on both x "
             "faces, FID/population/MSD per region (electrode-, bulk, electrode+)", sub=64, regions=True),
    "supercapacitor_1024x256x128": dict(
        make=lambda: lpc_inputs.supercapacitor(nx=1024, ny=256, nz=128, electrode=448, bulk=128),
        desc="1024x256x128 electrode/bulk/electrode slab (the supercapacitor recipe at a quarter of its sites, "
             "for profiling), x walls, BF16 weights, MSD along x", sub=64),
    "supercapacitor_regions_1024x256x128": dict(
        make=lambda: _with_bulk_reservoirs(lpc_inputs.supercapacitor(nx=1024, ny=256, nz=128, electrode=448,
                                                                     bulk=128)),
        desc="1024x256x128 electrode/bulk/electrode slab (the region workload at a quarter of its sites, "
             "for profiling), BF16 weights, MSD along x, bulk reservoirs, three regions", sub=64, regions=True),
    "particle_32": dict(make=lambda: lpc_inputs.particle(msd_axes=0), desc="32^3 particle, FP32",
                        sub=32),
}


def _with_bulk_reservoirs(inp):
    """Reservoir faces at x = -1 and x = nx holding bulk electrolyte
    (F = 0, rho = 1, m = 1)."""
    inp.reservoirs = ((0.0, 1.0, 1.0), (0.0, 1.0, 1.0), None, None, None, None)
    return inp


def region_kwargs(wl, inp):
    """Lattice keyword arguments for a workload with region-resolved sums."""
    if not wl.get("regions"):
        return {}
    lab, names = lpc_inputs.region_labels(inp)
    return {"region": lab, "n_regions": len(names)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="monolith_512",
                    choices=sorted(WORKLOADS) + ["serving_stream", "serving_mix_mid", "serving_mix_small"])
    ap.add_argument("--block", type=int, default=64, help="lattice steps per bench step")
    ap.add_argument("--schedule", default="auto", help="auto | step1 | tb:K")
    ap.add_argument("--static-form", default="auto", choices=["auto", "gather", "link"],
                    help="static data of the TMA-fed one-step kernel")
    ap.add_argument("--decomp", default="replicas", choices=["replicas", "slabs"],
                    help="under torchrun: an independent lattice per rank (weak scaling) or one lattice cut "
                         "into one z slab per rank with halo exchange (strong scaling)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-step-scale", type=float, default=0.25)
    ap.add_argument("--serve-slots", type=int, default=48)
    ap.add_argument("--serve-quantum", type=int, default=250)
    ap.add_argument("--serve-budget-gb", type=float, default=200.0)
    ap.add_argument("--serve-policy", default="sjf", choices=["fifo", "sjf"],
                    help="admission order of the served pass (the comparator runs in arrival order)")
    ap.add_argument("--serve-mode", default="streams", choices=["streams", "batched"],
                    help="served lattices on their own streams, or in multi-lattice / batched launches")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device):
    """The largest value of ``x`` over the ranks (the slowest rank's time):
    an all-reduce with MAX when more than one rank runs."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(ws, sites, lattice_steps, seconds):
    """Site updates of all ranks (one replica each) per second of the slowest."""
    return ws * sites * lattice_steps / seconds


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def physical_gpu(dev):
    """nvidia-smi index of torch device ``dev`` (CUDA_VISIBLE_DEVICES maps them)."""
    vis = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    if dev < len(vis) and vis[dev].strip().isdigit():
        return int(vis[dev])
    return dev


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        import tempfile
        self.idx = gpu_index
        self.proc = None
        # the raw samples go to a scratch file (LPC_BENCH_CLOCKS_DIR to keep them)
        out_dir = os.environ.get("LPC_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, "bench_clocks_%d_%d.csv" % (gpu_index, os.getpid()))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("kernels_step.cu", "kernels_tb.cu", "kernels_tma1.cu", "tma_ptx.cuh", "lpc_internal.cuh"):
        p = os.path.join(ROOT, "paper_2603_22553_b300", "csrc", name)
        if os.path.exists(p):
            h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, workload, sites):
    """DRAM bytes per launch from the committed ncu summary (profiles/), or
    None when no capture covers this workload's kernel variant or the kernel
    source changed since the counters were taken.  A capture of a smaller
    lattice of the same kernel variant is scaled by the number of sites (the
    traffic of these kernels is proportional to the sites)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[kernel][workload]
    except Exception:
        return None
    if e.get("source_hash") != kernel_source_hash():
        return None
    return float(e["dram_bytes_per_launch"]) * sites / float(e["sites"])


def oracle_sample(inp_sub, seconds, nthreads=0):
    """Time the FP64 oracle on a sub-lattice for about ``seconds``."""
    import oracle
    pk = oracle.pack_input(inp_sub, oracle.MODE_EXACT)
    rho0 = inp_sub.uniform_rho0()
    n_probe, t_probe = 10, 0.0
    while True:        # probe until the per-step cost is measured over >= 0.5 s
        t0 = time.perf_counter()
        oracle.run(pk, rho0, n_probe, msd_axes=inp_sub.msd_axes, nthreads=nthreads)
        t_probe = time.perf_counter() - t0
        if t_probe >= 0.5 or n_probe * inp_sub.n_sites > 1e11:
            break
        n_probe *= 4
    steps = max(10, int(n_probe * seconds / max(t_probe, 1e-3)))
    t0 = time.perf_counter()
    res = oracle.run(pk, rho0, steps, msd_axes=inp_sub.msd_axes, nthreads=nthreads)
    t = time.perf_counter() - t0
    return inp_sub.n_sites * steps / t, steps, t, res


def sub_lattice(inp, e):
    """The periodic [0, e)^3 corner of a workload's fields (same seeds)."""
    sub = lpc_inputs.LatticeInput(inp.name + "_sub", e, e, e, (1, 1, 1), inp.alpha, inp.dt, inp.kT,
                                  np.ascontiguousarray(inp.F[:e, :e, :e]),
                                  np.ascontiguousarray(inp.omega[:e, :e, :e]),
                                  np.ascontiguousarray(inp.solid[:e, :e, :e]), None, inp.steps,
                                  inp.weight_dtype, inp.msd_axes)
    return sub


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times single-lattice workloads; "
                          "%s is a serving workload" % args.workload}), flush=True)
        return 0
    wl = WORKLOADS[args.workload]
    inp = wl["make"]()
    sub = sub_lattice(inp, wl["sub"])
    del inp
    per_step = max(1.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(sub, per_step / 4)
    rates = []
    t_all = 0.0
    steps_all = 0
    for _ in range(args.steps):
        r, s, t, _ = oracle_sample(sub, per_step)
        rates.append(r)
        t_all += t
        steps_all += s
    value = sub.n_sites * steps_all / t_all
    sample = "%d^3 periodic corner of the %s fields, FP64, %d lattice steps over %d bench steps" % (
        wl["sub"], args.workload, steps_all, args.steps)
    line = {"impl": "reference", "metric": "site-updates/s", "value": value, "unit": "site-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_all / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": wl["desc"], "sample": sample},
            "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": oracle.max_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


STATIC_FORMS = {1: "gather", 2: "link"}


def parse_schedule(s):
    from paper_2603_22553_b300 import binding as B
    if s == "auto":
        return None
    if s == "step1":
        return (B.LPC_KERNEL_STEP1, 1)
    if s.startswith("tb:"):
        return (B.LPC_KERNEL_TB, int(s[3:]))
    raise SystemExit("bad --schedule " + s)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2603_22553_b300 import binding as B
    from paper_2603_22553_b300.lattice import Lattice

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    B.load()

    wl = WORKLOADS[args.workload]
    inp = wl["make"]()
    N = inp.n_sites
    sched = parse_schedule(args.schedule)
    ghost = (sched[1] + 1) // 2 * 2 if sched and sched[0] == B.LPC_KERNEL_TB else 0

    rkw = region_kwargs(wl, inp)
    form = {"auto": B.LPC_STATIC_AUTO, "gather": B.LPC_STATIC_GATHER, "link": B.LPC_STATIC_LINK}[args.static_form]
    lat = Lattice.from_input(inp, ghost=ghost, **rkw)
    if sched:
        lat.set_schedule(*sched)
    if form != B.LPC_STATIC_AUTO:
        lat.set_static_form(form)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        lat.step(args.block)
    torch.cuda.synchronize()
    info = lat.info()          # after the first launches: the static form is made by then
    if ws > 1:
        dist.barrier()
    clocks = ClockSampler(physical_gpu(dev))
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        lat.step(args.block)
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    ms = max_over_ranks(ms, ws, "cuda")
    lattice_steps = args.steps * args.block
    value = aggregate_rate(ws, N, lattice_steps, ms / 1e3)
    if info["kernel"] == B.LPC_KERNEL_TB:
        kernel_name = "k_step_tma1" if info["block_steps"] == 1 else "k_step_tb"
    else:
        kernel_name = "k_step1"
    launches = args.steps * (args.block // max(1, info["block_steps"]))
    bpu = info["bytes_per_site_update"]
    per_launch_ms = ms / launches
    achieved = bpu * N * info["block_steps"] / (per_launch_ms / 1e3) / 1e9
    peak, peak_kind = peaks()
    traffic = measured_traffic(kernel_name, args.workload, N)
    lat.close()
    del lat
    torch.cuda.empty_cache()

    cpu = None
    parity = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        import oracle
        sub = sub_lattice(inp, wl["sub"])
        r, s, t, res = oracle_sample(sub, args.cpu_seconds)
        cpu = {"value": r, "unit": "site-updates/s", "cores": oracle.max_threads(), "kind": "oracle",
               "sample": "%d^3 periodic corner of the workload fields, %d steps, FP64 (%.1f s)" % (
                   wl["sub"], s, t)}
        # parity of the same sample on the GPU (FID relative L2 vs the exact
        # oracle), in the kernel and static-data form the timed lattice used
        g = Lattice.from_input(sub, ghost=ghost)
        g.set_schedule(info["kernel"], info["block_steps"])
        if kernel_name == "k_step_tma1":
            g.set_static_form(info["static_form"])
        g.step(s)
        gi = g.info()
        M = g.fid()
        rho = g.density().astype(np.float64)
        g.close()
        same = (gi["kernel"], gi["block_steps"], gi["static_form"]) == (
            info["kernel"], info["block_steps"], info["static_form"])
        parity = {"fid_rel_l2": float(np.linalg.norm(M - res.M) / np.linalg.norm(res.M)),
                  "density_rel_l2": float(np.linalg.norm(rho - res.rho) / np.linalg.norm(res.rho)),
                  "kernel": kernel_name, "block_steps": gi["block_steps"],
                  "static_form": STATIC_FORMS.get(gi["static_form"], "none"),
                  "same_kernel_and_form_as_timed": bool(same),
                  "sample": "%d^3 corner, %d steps, GPU in the timed kernel and static form vs FP64 oracle%s" % (
                      wl["sub"], s, " (the corner carries no regions or reservoir faces)" if wl.get("regions")
                      else "")}

    e2e = None
    if not args.no_e2e:
        # the whole job through the public API from pinned host buffers:
        # create (H2D of F, omega, mask + pack), K bench steps, FID + density read-back
        Fp = torch.from_numpy(np.ascontiguousarray(inp.F)).pin_memory()
        Op = torch.from_numpy(np.ascontiguousarray(inp.omega)).pin_memory()
        Sp = torch.from_numpy(np.ascontiguousarray(inp.solid)).pin_memory()
        # the result buffer is pinned host memory too, allocated (like the
        # inputs) before the timed region
        Rp = torch.empty(N, dtype=torch.float32, pin_memory=True)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        lat = Lattice(inp.nx, inp.ny, inp.nz, Fp.numpy(), Op.numpy(), Sp.numpy(),
                      periodic=inp.periodic, alpha=inp.alpha, dt=inp.dt, kT=inp.kT,
                      weight_dtype=inp.weight_dtype, msd_axes=inp.msd_axes, ghost=ghost,
                      reservoirs=inp.reservoirs, **rkw)
        if sched:
            lat.set_schedule(*sched)
        if form != B.LPC_STATIC_AUTO:
            lat.set_static_form(form)
        for _ in range(args.steps):
            lat.step(args.block)
        M = lat.fid()
        rho = lat.density(out=Rp.numpy())
        t1 = time.perf_counter()
        lat.close()
        te = max_over_ranks(t1 - t0, ws, "cuda")
        h2d = Fp.numel() * 8 + Op.numel() * 8 + Sp.numel() + (inp.n_sites if rkw else 0)
        d2h = M.size * 16 + rho.size * 4
        e2e = {"value": aggregate_rate(ws, N, lattice_steps, te), "unit": "site-updates/s",
               "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": int(d2h / args.steps),
               "seconds": te}

    if rank == 0:
        line = {
            "metric": "site-updates/s", "value": value, "unit": "site-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if inp.weight_dtype == 0 else "f32/bf16-weights", "data": "synthetic",
            "config": {"workload": args.workload, "description": wl["desc"],
                       "sites": N, "lattice_steps_per_step": args.block, "kernel": kernel_name,
                       "block_steps": info["block_steps"], "ghost": info["ghost"],
                       "static_form": STATIC_FORMS.get(info["static_form"], "none"),
                       "l2": "inputs larger than L2 (%.1f GB on device)" % (info["device_bytes"] / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "bytes_per_site_update": bpu},
            "cpu_baseline": cpu,
            "parity": parity,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_slabs(args):
    """One lattice cut along z into one slab per rank (strong scaling): every
    lattice step is a step of each slab and the halo exchange (NCCL
    point-to-point between ranks; a single rank is its own neighbour through
    device copies).  ``value`` = the lattice's site updates per second of the
    slowest rank; the FID is the slabs' histories added in rank order."""
    import torch
    import torch.distributed as dist

    from paper_2603_22553_b300 import binding as B
    from paper_2603_22553_b300 import slabs as S

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    B.load()
    wl = WORKLOADS[args.workload]
    if wl.get("regions"):
        raise SystemExit("slabs take no region labels")
    inp = wl["make"]()
    N = inp.n_sites
    plan = S.SlabPlan(inp.nz, ws, inp.periodic[2])
    slab = S.Slab(inp, plan, rank)
    kern = torch.tensor([slab.lattice.info()["kernel"]], dtype=torch.int32, device="cuda")
    if ws > 1:
        dist.all_reduce(kern, op=dist.ReduceOp.MIN)        # every slab on one kernel
    slab.lattice.set_schedule(*S.common_schedule([int(kern.item())]))
    transport = S.DistTransport() if ws > 1 else S.LocalTransport()
    mine = {rank: slab} if ws > 1 else [slab]

    def lattice_steps(n):
        for _ in range(n):
            slab.step()
            transport.exchange(plan, mine)

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        lattice_steps(args.block)
    torch.cuda.synchronize()
    info = slab.lattice.info()
    if ws > 1:
        dist.barrier()
    clocks = ClockSampler(physical_gpu(dev))
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ev0.record(stream)
    for _ in range(args.steps):
        lattice_steps(args.block)
    ev1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    ms = max_over_ranks(ms, ws, "cuda")
    lattice_steps_total = args.steps * args.block
    value = N * lattice_steps_total / (ms / 1e3)
    kernel_name = "k_step_tma1" if info["kernel"] == B.LPC_KERNEL_TB else "k_step1"
    n_local = info["n_sites"]
    launches = lattice_steps_total
    bpu = info["bytes_per_site_update"]
    achieved = bpu * n_local / (ms / launches / 1e3) / 1e9
    peak, peak_kind = peaks()
    hist = slab.history()
    M, P, _ = S.gather_histories(hist) if ws > 1 else S.reduce_histories([hist])
    slab.close()
    if rank == 0:
        line = {
            "metric": "site-updates/s", "value": value, "unit": "site-updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32" if inp.weight_dtype == 0 else "f32/bf16-weights", "data": "synthetic",
            "config": {"workload": args.workload, "description": wl["desc"], "sites": N,
                       "lattice_steps_per_step": args.block, "kernel": kernel_name,
                       "static_form": STATIC_FORMS.get(info["static_form"], "none"),
                       "parallelism": "z slabs x%d (halo exchange %s)" % (ws, "NCCL" if ws > 1 else "self copy"),
                       "slab_planes": [z1 - z0 for z0, z1 in plan.bounds],
                       "l2": "inputs larger than L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                         "bytes_per_site_update": bpu, "note": "one slab (the slowest rank), exchange included"},
            "population_drift": float(np.max(np.abs(P / P[0] - 1.0))),
            "fid_modulus_bounded": bool(np.all(np.abs(M) <= P[0] * (1 + 1e-6))),
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


MIXES = {"serving_mix_mid": [104, 112, 120, 128, 136, 144, 152, 160, 168, 176, 184, 192],
         "serving_mix_small": list(range(24, 101, 4))}


def run_mix(args):
    """Resident particle lattices of the serving recipe (edges of the mix,
    FP32), advanced ``--block`` steps per bench step either on their own
    streams (``--serve-mode streams``: graphs of one-step launches, queued
    before any wait) or together (``batched``: lattice_step_many, the
    multi-lattice TMA launch for the mid-size ones, the batched
    register-pipelined kernel for the small ones)."""
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch

    from paper_2603_22553_b300 import binding as B
    from paper_2603_22553_b300.lattice import Lattice, step_many

    torch.cuda.set_device(0)
    B.load()
    edges = MIXES[args.workload]
    lats = []
    for i, e in enumerate(edges):
        inp = lpc_inputs.Request(7000 + i, 0.0, e, args.block, 7000 + i).lattice()
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            lat = Lattice.from_input(inp, stream=s.cuda_stream)
        lat._stream = s
        lats.append(lat)
    sites = sum(e ** 3 for e in edges)

    def one():
        if args.serve_mode == "batched":
            step_many(lats, [args.block] * len(lats))
        else:
            for lat in lats:
                lat.step(args.block)

    for _ in range(args.warmup):
        one()
    torch.cuda.synchronize()
    clocks = ClockSampler(physical_gpu(torch.cuda.current_device()))
    clocks.start()
    time.sleep(0.3)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    clk = clocks.stop()
    for lat in lats:
        lat.close()
    line = {"metric": "site-updates/s", "value": sites * args.block * args.steps / t, "unit": "site-updates/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "edges": edges, "sites": sites,
                       "lattice_steps_per_step": args.block, "mode": args.serve_mode,
                       "timing": "host clock around the device work, synchronised on both sides"},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """Served stream: continuous batching vs one-at-a-time plain solves.

    The request stream is the 1000-request recipe (edges log-uniform in
    [24, 192], steps uniform in [1000, 20000], Poisson arrivals at 50/s),
    truncated to ``--serve-requests`` requests with step counts scaled by
    ``--serve-step-scale`` so that both passes fit in a few minutes.  Fields
    are generated before the timed passes.
    """
    # more hardware work queues than the default 8, so that the streams of
    # the resident lattices do not alias (read when CUDA initialises)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    import torch

    from paper_2603_22553_b300 import binding as B
    from paper_2603_22553_b300.serve import GpuEngine, Server, serve_sequential, summary

    torch.cuda.set_device(0)
    B.load()
    reqs = lpc_inputs.request_stream()[:args.serve_requests]
    for r in reqs:
        r.steps = max(10, int(round(r.steps * args.serve_step_scale)))
    cache = {r.rid: r.lattice() for r in reqs}

    class CachedEngine(GpuEngine):
        def lattice_input(self, req):
            return cache[req.rid]

    eng = CachedEngine(keep_fid=True, mode=args.serve_mode)
    budget = int(args.serve_budget_gb * (1 << 30))
    warm = [lpc_inputs.Request(10 ** 6 + i, 0.0, 24, 20, 7) for i in range(2)]
    for w in warm:
        cache[w.rid] = w.lattice()
    Server(eng, budget, max_active=args.serve_slots, quantum=args.serve_quantum, policy=args.serve_policy).run(warm)
    torch.cuda.synchronize()
    clocks = ClockSampler(physical_gpu(torch.cuda.current_device()))
    clocks.start()
    recs = Server(eng, budget, max_active=args.serve_slots, quantum=args.serve_quantum,
                  policy=args.serve_policy).run(reqs)
    torch.cuda.synchronize()
    clk_served = clocks.stop()
    s_batch = summary(recs)
    clocks = ClockSampler(physical_gpu(torch.cuda.current_device()))
    clocks.start()
    seq = serve_sequential(eng, reqs)
    clk_seq = clocks.stop()
    s_seq = summary(seq)
    same = all(np.allclose(a.fid, b.fid, rtol=1e-5, atol=1e-5 * abs(b.fid[0])) for a, b in zip(recs, seq))
    line = {"metric": "site-updates/s (served aggregate)", "value": s_batch["aggregate_site_updates_per_s"],
            "unit": "site-updates/s", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "dtype": "f32",
            "config": {"workload": "serving_stream", "requests": len(reqs),
                       "step_scale": args.serve_step_scale, "slots": args.serve_slots,
                       "quantum": args.serve_quantum, "hbm_budget_gb": args.serve_budget_gb,
                       "policy": args.serve_policy, "mode": args.serve_mode,
                       "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS")},
            "served": s_batch, "one_at_a_time": s_seq,
            "speedup_vs_one_at_a_time": s_batch["aggregate_site_updates_per_s"] / s_seq["aggregate_site_updates_per_s"],
            "fid_same_as_one_at_a_time_1e-5": bool(same),
            "clocks": {"served": clk_served, "one_at_a_time": clk_seq}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving_stream":
        return run_serving(args)
    if args.workload in MIXES:
        return run_mix(args)
    if args.decomp == "slabs":
        return run_slabs(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
