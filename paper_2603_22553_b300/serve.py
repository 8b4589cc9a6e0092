"""Serving loop: lattice solves of different sizes and lengths as they arrive.

Continuous batching on one GPU:
* requests enter a FIFO queue at their arrival times;
* a request is admitted when its device footprint (``lattice_footprint``:
  state, weights, history and create-time transients) fits the HBM budget
  beside the resident lattices and an active slot is free; a preparation
  thread builds its fields and creates the lattice (its state then stays
  resident on the device until it finishes);
* every round advances all resident lattices together by up to ``quantum``
  steps.  ``mode="streams"`` (the default): every lattice queues its steps
  on its own stream (captured graphs of 32 launches of its one-step
  kernel), so the launches of all resident lattices overlap on the device;
  ``mode="batched"``: one ``lattice_step_many`` call, where the lattices of
  the TMA-fed one-step kernel share one multi-lattice launch per step and
  the small ones one persistent launch of the batched register-pipelined
  kernel.  On the B300 the streams win (8.8e10 against 7.1e10 site-updates/s
  for twelve lattices of 104^3 to 192^3, 3.9e10 against 2.1e10 for twenty of
  24^3 to 100^3): a mid-size lattice's state and static data nearly fit the
  126 MB L2, so consecutive steps of one lattice reuse it, while a launch
  over all resident lattices streams gigabytes per step;
* admission order: ``policy="fifo"`` (arrival order, no overtaking) or
  ``"sjf"`` (the pending request with the least work, sites x steps, first:
  short requests are not held behind long ones; ``max_wait_s`` lets a
  request that has waited that long go first, so none starves);
* a lattice that has done its steps has its FID read back and is destroyed,
  which frees its slot and memory for the next admission.

Latency = finish - arrival; aggregate throughput = sum(sites * steps) / makespan.
``serve_sequential`` is the comparator: the same stream solved one at a time
with plain ``lattice_step_n``.
"""
from __future__ import annotations

import collections
import ctypes
import dataclasses
import queue
import threading
import time

import numpy as np

from . import binding as B


@dataclasses.dataclass
class Record:
    rid: int
    edge: int
    steps: int
    sites: int
    arrival: float
    admit: float = float("nan")
    finish: float = float("nan")
    fid: np.ndarray | None = None

    @property
    def latency(self):
        return self.finish - self.arrival


def footprint(edge, steps, weight_dtype=0, msd_axes=0):
    """Device bytes a cubic lattice of this edge would hold (C ABI query)."""
    lib = B.load()
    p = B.lpc_params(edge, edge, edge, (ctypes.c_int32 * 3)(1, 1, 1), 0.005, 5e-6, 1.0,
                     int(weight_dtype), int(msd_axes), 0, 0)
    out = ctypes.c_int64()
    B.check(lib.lattice_footprint(ctypes.byref(p), int(steps), ctypes.byref(out)), lib)
    return out.value


class GpuEngine:
    """Creates, advances and reads lattices through the C ABI.

    Every live lattice has a caller stream of its own, taken from a pool at
    create and returned at finish.  The library orders a lattice's work after
    its caller stream and the caller stream after that work, so lattices
    that shared one caller stream would run one after another; with their
    own streams, the launches of different lattices (and the creation of new
    ones) overlap on the device.  Reusing pooled streams lets PyTorch's
    caching allocator hand a finished lattice's memory to the next one.
    """

    def __init__(self, keep_fid=True, mode="streams"):
        import torch
        from . import lattice as L
        if mode not in ("streams", "batched"):
            raise ValueError("mode must be 'streams' or 'batched'")
        self.L = L
        self.torch = torch
        self.keep_fid = keep_fid
        self.mode = mode
        self.device = torch.cuda.current_device()    # preparation threads start on device 0
        self._streams = []
        self._lock = threading.Lock()

    def footprint(self, req):
        return footprint(req.edge, req.steps)

    def lattice_input(self, req):
        """The request's fields (``lpc_inputs.LatticeInput``)."""
        return req.lattice()

    def create(self, req):
        inp = self.lattice_input(req)
        with self._lock:
            s = self._streams.pop() if self._streams else self.torch.cuda.Stream(device=self.device)
        try:
            with self.torch.cuda.stream(s):
                lat = self.L.Lattice.from_input(inp, stream=s.cuda_stream)
        except Exception:
            with self._lock:
                self._streams.append(s)
            raise
        lat._serve_stream = s
        return lat

    def step_many(self, lats, steps):
        """Advance every resident lattice: on its own stream (``streams``),
        all queued before any wait, or in one lattice_step_many call
        (``batched``: multi-lattice and batched launches)."""
        if not lats:
            return
        if self.mode == "batched":
            self.L.step_many(list(lats), list(steps))
            return
        for lat, n in zip(lats, steps):
            lat.step(n)

    def finish(self, lat):
        fid = lat.fid() if self.keep_fid else None
        self.discard(lat)
        return fid

    def discard(self, lat):
        """Destroy a lattice without reading it and return its stream to the pool."""
        lat.close()
        s = getattr(lat, "_serve_stream", None)
        if s is not None:
            lat._serve_stream = None
            with self._lock:
                self._streams.append(s)


class Server:
    """Continuous-batching server over an engine (GPU or a test fake)."""

    def __init__(self, engine, hbm_budget, max_active=48, quantum=250, prefetch=4, policy="fifo",
                 max_wait_s=None):
        if policy not in ("fifo", "sjf"):
            raise ValueError("policy must be 'fifo' or 'sjf'")
        self.engine = engine
        self.budget = int(hbm_budget)
        self.max_active = int(max_active)
        self.quantum = int(quantum)
        self.prefetch = int(prefetch)
        self.policy = policy
        self.max_wait_s = max_wait_s

    def _next(self, pending, t):
        """Index of the pending request to admit next."""
        if self.policy == "fifo":
            return 0
        if self.max_wait_s is not None:
            for i, r in enumerate(pending):       # pending is in arrival order
                if t - r.arrival_s >= self.max_wait_s:
                    return i
        return min(range(len(pending)), key=lambda i: (pending[i].edge ** 3 * pending[i].steps, i))

    def run(self, requests, realtime=True):
        """Serve ``requests`` (sorted by arrival); returns the list of Records."""
        eng = self.engine
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        recs = {r.rid: Record(r.rid, r.edge, r.steps, r.edge ** 3, r.arrival_s) for r in reqs}
        fp = {r.rid: eng.footprint(r) for r in reqs}
        for r in reqs:
            if fp[r.rid] > self.budget:
                raise ValueError("request %d needs %d bytes, above the HBM budget" % (r.rid, fp[r.rid]))
        arrivals = collections.deque(reqs)
        pending = collections.deque()        # arrived, not admitted
        ready = queue.Queue()                # created lattices
        work = queue.Queue()                 # admitted requests to prepare
        active = []                          # [req, lattice, remaining]
        used = 0
        preparing = 0
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if realtime else None
        vclock = [0.0]
        now = clock if realtime else (lambda: vclock[0])
        errors = []

        def preparer():
            while True:
                req = work.get()
                if req is None:
                    return
                try:
                    ready.put((req, eng.create(req)))
                except Exception as e:   # surfaced to the caller below
                    errors.append(e)
                    ready.put((req, None))

        threads = [threading.Thread(target=preparer, daemon=True) for _ in range(max(1, self.prefetch))]
        for th in threads:
            th.start()
        done = 0
        try:
            while done < len(reqs):
                t = now()
                while arrivals and arrivals[0].arrival_s <= t:
                    pending.append(arrivals.popleft())
                # admission by footprint and free slots, in the policy's order
                # (the chosen request waits for memory; nothing overtakes it)
                while pending and len(active) + preparing < self.max_active:
                    k = self._next(pending, t)
                    if used + fp[pending[k].rid] > self.budget:
                        break
                    req = pending[k]
                    del pending[k]
                    used += fp[req.rid]
                    preparing += 1
                    recs[req.rid].admit = now()
                    work.put(req)
                # lattices whose creation finished join the batch
                block = not active and preparing > 0
                while True:
                    try:
                        req, lat = ready.get(block=block, timeout=60.0 if block else None)
                    except queue.Empty:
                        break
                    block = False
                    preparing -= 1
                    if lat is None:
                        raise errors[-1]
                    active.append([req, lat, req.steps])
                if not active:
                    if arrivals and preparing == 0:
                        if realtime:
                            time.sleep(max(0.0, min(0.002, arrivals[0].arrival_s - now())))
                        else:
                            vclock[0] = max(vclock[0], arrivals[0].arrival_s)
                    continue
                n = [min(self.quantum, a[2]) for a in active]
                eng.step_many([a[1] for a in active], n)
                if not realtime:
                    vclock[0] += sum(a[0].edge ** 3 * k for a, k in zip(active, n)) * 1e-11
                for a, k in zip(active, n):
                    a[2] -= k
                still = []
                for a in active:
                    if a[2] == 0:
                        fid = eng.finish(a[1])
                        rec = recs[a[0].rid]
                        rec.finish = now()
                        rec.fid = fid
                        used -= fp[a[0].rid]
                        done += 1
                    else:
                        still.append(a)
                active = still
        except BaseException:
            # a failed run releases what it still holds: the resident
            # lattices and those whose creation ends after the failure
            discard = getattr(eng, "discard", None)
            for _ in threads:
                work.put(None)
            for th in threads:
                th.join()
            if discard is not None:
                for a in active:
                    discard(a[1])
                while True:
                    try:
                        _, lat = ready.get_nowait()
                    except queue.Empty:
                        break
                    if lat is not None:
                        discard(lat)
            raise
        for _ in threads:
            work.put(None)
        return [recs[r.rid] for r in reqs]


def serve_sequential(engine, requests, realtime=True):
    """One request at a time in arrival order with plain lattice_step_n."""
    reqs = sorted(requests, key=lambda r: r.arrival_s)
    out = []
    t0 = time.perf_counter()
    vclock = 0.0
    for r in reqs:
        now = (time.perf_counter() - t0) if realtime else vclock
        if now < r.arrival_s:
            if realtime:
                time.sleep(r.arrival_s - now)
            else:
                vclock = r.arrival_s
        rec = Record(r.rid, r.edge, r.steps, r.edge ** 3, r.arrival_s)
        rec.admit = (time.perf_counter() - t0) if realtime else vclock
        lat = engine.create(r)
        lat.step(r.steps)
        rec.fid = engine.finish(lat)
        if realtime:
            rec.finish = time.perf_counter() - t0
        else:
            vclock += r.edge ** 3 * r.steps * 1e-11
            rec.finish = vclock
        out.append(rec)
    return out


def summary(records):
    lat = np.array([r.latency for r in records])
    work = float(sum(r.sites * r.steps for r in records))
    t_start = min(r.arrival for r in records)
    t_end = max(r.finish for r in records)
    return {"requests": len(records), "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "makespan_s": t_end - t_start,
            "site_updates": work, "aggregate_site_updates_per_s": work / (t_end - t_start)}
