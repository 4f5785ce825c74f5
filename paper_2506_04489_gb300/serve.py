"""Continuous-batching solve server.

Requests (a density on an n^3 grid of a fixed box, and an accuracy target) arrive at
any time; a scheduler thread admits them onto the GPU as stream slots and device memory
free up, so that work of different requests overlaps on the device:

* accuracy routing: a target of 1e-6 or looser runs on FP32 plans (parity bar 1e-5),
  tighter targets on double-float plans (FP64 in/out, parity bar 1e-12);
* per-(grid, precision) plans stay resident on the device with their multiplier and
  workspace (the one-time precompute of Alg. 1 is paid once per plan);
* same-key requests waiting together are solved as one batch (sp_solve_batched);
* a device-memory budget bounds everything the server allocates (plans, batch buffers);
  a new plan is admitted only within the budget, evicting idle plans of other keys first,
  otherwise the request waits for a plan of its key to free up;
* each batch runs on one of several CUDA streams (slots): host-to-device copy of the
  inputs, the solve, device-to-host copy of the results, then an event the scheduler
  polls.  Latency is completion (event observed) minus arrival, host monotonic clock.

A request whose input is invalid fails alone: its future gets the exception, the rest
of its batch and all other requests proceed.
"""
from __future__ import annotations

import collections
import math
import threading
import time
from concurrent.futures import Future

import numpy as np

from .plan import Plan


def precision_for(accuracy: float) -> str:
    """Accuracy target -> plan precision."""
    return "fp32" if accuracy >= 1e-6 else "df32"


def entry_bytes(n: int, precision: str, max_batch: int) -> int:
    """Device bytes of one resident plan of an n^3 grid with batch buffers for max_batch
    requests: workspace, multiplier octant and its pass-precision copy, twiddles, and the
    input and output batch buffers (plus 1 MiB for small tables)."""
    c = 16 if precision in ("fp64", "df32") else 8
    r = 4 if precision == "fp32" else 8
    ldz = (n + 1 + 7) // 8 * 8
    work = max_batch * c * n * 2 * n * ldz
    tables = (n + 1) * (n + 1) * ldz * (8 + (8 if precision == "df32" else 4)) + 3 * 2 * n * 32
    io = 2 * max_batch * n ** 3 * r
    return work + tables + io + (1 << 20)


Done = collections.namedtuple("Done", "arrival done_at key launched_at", defaults=(None,))


class Request:
    __slots__ = ("rho", "out", "accuracy", "n", "precision", "arrival", "future", "done_at", "launched_at")

    def __init__(self, rho, accuracy, arrival, out=None):
        self.rho = rho
        self.out = out
        self.accuracy = accuracy
        self.n = int(rho.shape[0])
        self.precision = precision_for(accuracy)
        self.arrival = arrival
        self.future = Future()
        self.done_at = None
        self.launched_at = None


class _Entry:
    """One resident plan with its batch buffers; used by one slot at a time."""

    def __init__(self, key, plan, in_buf, out_buf, nbytes):
        self.key = key
        self.plan = plan
        self.in_buf = in_buf
        self.out_buf = out_buf
        self.nbytes = nbytes
        self.busy = False
        self.last_used = time.monotonic()


def batch_cap(n: int, max_batch: int, max_points: int) -> int:
    """Requests of an n^3 grid per launch: at most max_batch, at most max_points grid
    points, and always at least one."""
    return max(1, min(int(max_batch), int(max_points) // n ** 3))


def pick_slot(free, priority_slots: int, small: bool) -> int:
    """Free slot for a batch: slots [0, priority_slots) are high-priority streams, taken
    first by small batches and last by large ones."""
    hi = [i for i in free if i < priority_slots]
    lo = [i for i in free if i >= priority_slots]
    order = hi + lo if small else lo + hi
    return order[0]


class Server:
    """Continuous-batching server for solves on the box [lo, hi]^3.

    budget_bytes  : device memory the server may hold (plans + batch buffers).
    max_batch     : largest batch per launch.
    max_batch_points : largest number of grid points per launch (batch x n^3); a batch of
                    large grids is cut at this size so a request queued behind it waits for
                    a bounded amount of work, not for max_batch full-size solves.
    slots         : concurrent batches (CUDA streams).
    priority_slots: how many of the slots run on high-priority streams.  Batches of at
                    most small_points grid points go to those first, so the block
                    scheduler runs their kernels' blocks ahead of a large solve's
                    waiting blocks instead of queueing them behind whole passes.
    plans_per_key : resident plans per (n, precision); further requests of a busy key wait
                    and are batched together when a plan frees up.
    """

    def __init__(self, lo: float = -1.0, hi: float = 1.0, budget_bytes: float = 120e9, max_batch: int = 8,
                 slots: int = 4, device: int = 0, plans_per_key: int = 2, priority_slots: int = 2,
                 small_points: int = 2 * 128 ** 3,
                 max_batch_points: int = 256 ** 3):
        import torch
        self.torch = torch
        self.plans_per_key = int(plans_per_key)
        self.lo, self.hi = float(lo), float(hi)
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)
        self.max_batch_points = int(max_batch_points)
        self.device = torch.device("cuda", device)
        hi_prio = torch.cuda.Stream.priority_range()[1] if hasattr(torch.cuda.Stream, "priority_range") else -1
        self.priority_slots = max(0, min(int(priority_slots), slots - 1))
        self.small_points = int(small_points)
        self.streams = [torch.cuda.Stream(device=self.device, priority=hi_prio if i < self.priority_slots else 0)
                        for i in range(slots)]
        self.slot_busy = [None] * slots  # (event, entry, [(request, host_out)])
        self.pending = collections.OrderedDict()  # key -> deque of requests
        self.entries = {}  # key -> [_Entry]
        self.used_bytes = 0
        self.peak_bytes = 0
        self.completed = []
        self.batches = 0
        self._lock = threading.Lock()
        self._wake = threading.Event()
        self._stop = False
        self._thread = None

    # ------------------------------------------------------------------ client side
    def start(self):
        self._thread = threading.Thread(target=self._loop, name="superpot-scheduler", daemon=True)
        self._thread.start()
        return self

    def submit(self, rho, accuracy: float, arrival: float = None, out=None) -> Future:
        """Queue one solve.  rho: a CPU torch tensor (pinned for asynchronous copies) of
        shape (n, n, n), float32 for accuracy >= 1e-6 else float64.  The future yields
        the potential as a CPU tensor of the same shape and type: `out` if given (a
        pinned CPU tensor like rho, which the caller must not touch until the future is
        done), else a new pinned tensor."""
        req = Request(rho, accuracy, time.monotonic() if arrival is None else arrival, out)
        with self._lock:
            self.pending.setdefault((req.n, req.precision), collections.deque()).append(req)
        self._wake.set()
        return req.future

    def stop(self):
        self._stop = True
        self._wake.set()
        if self._thread is not None:
            self._thread.join()
        self.torch.cuda.synchronize(self.device)
        for lst in self.entries.values():
            for e in lst:
                e.plan.close()
        self.entries.clear()
        self.used_bytes = 0

    # ------------------------------------------------------------------ memory
    def _entry_bytes(self, n, precision):
        return entry_bytes(n, precision, self.max_batch)

    def _evict_idle(self, need, keep_key):
        """Free idle plans of other keys, least recently used first, until `need` fits."""
        idle = [e for k, lst in self.entries.items() if k != keep_key for e in lst if not e.busy]
        idle.sort(key=lambda e: e.last_used)
        for e in idle:
            if self.used_bytes + need <= self.budget:
                break
            self.entries[e.key].remove(e)
            e.plan.close()
            self.used_bytes -= e.nbytes
        return self.used_bytes + need <= self.budget

    def prepare(self, keys):
        """Build the resident plans of each (n, precision) key now, before traffic:
        plans_per_key of them while the budget allows (the rest are built on demand), so
        that no allocation or precompute stalls the device once requests flow."""
        for _ in range(self.plans_per_key):
            for key in keys:
                key = (int(key[0]), key[1])
                lst = self.entries.get(key, [])
                if len(lst) < self.plans_per_key and self.used_bytes + self._entry_bytes(*key) <= self.budget:
                    for e in lst:
                        e.busy = True  # force a new plan rather than reuse
                    self._get_entry(key)
                    for e in lst:
                        e.busy = False

    def _get_entry(self, key):
        lst = self.entries.setdefault(key, [])
        for e in lst:
            if not e.busy:
                return e
        if len(lst) >= self.plans_per_key:
            return None  # wait for a plan of this key: its requests batch up meanwhile
        need = self._entry_bytes(*key)
        if self.used_bytes + need > self.budget and not self._evict_idle(need, key):
            return None  # wait for a plan of this key (or memory) to free up
        n, precision = key
        torch = self.torch
        plan = Plan(n, self.lo, self.hi, precision=precision, max_batch=self.max_batch)
        in_buf = torch.empty((self.max_batch, n, n, n), dtype=plan.dtype, device=self.device)
        out_buf = torch.empty_like(in_buf)
        # the precompute ran on this thread's current stream; the slot streams are not
        # ordered after it, so the plan is published only once it has finished
        torch.cuda.synchronize(self.device)
        e = _Entry(key, plan, in_buf, out_buf, need)
        lst.append(e)
        self.used_bytes += need
        self.peak_bytes = max(self.peak_bytes, self.used_bytes)
        return e

    # ------------------------------------------------------------------ scheduler
    def _poll(self):
        now_done = False
        for i, slot in enumerate(self.slot_busy):
            if slot is None:
                continue
            ev, entry, items = slot
            if ev.query():
                t = time.monotonic()
                for req, host_out in items:
                    req.done_at = t
                    # only (arrival, completion, key) is kept: results belong to the client,
                    # so their pinned buffers return to the allocator's cache once dropped
                    self.completed.append(Done(req.arrival, t, (req.n, req.precision), req.launched_at))
                    req.future.set_result(host_out)
                entry.busy = False
                entry.last_used = t
                self.slot_busy[i] = None
                now_done = True
        return now_done

    def _launch(self, slot, entry, reqs):
        torch = self.torch
        st = self.streams[slot]
        items = []
        dtype = entry.plan.dtype
        good = []
        for r in reqs:
            if tuple(r.rho.shape) != (entry.key[0],) * 3 or r.rho.dtype != dtype or r.rho.is_cuda:
                r.future.set_exception(ValueError(
                    f"request needs a CPU {dtype} tensor of shape {(entry.key[0],) * 3}"))
                continue
            if r.out is not None and (tuple(r.out.shape) != tuple(r.rho.shape) or r.out.dtype != dtype
                                      or r.out.is_cuda or not r.out.is_contiguous()):
                r.future.set_exception(ValueError(f"out must be a contiguous CPU {dtype} tensor like rho"))
                continue
            good.append(r)
        if not good:
            entry.busy = False
            return
        b = len(good)
        t_launch = time.monotonic()
        for r in good:
            r.launched_at = t_launch
        with torch.cuda.stream(st):
            for i, r in enumerate(good):
                entry.in_buf[i].copy_(r.rho, non_blocking=True)
            entry.plan.solve_batched(entry.in_buf[:b], entry.out_buf[:b], st)
            for i, r in enumerate(good):
                host = r.out if r.out is not None else torch.empty(r.rho.shape, dtype=dtype, pin_memory=True)
                host.copy_(entry.out_buf[i], non_blocking=True)
                items.append((r, host))
            ev = torch.cuda.Event()
            ev.record(st)
        self.slot_busy[slot] = (ev, entry, items)
        self.batches += 1

    def _schedule(self):
        launched = False
        while True:
            free = [i for i, s in enumerate(self.slot_busy) if s is None]
            if not free:
                return launched
            with self._lock:
                keys = [k for k, q in self.pending.items() if q]
                keys.sort(key=lambda k: self.pending[k][0].arrival)  # oldest waiting request first
            started = False
            for key in keys:
                if self._entry_bytes(*key) > self.budget:  # can never be admitted
                    with self._lock:
                        q = self.pending[key]
                        while q:
                            q.popleft().future.set_exception(MemoryError(
                                f"a {key[0]}^3 {key[1]} plan needs more than the {self.budget} B budget"))
                    continue
                entry = self._get_entry(key)
                if entry is None:
                    continue
                with self._lock:
                    q = self.pending[key]
                    cap = batch_cap(key[0], self.max_batch, self.max_batch_points)
                    reqs = [q.popleft() for _ in range(min(cap, len(q)))]
                entry.busy = True
                self._launch(pick_slot(free, self.priority_slots, len(reqs) * key[0] ** 3 <= self.small_points),
                             entry, reqs)
                launched = started = True
                break
            if not started:
                return launched

    def _loop(self):
        torch = self.torch
        torch.cuda.set_device(self.device)
        while not self._stop:
            progressed = self._poll()
            progressed = self._schedule() or progressed
            if not progressed:
                busy = any(s is not None for s in self.slot_busy)
                if busy:
                    time.sleep(2e-5)
                else:
                    self._wake.wait(timeout=1e-3)
                    self._wake.clear()
        # drain
        while any(s is not None for s in self.slot_busy):
            self._poll()
            time.sleep(1e-4)


def poisson_stream(server: Server, rate: float, duration: float, sizes, accuracies, seed: int = 0,
                   densities=None, warmup: float = 0.0, outputs=None):
    """Drive `server` with Poisson arrivals (mean `rate` per second) for `warmup + duration`
    seconds; each request draws its grid size and accuracy uniformly from the lists.
    `densities[(n, precision)]` supplies the (pinned CPU) input of a key.  With `outputs`
    (key -> list of pinned CPU tensors like the density), results land in buffers taken
    from that pool and returned to it on completion, as a client that owns its result
    memory would do; the pool grows when every buffer of a key is in flight.  Returns
    the requests that arrived after the warm-up, completed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t0 = time.monotonic()
    t = 0.0
    keys = []
    outstanding = [0]
    cv = threading.Condition()

    def finished(fut, key=None):
        res = fut.result()  # raise here if the solve failed; the result itself is dropped
        with cv:
            if outputs is not None:
                outputs[key].append(res)
            outstanding[0] -= 1
            cv.notify_all()

    while t < warmup + duration:
        n = int(sizes[rng.integers(len(sizes))])
        acc = float(accuracies[rng.integers(len(accuracies))])
        key = (n, precision_for(acc))
        due = t0 + t
        now = time.monotonic()
        if due > now:
            time.sleep(due - now)
        out = None
        with cv:
            outstanding[0] += 1
            if outputs is not None:
                pool = outputs.setdefault(key, [])
                out = pool.pop() if pool else densities[key].new_empty(densities[key].shape).pin_memory()
        server.submit(densities[key], acc, arrival=due, out=out).add_done_callback(
            lambda f, k=key: finished(f, k))
        keys.append((t, key))
        t += float(rng.exponential(1.0 / rate))
    with cv:
        cv.wait_for(lambda: outstanding[0] == 0)
    return [(t, key) for t, key in keys if t >= warmup]


def percentile(sorted_values, p: float):
    """Nearest-rank percentile of an ascending list."""
    return sorted_values[min(len(sorted_values) - 1, max(0, int(math.ceil(p / 100.0 * len(sorted_values))) - 1))]


def summarize(completed, t_start: float, t_end: float):
    """p50/p99/mean latency (ms) and throughput of the completed requests that arrived in
    [t_start, t_end); throughput counts them over [t_start, last completion]."""
    sel = [r for r in completed if t_start <= r.arrival < t_end]
    if not sel:
        return None
    lat = sorted((r.done_at - r.arrival) * 1e3 for r in sel)
    span = max(r.done_at for r in sel) - t_start
    by_key = collections.defaultdict(list)
    for r in sel:
        key = getattr(r, "key", None)
        if key is not None:
            by_key[f"n{key[0]}_{key[1]}"].append((r.done_at - r.arrival) * 1e3)
    per_key = {k: {"requests": len(v), "p50_ms": percentile(sorted(v), 50), "p99_ms": percentile(sorted(v), 99)}
               for k, v in sorted(by_key.items())}
    out = {"requests": len(lat), "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
           "mean_ms": sum(lat) / len(lat), "solves_per_s": len(lat) / span, "by_key": per_key}
    # split of the latency: waiting for a slot or plan (arrival -> launch) and on the
    # device (launch -> completion observed)
    launched = [r for r in sel if getattr(r, "launched_at", None) is not None]
    if launched:
        wait = sorted((r.launched_at - r.arrival) * 1e3 for r in launched)
        run = sorted((r.done_at - r.launched_at) * 1e3 for r in launched)
        out.update({"wait_p50_ms": percentile(wait, 50), "wait_p99_ms": percentile(wait, 99),
                    "run_p50_ms": percentile(run, 50), "run_p99_ms": percentile(run, 99)})
    return out


def latency_summary(server: Server, t_start: float, t_end: float):
    out = summarize(server.completed, t_start, t_end)
    if out is not None:
        out.update({"batches": server.batches, "peak_bytes": server.peak_bytes})
    return out
