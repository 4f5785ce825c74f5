"""Continuous-batching solve server: Python face of the library's native server
(sp_server_* in include/superpot.h).

Requests (a density on an n^3 grid of a fixed box, and an accuracy target) arrive at
any time; the library's scheduler thread admits them onto the GPU as stream slots and
device memory free up, so that work of different requests overlaps on the device:

* accuracy routing: a target of 1e-6 or looser runs on FP32 plans (parity bar 1e-5),
  tighter targets on double-float plans (FP64 in/out, parity bar 1e-12);
* per-(grid, precision) plans stay resident on the device with their multiplier and
  workspace (the one-time precompute of Alg. 1 is paid once per plan);
* same-key requests waiting together are solved as one batch (sp_solve_batched);
* a device-memory budget bounds everything the server allocates (plans, batch buffers);
  a new plan is admitted only within the budget, evicting idle plans of other keys first,
  otherwise the request waits for a plan of its key to free up;
* each batch runs on one of several CUDA streams (slots): host-to-device copy of the
  inputs, the solve, device-to-host copy of the results, then a host callback that stamps
  completion.  Latency is completion minus arrival on the host's monotonic clock.

A request whose input is invalid fails alone: its future gets the exception, the rest
of its batch and all other requests proceed.  This module validates requests, keeps
their host buffers alive, resolves futures, and holds the host-side helpers (routing,
the memory estimate, percentiles).
"""
from __future__ import annotations

import collections
import math
import threading
import time
from concurrent.futures import Future

import numpy as np



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


_PREC_CODE = {"fp64": 0, "fp32": 1, "mixed": 2, "df32": 3}
_PREC_NAME = {v: k for k, v in _PREC_CODE.items()}


def batch_cap(n: int, max_batch: int, max_points: int) -> int:
    """Requests of an n^3 grid per launch: at most max_batch, at most max_points grid
    points, and always at least one (the rule the native scheduler applies)."""
    return max(1, min(int(max_batch), int(max_points) // n ** 3))


def pick_slot(free, priority_slots: int, small: bool) -> int:
    """Free slot for a batch: slots [0, priority_slots) are high-priority streams, taken
    first by small batches and last by large ones (the rule the native scheduler applies)."""
    hi = [i for i in free if i < priority_slots]
    lo = [i for i in free if i >= priority_slots]
    order = hi + lo if small else lo + hi
    return order[0]


class Server:
    """Continuous-batching server for solves on the box [lo, hi]^3: the library's native
    server (sp_server_* in include/superpot.h) with Python futures.

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
    The scheduling, batching, admission and completion stamping all run in the library;
    this class validates requests, keeps their host buffers alive and resolves futures.
    """

    def __init__(self, lo: float = -1.0, hi: float = 1.0, budget_bytes: float = 120e9, max_batch: int = 8,
                 slots: int = 4, device: int = 0, plans_per_key: int = 2, priority_slots: int = 2,
                 small_points: int = 2 * 128 ** 3,
                 max_batch_points: int = 256 ** 3):
        import ctypes

        import torch

        from . import _native as N
        self.torch = torch
        self._N = N
        self.lo, self.hi = float(lo), float(hi)
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch)
        self.device = torch.device("cuda", device)
        self.cfg = N.ServerConfig(self.lo, self.hi, float(self.budget), self.max_batch, int(slots),
                                  max(0, min(int(priority_slots), int(slots) - 1)), int(plans_per_key),
                                  int(small_points), int(max_batch_points))
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            N.check(N.lib.sp_server_create(ctypes.byref(h), ctypes.byref(self.cfg)), "sp_server_create")
        self._h = h
        self._lock = threading.Lock()
        self._pending = {}  # ticket -> (future, result tensor, input tensor)
        self._thread = None
        self._closed = False

    # ------------------------------------------------------------------ client side
    def start(self):
        """Start the thread that reports finished requests to their futures."""
        if self._thread is None:
            self._thread = threading.Thread(target=self._complete, name="superpot-completions", daemon=True)
            self._thread.start()
        return self

    def prepare(self, keys):
        """Build the resident plans of each (n, precision) key now, before traffic, so that
        no allocation or precompute stalls the device once requests flow."""
        with self.torch.cuda.device(self.device):
            for n, precision in keys:
                self._N.check(self._N.lib.sp_server_prepare(self._h, int(n), _PREC_CODE[precision]),
                              "sp_server_prepare")

    def _check(self, rho, precision, out):
        torch = self.torch
        dtype = torch.float32 if precision == "fp32" else torch.float64
        n = int(rho.shape[0])
        if (not isinstance(rho, torch.Tensor) or rho.is_cuda or rho.dtype != dtype or tuple(rho.shape) != (n,) * 3
                or not rho.is_contiguous()):
            raise ValueError(f"request needs a contiguous CPU {dtype} tensor of shape {(n,) * 3}")
        if out is not None and (tuple(out.shape) != tuple(rho.shape) or out.dtype != dtype or out.is_cuda
                                or not out.is_contiguous()):
            raise ValueError(f"out must be a contiguous CPU {dtype} tensor like rho")
        return n, dtype

    def submit(self, rho, accuracy: float, arrival: float = None, out=None) -> Future:
        """Queue one solve.  rho: a CPU torch tensor (pinned for asynchronous copies) of
        shape (n, n, n), float32 for accuracy >= 1e-6 else float64.  The future yields
        the potential as a CPU tensor of the same shape and type: `out` if given (a
        pinned CPU tensor like rho, which the caller must not touch until the future is
        done), else a new pinned tensor.  arrival: monotonic seconds (time.monotonic)."""
        import ctypes
        fut = Future()
        precision = precision_for(accuracy)
        try:
            n, dtype = self._check(rho, precision, out)
        except ValueError as e:
            fut.set_exception(e)
            return fut
        if out is None:
            out = self.torch.empty(rho.shape, dtype=dtype, pin_memory=True)
        ticket = ctypes.c_longlong()
        with self._lock:  # registered before the completion thread can report it
            rc = self._N.lib.sp_server_submit(self._h, n, _PREC_CODE[precision], ctypes.c_void_p(rho.data_ptr()),
                                              ctypes.c_void_p(out.data_ptr()),
                                              -1.0 if arrival is None else float(arrival), ctypes.byref(ticket))
            if rc != 0:
                fut.set_exception(self._N.SuperpotError(rc, "sp_server_submit"))
                return fut
            self._pending[ticket.value] = (fut, out, rho)
        return fut

    def replay(self, arrivals, keys, inputs, outputs):
        """Requests submitted by the library at their arrival times (monotonic seconds,
        non-decreasing): keys[i] = (n, precision), inputs[i] / outputs[i] pinned CPU
        tensors.  Returns one future per request."""
        import ctypes
        count = len(arrivals)
        futs = [Future() for _ in range(count)]
        for key, x, y in zip(keys, inputs, outputs):
            self._check(x, key[1], y)
        arr = (ctypes.c_double * max(count, 1))(*arrivals)
        ns = (ctypes.c_int * max(count, 1))(*[int(k[0]) for k in keys])
        ps = (ctypes.c_int * max(count, 1))(*[_PREC_CODE[k[1]] for k in keys])
        ins = (ctypes.c_void_p * max(count, 1))(*[x.data_ptr() for x in inputs])
        outs = (ctypes.c_void_p * max(count, 1))(*[y.data_ptr() for y in outputs])
        tickets = (ctypes.c_longlong * max(count, 1))()
        with self._lock:
            self._N.check(self._N.lib.sp_server_replay(self._h, count, arr, ns, ps, ins, outs, tickets),
                          "sp_server_replay")
            for i in range(count):
                self._pending[tickets[i]] = (futs[i], outputs[i], inputs[i])
        return futs

    def _complete(self):
        import ctypes
        N = self._N
        ticket = ctypes.c_longlong()
        times = (ctypes.c_double * 3)()
        while True:
            ticket.value = -1
            rc = N.lib.sp_server_next_done(self._h, 0.05, ctypes.byref(ticket), times)
            if rc == 6:  # SP_ERR_NOT_READY: nothing finished within the wait
                continue
            if ticket.value < 0:  # the server has stopped and reported everything
                return
            with self._lock:
                entry = self._pending.pop(ticket.value, None)
            if entry is None:  # not a request of this client (cannot happen): keep serving
                continue
            fut, out, _ = entry
            if rc == 0:
                fut.set_result(out)
            elif rc == 3:  # SP_ERR_OOM: the key's plan can never fit the budget
                fut.set_exception(MemoryError(f"the request's plan needs more than the {self.budget} B budget"))
            else:
                fut.set_exception(N.SuperpotError(rc, "served request"))

    def stop(self):
        """Finish the batches in flight, fail requests still waiting, free the device."""
        if self._closed:
            return
        self._N.lib.sp_server_shutdown(self._h)
        self._stats()  # kept for reading after the server is gone
        _ = self.completed
        if self._thread is not None:
            self._thread.join()
        else:  # no completion thread: report what is left to the futures here
            self._complete()
        self._N.lib.sp_server_destroy(self._h)
        self._closed = True

    # ------------------------------------------------------------------ statistics
    def _stats(self):
        import ctypes
        b = ctypes.c_longlong()
        peak = ctypes.c_double()
        used = ctypes.c_double()
        if not self._closed:
            self._N.check(self._N.lib.sp_server_stats(self._h, ctypes.byref(b), ctypes.byref(peak),
                                                      ctypes.byref(used)), "sp_server_stats")
            self._last_stats = (b.value, peak.value, used.value)
        return self._last_stats

    @property
    def batches(self) -> int:
        return self._stats()[0]

    @property
    def peak_bytes(self) -> float:
        return self._stats()[1]

    @property
    def completed(self):
        """Completed requests: Done(arrival, done_at, key, launched_at), completion order."""
        if not self._closed:
            count = self._N.lib.sp_server_records(self._h, 0, None)
            recs = (self._N.ServerRecord * max(count, 1))()
            count = self._N.lib.sp_server_records(self._h, count, recs)
            self._last_records = [Done(r.arrival, r.done, (r.n, _PREC_NAME[r.precision]), r.launched)
                                  for r in recs[:count]]
        return self._last_records


def poisson_stream(server: Server, rate: float, duration: float, sizes, accuracies, seed: int = 0,
                   densities=None, warmup: float = 0.0, outputs=None, t0: float = None):
    """Drive `server` with Poisson arrivals (mean `rate` per second) for `warmup + duration`
    seconds from t0 (monotonic seconds; default now + 50 ms); each request draws its grid
    size and accuracy uniformly from the lists.  `densities[(n, precision)]` supplies the
    (pinned CPU) input of a key, `outputs[key]` a list of pinned result buffers used in
    turn (one new buffer per request when absent).  The library submits every request at
    its arrival time (sp_server_replay), so the client's own delays do not enter the
    latencies.  Waits for all of them and returns [(arrival offset, key)] of the requests
    that arrived after the warm-up."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    sched = []
    while t < warmup + duration:
        n = int(sizes[rng.integers(len(sizes))])
        acc = float(accuracies[rng.integers(len(accuracies))])
        sched.append((t, (n, precision_for(acc))))
        t += float(rng.exponential(1.0 / rate))
    if t0 is None:
        t0 = time.monotonic() + 0.05
    turn = collections.defaultdict(int)
    ins, outs = [], []
    for _, key in sched:
        ins.append(densities[key])
        if outputs is not None and outputs.get(key):
            pool = outputs[key]
            outs.append(pool[turn[key] % len(pool)])
            turn[key] += 1
        else:
            outs.append(densities[key].new_empty(densities[key].shape).pin_memory())
    futs = server.replay([t0 + s for s, _ in sched], [k for _, k in sched], ins, outs)
    deadline = t0 + warmup + duration + max(60.0, 2.0 * (warmup + duration))
    for f in futs:
        f.result(timeout=max(0.0, deadline - time.monotonic()))  # raise if a solve failed or never finished
    return [(s, key) for s, key in sched if s >= warmup]


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
