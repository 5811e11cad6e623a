"""Continuous-batching server for landmark-label distance queries.

The graph's labels stay resident on the GPU (``cbfs.Labels``, built from
C-BFS outputs).  Requests -- arrays of vertex pairs of any size -- arrive at
any time through ``submit`` and get a ticket whose ``result()`` returns the
answers.  Scheduling is native (``cbfs_server_*`` in libcbfs.so): a
dispatcher thread packs waiting requests, in arrival order, into batches of
at most ``max_batch`` pairs and launches each batch on one of ``slots`` CUDA
streams as soon as a slot and its memory are free (page-locked staging -> H2D
copy -> query kernel -> D2H copy); batches launched while others are still on
the GPU overlap with them (continuous batching, not a queue in front of one
batch at a time).  One waiter thread per stream completes requests as soon as
their batch finishes, whatever the order batches were launched in.  Latency
is measured natively, from ``submit`` to the answers being in host memory.

Admission by memory: the server's batch buffers (10 bytes per pair: int32
pair + uint16 answer, ``slots * max_batch`` pairs) are allocated at start
inside ``memory_budget_bytes`` (default: a quarter of the device memory free
at that moment; ``max_batch`` shrinks to fit), and a batch is launched only
when the bytes of the batches in flight plus its own fit that budget.
Requests larger than ``max_batch`` are split over several batches and
resolved when the last part is done.  The answers of a request do not depend
on what else is in flight: every pair is answered independently by the same
kernel.
"""
from __future__ import annotations

import concurrent.futures
import ctypes
import gc
import sys
import threading
import time

import numpy as np
import torch

from . import cbfs


class Ticket:
    """A submitted request; ``result()`` blocks until its answers are in."""

    __slots__ = ("_server", "_id", "_pairs", "_out", "_done", "_exc", "_lock")

    def __init__(self, server: "QueryServer", ticket: int, pairs: np.ndarray, out: np.ndarray):
        self._server, self._id, self._pairs, self._out = server, ticket, pairs, out
        self._done, self._exc = False, None
        self._lock = threading.Lock()

    def _wait(self, timeout_s: float) -> bool:
        with self._lock:
            if self._done:
                return True
            rc = cbfs.lib().cbfs_server_wait(self._server._h, ctypes.c_uint64(self._id), float(timeout_s))
            if rc == cbfs.E_TIMEOUT:
                return False
            self._done = True
            self._pairs = None  # the server no longer reads it
            if rc != cbfs.OK:
                self._exc = cbfs.CbfsError(rc, "cbfs_server_wait")
            self._server._forget(self._id)
            return True

    def done(self) -> bool:
        return self._wait(0.0)

    def result(self, timeout: float | None = None) -> np.ndarray:
        """uint16 [q] answers (0xFFFF: no common landmark)."""
        if not self._wait(-1.0 if timeout is None else timeout):
            raise concurrent.futures.TimeoutError()
        if self._exc is not None:
            raise self._exc
        return self._out


class QueryServer:
    def __init__(self, labels: "cbfs.Labels", max_batch: int = 65536, slots: int = 4,
                 memory_budget_bytes: int | None = None, device=None, pause_gc: bool = False,
                 switch_interval_s: float | None = None):
        """``pause_gc`` disables Python's cyclic garbage collector while the
        server runs and ``switch_interval_s`` shortens the interpreter's
        thread switch interval: both only help the Python clients that submit
        and wait (scheduling itself is native).  Both are process-wide
        settings, restored by ``close``."""
        if device is not None and torch.device(device).index not in (None, torch.cuda.current_device()):
            raise ValueError("the server runs on the current CUDA device")
        self._gc_was_enabled = gc.isenabled()
        self._old_switch = sys.getswitchinterval()
        self._pause_gc = pause_gc
        self.labels = labels
        self._h = ctypes.c_void_p()
        cbfs._check(cbfs.lib().cbfs_server_create(labels._h, int(max_batch), int(slots),
                                                  int(memory_budget_bytes or 0), ctypes.byref(self._h)),
                    "cbfs_server_create")
        if pause_gc:
            gc.disable()
        if switch_interval_s:
            sys.setswitchinterval(switch_interval_s)
        self._open = {}  # ticket id -> Ticket not yet waited for
        self._mu = threading.Lock()
        c = self._counts()
        self.max_batch, self.budget = int(c[3]), int(c[4])

    # ----------------------------------------------------------------- API
    def submit(self, pairs, out: np.ndarray | None = None) -> Ticket:
        """Queue a request (int32 [q, 2] vertex pairs); ``result()`` yields
        uint16 [q], written into ``out`` when given (a contiguous uint16 array
        of q entries).  Page-locked buffers (``cbfs.pinned_empty``) are copied
        by DMA with no host copy in the server; both must stay untouched
        until ``result()`` returns."""
        if isinstance(pairs, torch.Tensor):
            pairs = pairs.numpy()
        p = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        if out is None:
            out = np.empty(p.shape[0], dtype=np.uint16)
        elif out.dtype != np.uint16 or out.shape != (p.shape[0],) or not out.flags.c_contiguous:
            raise ValueError("out must be a contiguous uint16 array with one entry per pair")
        tid = ctypes.c_uint64()
        cbfs._check(cbfs.lib().cbfs_server_submit(self._h, p.ctypes.data if p.size else None, int(p.shape[0]),
                                                  out.ctypes.data if p.size else None, ctypes.byref(tid)),
                    "cbfs_server_submit")
        t = Ticket(self, tid.value, p, out)
        with self._mu:
            self._open[tid.value] = t
        return t

    def _forget(self, tid: int):
        with self._mu:
            self._open.pop(tid, None)

    def close(self):
        if not self._h.value:
            return
        with self._mu:
            left = list(self._open.values())
        for t in left:  # every request is answered before the server goes
            t._wait(-1.0)
        cbfs.lib().cbfs_server_destroy(self._h)
        self._h = ctypes.c_void_p()
        sys.setswitchinterval(self._old_switch)
        if self._pause_gc and self._gc_was_enabled:
            gc.enable()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _counts(self):
        c = (ctypes.c_uint64 * 5)()
        cbfs._check(cbfs.lib().cbfs_server_stats(self._h, c, None, 0, None), "cbfs_server_stats")
        return list(c)

    def stats(self) -> dict:
        """Completed requests, batches, pairs answered and the latency
        percentiles (ms, arrival to answers on the host)."""
        n = ctypes.c_int64()
        cbfs._check(cbfs.lib().cbfs_server_stats(self._h, None, None, 0, ctypes.byref(n)), "cbfs_server_stats")
        lat = np.zeros(max(n.value, 1), dtype=np.float64)
        c = (ctypes.c_uint64 * 5)()
        cbfs._check(cbfs.lib().cbfs_server_stats(self._h, c, lat.ctypes.data, lat.size, ctypes.byref(n)),
                    "cbfs_server_stats")
        lat = lat[:max(min(n.value, lat.size), 1)]
        return {"requests": int(c[0]), "batches": int(c[1]), "pairs": int(c[2]),
                "p50_ms": float(np.percentile(lat, 50)), "p90_ms": float(np.percentile(lat, 90)),
                "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
                "mean_ms": float(lat.mean()), "max_batch": int(c[3]), "budget_bytes": int(c[4])}


class RequestPool:
    """Requests of a load generator: slices of one pool of uniform random
    pairs, and answer buffers from a ring (the ticket that last used a ring
    entry is waited for before the entry is reused).  ``pinned`` puts both in
    page-locked memory, which the server copies by DMA."""

    def __init__(self, n: int, max_pairs: int, seed: int, pinned: bool = False, ring: int = 512):
        rng = np.random.Generator(np.random.PCG64(seed))
        pairs = rng.integers(0, n, size=(4 * max_pairs, 2), dtype=np.int64).astype(np.int32)
        if pinned:
            self.pairs = cbfs.pinned_empty(pairs.shape, torch.int32).numpy()
            self.pairs[:] = pairs
            self.outs = cbfs.pinned_empty((ring, max_pairs), torch.int16).numpy().view(np.uint16)
        else:
            self.pairs = pairs
            self.outs = np.empty((ring, max_pairs), np.uint16)
        self.users = [None] * ring
        self.next = 0

    def submit(self, server: QueryServer, start: int, q: int) -> Ticket:
        i = self.next
        self.next = (i + 1) % len(self.users)
        if self.users[i] is not None:
            self.users[i].result()
        t = server.submit(self.pairs[start:start + q], out=self.outs[i, :q])
        self.users[i] = t
        return t


def poisson_load(server: QueryServer, n: int, rate_rps: float, duration_s: float, max_pairs: int, seed: int,
                 pinned: bool = False):
    """Offers requests with exponential inter-arrival times (rate_rps per
    second) and sizes uniform in 1..max_pairs for duration_s seconds; each
    request is a slice of a pregenerated pool of uniform random pairs
    (``RequestPool``; page-locked with ``pinned``), so the client itself is
    not the bottleneck.  Returns (tickets, pairs offered, elapsed seconds).
    With ``pinned`` a ticket's answers stay valid only until its answer
    buffer is reused, 512 requests later."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pool = RequestPool(n, max_pairs, seed=int(rng.integers(1 << 62)), pinned=pinned)
    gaps = rng.exponential(1.0 / rate_rps, size=1 << 16)
    sizes = rng.integers(1, max_pairs + 1, size=1 << 16)
    starts = rng.integers(0, 3 * max_pairs + 1, size=1 << 16)
    futs, offered = [], 0
    t0 = time.perf_counter()
    t_next = t0
    i = 0
    while True:
        t_next += gaps[i % gaps.size]
        if t_next - t0 > duration_s:
            break
        now = time.perf_counter()
        if t_next > now:
            time.sleep(t_next - now)
        q, s0 = int(sizes[i % sizes.size]), int(starts[i % starts.size])
        futs.append(pool.submit(server, s0, q))
        offered += q
        i += 1
    for f in futs:
        f.result()
    return futs, offered, time.perf_counter() - t0
