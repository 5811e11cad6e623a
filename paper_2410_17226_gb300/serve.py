"""Continuous-batching server for landmark-label distance queries.

The graph's labels stay resident on the GPU (``cbfs.Labels``, built from
C-BFS outputs).  Requests -- arrays of vertex pairs of any size -- arrive at
any time through ``submit`` and get a future.  A scheduler thread packs
waiting requests, in arrival order, into batches of at most ``max_batch``
pairs and launches each batch on one of ``slots`` CUDA streams as soon as a
slot and its memory are free: pinned host staging -> H2D copy -> query kernel
(``cbfs_query_distance``) -> D2H copy.  Batches launched while others are
still on the GPU overlap with them (continuous batching, not a queue in front
of one batch at a time).  A completion thread resolves the futures when a
batch's event fires and records each request's latency from its arrival to
its answer being on the host.

Admission by memory: every in-flight batch holds ``pairs * 10`` bytes of
device buffers (8 B pair + 2 B answer) from a budget of
``memory_budget_bytes``; a batch starts only when its bytes fit.  Requests
larger than ``max_batch`` are split over several batches and resolved when
the last part is done.  The answers of a request do not depend on what else
is in flight: every pair is answered independently by the same kernel.
"""
from __future__ import annotations

import collections
import gc
import sys
import threading
import time
from concurrent.futures import Future

import numpy as np
import torch

from . import cbfs

PAIR_BYTES = 8 + 2  # int32 pair + uint16 answer


class _Request:
    __slots__ = ("pairs", "future", "t_arrival", "answers", "remaining", "t_done")

    def __init__(self, pairs: np.ndarray, t_arrival: float):
        self.pairs = pairs
        self.future = Future()
        self.t_arrival = t_arrival
        self.answers = np.empty(pairs.shape[0], dtype=np.uint16)
        self.remaining = pairs.shape[0]
        self.t_done = None


class _Slot:
    """One stream with its pinned staging and device buffers."""

    def __init__(self, max_batch: int, device):
        self.stream = torch.cuda.Stream(device=device)
        self.h_pairs = cbfs.pinned_empty((max_batch, 2), torch.int32)
        self.h_out = cbfs.pinned_empty(max_batch, torch.int16)
        self.d_pairs = torch.empty((max_batch, 2), dtype=torch.int32, device=device)
        self.d_out = torch.empty(max_batch, dtype=torch.int16, device=device)
        self.event = torch.cuda.Event()
        self.parts = []  # (request, offset in request, offset in batch, count)
        self.count = 0
        self.bytes = 0


class QueryServer:
    def __init__(self, labels: "cbfs.Labels", max_batch: int = 65536, slots: int = 4,
                 memory_budget_bytes: int | None = None, device=None, pause_gc: bool = False,
                 switch_interval_s: float | None = None):
        """``pause_gc`` disables Python's cyclic garbage collector while the
        server runs (its pauses over many live requests were the latency
        tail); ``switch_interval_s`` shortens the interpreter's thread switch
        interval so the scheduler and completion threads do not wait 5 ms
        turns.  Both are process-wide settings, restored by ``close``."""
        self._gc_was_enabled = gc.isenabled()
        self._old_switch = sys.getswitchinterval()
        self._pause_gc = pause_gc
        if pause_gc:
            gc.disable()
        if switch_interval_s:
            sys.setswitchinterval(switch_interval_s)
        self.labels = labels
        self.max_batch = int(max_batch)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.budget = int(memory_budget_bytes) if memory_budget_bytes else slots * self.max_batch * PAIR_BYTES
        if self.budget < PAIR_BYTES:
            raise ValueError("memory budget below one pair")
        self._free_slots = collections.deque(_Slot(self.max_batch, self.device) for _ in range(slots))
        self._inflight = collections.deque()
        self._pending = collections.deque()  # [request, offset]
        self._used = 0
        self._cv = threading.Condition()
        self._stop = False
        self.latencies_ms = []
        self.batches = 0
        self.pairs_done = 0
        self.errors = []
        self._sched = threading.Thread(target=self._schedule, name="cbfs-serve-sched", daemon=True)
        self._compl = threading.Thread(target=self._complete, name="cbfs-serve-done", daemon=True)
        self._sched.start()
        self._compl.start()

    # ----------------------------------------------------------------- API
    def submit(self, pairs) -> Future:
        """Queue a request (int32 [q, 2] vertex pairs); the future yields uint16 [q]."""
        p = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        req = _Request(p, time.perf_counter())
        if p.shape[0] == 0:
            req.t_done = req.t_arrival
            req.future.set_result(req.answers)
            return req.future
        with self._cv:
            if self._stop:
                raise RuntimeError("server closed")
            self._pending.append([req, 0])
            self._cv.notify_all()
        return req.future

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        self._sched.join()
        self._compl.join()
        sys.setswitchinterval(self._old_switch)
        if self._pause_gc and self._gc_was_enabled:
            gc.enable()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def stats(self) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"requests": len(self.latencies_ms), "batches": self.batches, "pairs": self.pairs_done,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean())}

    # ------------------------------------------------------------ threads
    def _schedule(self):
        while True:
            with self._cv:
                while True:
                    if self._stop and not self._pending:
                        self._cv.notify_all()
                        return
                    if self._pending and self._free_slots and self._used + PAIR_BYTES <= self.budget:
                        break
                    self._cv.wait()
                slot = self._free_slots.popleft()
                # pack waiting requests in arrival order until the batch or the budget is full
                room = min(self.max_batch, (self.budget - self._used) // PAIR_BYTES)
                slot.parts, slot.count = [], 0
                while self._pending and slot.count < room:
                    item = self._pending[0]
                    req, off = item
                    take = min(req.pairs.shape[0] - off, room - slot.count)
                    slot.parts.append((req, off, slot.count, take))
                    slot.count += take
                    if off + take == req.pairs.shape[0]:
                        self._pending.popleft()
                    else:
                        item[1] = off + take
                slot.bytes = slot.count * PAIR_BYTES
                self._used += slot.bytes
            try:
                self._launch(slot)
            except Exception as exc:  # surface kernel/launch failures on the futures
                self.errors.append(exc)
                for req, _, _, _ in slot.parts:
                    if not req.future.done():
                        req.future.set_exception(exc)
                with self._cv:
                    self._used -= slot.bytes
                    self._free_slots.append(slot)
                    self._cv.notify_all()
                continue
            with self._cv:
                self._inflight.append(slot)
                self._cv.notify_all()

    def _launch(self, slot: _Slot):
        hp = slot.h_pairs.numpy()
        for req, off, pos, cnt in slot.parts:
            hp[pos:pos + cnt] = req.pairs[off:off + cnt]
        q = slot.count
        with torch.cuda.stream(slot.stream):
            slot.d_pairs[:q].copy_(slot.h_pairs[:q], non_blocking=True)
            self.labels.query(slot.d_pairs[:q], out=slot.d_out[:q], stream=slot.stream)
            slot.h_out[:q].copy_(slot.d_out[:q], non_blocking=True)
            slot.event.record(slot.stream)

    def _complete(self):
        while True:
            with self._cv:
                while not self._inflight:
                    if self._stop and not self._pending and not self._sched.is_alive():
                        return
                    self._cv.wait(timeout=0.05)
                slot = self._inflight[0]
            slot.event.synchronize()
            now = time.perf_counter()
            ho = slot.h_out.numpy().view(np.uint16)
            finished = []
            for req, off, pos, cnt in slot.parts:
                req.answers[off:off + cnt] = ho[pos:pos + cnt]
                req.remaining -= cnt
                if req.remaining == 0:
                    req.t_done = now
                    finished.append(req)
            with self._cv:
                self._inflight.popleft()
                self._used -= slot.bytes
                self.batches += 1
                self.pairs_done += slot.count
                for req in finished:
                    self.latencies_ms.append((req.t_done - req.t_arrival) * 1e3)
                self._free_slots.append(slot)
                self._cv.notify_all()
            for req in finished:
                req.future.set_result(req.answers)


def poisson_load(server: QueryServer, n: int, rate_rps: float, duration_s: float, max_pairs: int, seed: int):
    """Offers requests with exponential inter-arrival times (rate_rps per
    second) and sizes uniform in 1..max_pairs for duration_s seconds; each
    request is a slice of a pregenerated pool of uniform random pairs, so the
    client itself is not the bottleneck.  Returns (futures, pairs offered,
    elapsed seconds)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pool = rng.integers(0, n, size=(4 * max_pairs, 2), dtype=np.int64).astype(np.int32)
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
        futs.append(server.submit(pool[s0:s0 + q]))
        offered += q
        i += 1
    for f in futs:
        f.result()
    return futs, offered, time.perf_counter() - t0
