"""Continuous-batching connected-components server over the FastSV pool.

Requests (CSR graphs in host memory) arrive on any thread through
``Server.submit``; one scheduler thread owns the device pool and loops:

  1. admit queued requests in arrival order while the pool has a free slot
     and enough of its HBM budget (a request that can never fit is failed);
  2. run ``iters_per_step`` FastSV iterations over every resident graph
     (``fastsv_pool_step``: one device-side loop over all slots), admitting
     the requests that arrive meanwhile so that their copies to the device
     overlap the step;
  3. harvest graphs that reached their early termination (Section 3.4 of the
     paper) -- their labels are copied to host memory and their slot and
     memory are freed for the next admissions.

Optional preemption under memory pressure (``preempt_after_steps``): when
the request at the head of the queue has not fitted for that many steps, the
largest resident graph that has run at least as long is checkpointed to host
memory (its f, f[f] and iteration count) and freed, and queued right behind
the head; restored later, it resumes exactly where it stopped.

Graphs admitted while others are on the device join the running batch at the
next iteration boundary; each graph's iteration sequence depends only on its
own edges, so its labels and iteration count are the same alone and in any
mix.  Latency is measured from ``submit`` to labels available on the host.
"""
from __future__ import annotations

import collections
import threading
import time
from concurrent.futures import Future

import numpy as np

from . import _lib


class PoolBackend:
    """The device pool of one libfastsv handle (C ABI fastsv_pool_*)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int, **opts):
        import torch
        from . import FastSV
        torch.cuda.init()
        self.solver = FastSV(rowptr_bits=32, **opts)
        self.h = self.solver.h
        _lib.check(_lib.fastsv_pool_create(self.h, int(hbm_budget_bytes), int(max_slots)), "fastsv_pool_create")
        self.max_slots = max_slots
        self.budget = hbm_budget_bytes
        self._done = np.zeros(max_slots, dtype=np.int32)
        self._iters = np.zeros(max_slots, dtype=np.int32)
        self._stream = torch.cuda.Stream()
        self._n: dict[int, int] = {}  # vertices of the graph in each occupied slot

    def host_buffer(self, n: int) -> np.ndarray:
        """int32 host buffer for a graph's labels, in pinned memory so that the
        device-to-host copy of a harvest runs at full link speed.  Pinning is
        slow: allocate these ahead of time and reuse them."""
        import torch
        return torch.empty(max(n, 1), dtype=torch.int32).pin_memory().numpy()

    def bytes_for(self, n: int, m: int) -> int:
        return _lib.fastsv_pool_bytes(n, m)

    def add(self, rp: np.ndarray, ci: np.ndarray, labels: np.ndarray):
        """Returns a slot id, or None if the pool is full right now."""
        n = len(rp) - 1
        st, slot = _lib.fastsv_pool_add(self.h, n, rp.ctypes.data, ci.ctypes.data if len(ci) else None,
                                        labels.ctypes.data if n > 0 else None)
        if st == _lib.FASTSV_ERR_FULL:
            return None
        _lib.check(st, "fastsv_pool_add")
        self._n[slot] = n
        return slot

    def step(self, iters: int):
        _lib.check(_lib.fastsv_pool_step(self.h, iters, int(self._stream.cuda_stream)), "fastsv_pool_step")

    def poll(self):
        """[(slot, iterations)] of graphs whose labels are now on the host,
        and the number still resident."""
        st, nd, na = _lib.fastsv_pool_poll(self.h, self._done.ctypes.data, self._iters.ctypes.data,
                                           self.max_slots)
        _lib.check(st, "fastsv_pool_poll")
        return [(int(self._done[i]), int(self._iters[i])) for i in range(nd)], na

    def evict(self, slot: int) -> np.ndarray:
        """Checkpoint a still-iterating slot to host memory and free it
        (fastsv_pool_evict).  Returns the checkpoint."""
        n = self.slot_vertices(slot)
        buf = self._pinned_bytes(_lib.fastsv_pool_checkpoint_bytes(n))
        _lib.check(_lib.fastsv_pool_evict(self.h, slot, buf.ctypes.data), "fastsv_pool_evict")
        return buf

    def restore(self, rp: np.ndarray, ci: np.ndarray, labels: np.ndarray, checkpoint: np.ndarray):
        """Admit a graph again from its checkpoint; a slot id, or None if the
        pool is full right now."""
        n = len(rp) - 1
        st, slot = _lib.fastsv_pool_restore(self.h, n, rp.ctypes.data, ci.ctypes.data if len(ci) else None,
                                            labels.ctypes.data if n > 0 else None, checkpoint.ctypes.data)
        if st == _lib.FASTSV_ERR_FULL:
            return None
        _lib.check(st, "fastsv_pool_restore")
        self._n[slot] = n
        return slot

    def slot_vertices(self, slot: int) -> int:
        return self._n[slot]

    def _pinned_bytes(self, nbytes: int) -> np.ndarray:
        import torch
        return torch.empty(max(nbytes, 1), dtype=torch.uint8).pin_memory().numpy()

    def kernel_launches(self) -> int:
        return self.solver.kernel_launches()

    def close(self):
        self.solver.close()


class Request:
    __slots__ = ("rp", "ci", "labels", "future", "t_submit", "t_admit", "t_done", "slot", "iterations",
                 "checkpoint", "blocked_steps", "resident_steps", "evictions")

    def __init__(self, rp, ci, labels=None):
        self.rp = np.ascontiguousarray(rp, dtype=np.int32)
        self.ci = np.ascontiguousarray(ci, dtype=np.int32)
        n = max(len(self.rp) - 1, 1)
        if labels is None:
            labels = np.empty(n, dtype=np.int32)
        assert labels.dtype == np.int32 and labels.flags.c_contiguous and len(labels) >= len(self.rp) - 1
        self.labels = labels
        self.future: Future = Future()
        self.t_submit = time.perf_counter()
        self.t_admit = None
        self.t_done = None
        self.slot = None
        self.iterations = None
        self.checkpoint = None   # host checkpoint while evicted
        self.blocked_steps = 0   # steps spent at the head of the queue without fitting
        self.resident_steps = 0  # steps since (re-)admission
        self.evictions = 0


class Server:
    """Continuous-batching CC server.  ``submit(rp, ci)`` returns a Future
    resolving to ``(labels, iterations)``."""

    def __init__(self, hbm_budget_bytes: int = 1 << 30, max_slots: int = 256, iters_per_step: int = 1,
                 backend=None, preempt_after_steps: int = 0, max_evictions: int = 1, **opts):
        self.backend = backend if backend is not None else PoolBackend(hbm_budget_bytes, max_slots, **opts)
        self.iters_per_step = iters_per_step
        # preemption under memory pressure (0 = off): when the request at the
        # head of the queue has not fitted for this many steps, the resident
        # graph that has run at least as many steps and holds the most memory
        # is checkpointed to host memory (fastsv_pool_evict) and queued right
        # behind the head; it resumes where it stopped (fastsv_pool_restore)
        self.preempt_after_steps = preempt_after_steps
        self.max_evictions = max_evictions
        self.evictions = 0
        self._queue: collections.deque[Request] = collections.deque()
        self._resident: dict[int, Request] = {}
        self._cv = threading.Condition()
        self._stop = False
        self.completed: list[Request] = []
        self.steps = 0
        self.error: BaseException | None = None
        self._thread = threading.Thread(target=self._run, name="fastsv-server", daemon=True)
        self._thread.start()

    # -- client side ------------------------------------------------------
    def submit(self, rp, ci, labels=None) -> Future:
        """Queue one graph (int32 CSR in host memory).  ``labels``: optional
        int32 host buffer of n entries that receives the result; a pinned one
        (e.g. from ``PoolBackend.host_buffer``, allocated ahead of time)
        makes the copy back asynchronous.  Pinning host memory is slow, so it
        is not done per request."""
        req = Request(rp, ci, labels)
        n = len(req.rp) - 1
        if self.backend.bytes_for(n, len(req.ci)) > self.backend.budget:
            req.future.set_exception(ValueError("graph larger than the pool's HBM budget"))
            return req.future
        with self._cv:
            if self._stop or self.error is not None:
                raise RuntimeError("server is closed")
            self._queue.append(req)
            self._cv.notify()
        return req.future

    def close(self, wait: bool = True):
        with self._cv:
            self._stop = True
            self._cv.notify()
        if wait:
            self._thread.join()
        self.backend.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- metrics ----------------------------------------------------------
    def latencies(self) -> np.ndarray:
        return np.array([r.t_done - r.t_submit for r in self.completed])

    def summary(self) -> dict:
        lat = self.latencies()
        if len(lat) == 0:
            return {"completed": 0}
        t0 = min(r.t_submit for r in self.completed)
        t1 = max(r.t_done for r in self.completed)
        return {"completed": len(lat), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "graphs_per_s": len(lat) / max(t1 - t0, 1e-9), "steps": self.steps}

    # -- scheduler thread -------------------------------------------------
    def _admit(self):
        while self._queue:
            req = self._queue[0]
            if req.checkpoint is not None:
                slot = self.backend.restore(req.rp, req.ci, req.labels, req.checkpoint)
            else:
                slot = self.backend.add(req.rp, req.ci, req.labels)
            if slot is None:
                if self._preempt_for(req):
                    continue  # memory was freed: try the head again
                return  # full: keep arrival order, wait for a harvest
            self._queue.popleft()
            req.slot = slot
            req.checkpoint = None
            req.resident_steps = 0
            req.blocked_steps = 0
            if req.t_admit is None:
                req.t_admit = time.perf_counter()
            self._resident[slot] = req

    def _preempt_for(self, head: Request) -> bool:
        k = self.preempt_after_steps
        if k <= 0 or head.blocked_steps < k or head.evictions > 0:
            return False  # off, not waiting long enough, or itself a preempted graph (no ping-pong)
        victims = [r for r in self._resident.values()
                   if r.resident_steps >= k and r.evictions < self.max_evictions]
        if not victims:
            return False
        v = max(victims, key=lambda r: len(r.ci) + len(r.rp))
        v.checkpoint = self.backend.evict(v.slot)
        del self._resident[v.slot]
        v.slot = None
        v.evictions += 1
        self.evictions += 1
        self._queue.insert(1, v)  # resumes right after the request it made room for
        return True

    def _run(self):
        try:
            while True:
                with self._cv:
                    while not self._stop and not self._queue and not self._resident:
                        self._cv.wait()
                    if self._stop and not self._queue and not self._resident:
                        return
                    self._admit()
                if self._resident:
                    self.backend.step(self.iters_per_step)
                    self.steps += 1
                    for r in self._resident.values():
                        r.resident_steps += 1
                    with self._cv:
                        # requests that arrived meanwhile start copying to the
                        # device while the step runs; they join the next one
                        self._admit()
                        if self._queue:
                            self._queue[0].blocked_steps += 1
                    done, _ = self.backend.poll()
                    now = time.perf_counter()
                    for slot, iters in done:
                        req = self._resident.pop(slot)
                        req.t_done = now
                        req.iterations = iters
                        n = len(req.rp) - 1
                        self.completed.append(req)
                        if iters < 0:
                            req.future.set_exception(_lib.FastSVError(_lib.FASTSV_ERR_MAX_ITERS, "serve"))
                        else:
                            req.future.set_result((req.labels[:n], iters))
        except BaseException as e:  # fail every outstanding request, never hang a client
            with self._cv:
                pending = list(self._queue) + list(self._resident.values())
                self._queue.clear()
                self._resident.clear()
            for r in pending:
                if not r.future.done():
                    r.future.set_exception(e)
            self.error = e
