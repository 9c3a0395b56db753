"""Continuous-batching PERMANOVA server on one GPU.

Requests (matrix id, one categorical factor, number of permutations, seed)
arrive at any time.  Distance matrices stay resident in HBM.  A request is
admitted as soon as an execution slot is free and its scratch fits the HBM
budget left by the requests already running; requests that arrive while
others run are admitted as slots and memory free up, so the GPU always holds
the work of several tests at once.  When a slot frees up, the waiting
requests on the same matrix with the same number of groups and permutations
are batched with the oldest one into a single ``permanova_test_batch`` call:
one permutation launch, one s_W launch over all their label rows (each test
with its own weights), one finalize launch.  Each slot owns a permanova
context (its own scratch arena) and a CUDA stream; slots run concurrently and
their kernels overlap on the device.

Results do not depend on the mix: every test's kernels are deterministic
(fixed-order reductions, per-row results independent of the other rows in a
launch, the kernel form chosen by a single test's sizes), so a test gives
bit-identical s_W, F and p alone, batched, and among other traffic.

Latency is measured from arrival (submit) to completion; the server reports
tests/s and p50/p99 latency.
"""
from __future__ import annotations

import collections
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

import paper_2505_04556_gb300 as pm


@dataclass(eq=False)   # requests compare by identity (they hold label arrays)
class Request:
    matrix_id: int
    grouping: object          # host int32 labels (numpy)
    n_groups: int
    n_perms: int
    seed: int
    t_arrival: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    result: dict | None = None
    error: str | None = None
    batch_size: int = 1       # tests that shared this request's launch
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


def take_batch(pending: "collections.deque[Request]", in_use: int, budget: int,
               max_batch: int) -> tuple[list[Request], int]:
    """Admission: the oldest waiting request, if its scratch fits the budget
    left, plus the waiting requests that can share its launch (same matrix,
    number of groups and permutations) and still fit, in arrival order, up to
    ``max_batch``.  Removes them from ``pending``; returns the batch (empty if
    the oldest does not fit) and the budget in use afterwards.  Requests carry
    their scratch estimate as ``_need``."""
    if not pending or pending[0]._need + in_use > budget:
        return [], in_use
    head = pending.popleft()
    in_use += head._need
    batch = [head]
    key = (head.matrix_id, head.n_groups, head.n_perms)
    for r in list(pending):
        if len(batch) >= max_batch:
            break
        if (r.matrix_id, r.n_groups, r.n_perms) == key and in_use + r._need <= budget:
            pending.remove(r)
            in_use += r._need
            batch.append(r)
    return batch, in_use


class Server:
    """``matrices``: dict id -> square fp32 CUDA tensor (resident)."""

    def __init__(self, matrices: dict, n_slots: int = 4, hbm_budget_bytes: int = 0,
                 device: int = 0, max_batch: int = 16):
        import torch
        self.torch = torch
        self.max_batch = max_batch
        self.device = device
        self.matrices = matrices
        free, _ = torch.cuda.mem_get_info(device)
        self.budget = hbm_budget_bytes or int(free * 0.8)
        self.in_use = 0
        self.cv = threading.Condition()
        self.pending: collections.deque[Request] = collections.deque()
        self.free_slots: queue.SimpleQueue = queue.SimpleQueue()
        self.slots = []
        for k in range(n_slots):
            ctx = pm.Context(device)
            stream = torch.cuda.Stream(device=device)
            self.slots.append((ctx, stream))
            self.free_slots.put(k)
        self.completed: list[Request] = []
        self.running = True
        self.dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self.dispatcher.start()

    # -- admission ----------------------------------------------------------
    def scratch_estimate(self, req: Request) -> int:
        n = self.matrices[req.matrix_id].shape[0]
        rows = req.n_perms + 1
        ctx = self.slots[0][0].handle
        sw = pm.permanova_scratch_bytes(ctx, pm.FORM_AUTO, n, req.n_groups, rows)
        return sw + rows * n * 2 + rows * 8 + (1 << 20)

    def submit(self, req: Request) -> Request:
        req.t_arrival = time.perf_counter()
        need = self.scratch_estimate(req)
        if need > self.budget:
            req.error = f"request needs {need} bytes, more than the HBM budget {self.budget}"
            req.t_done = time.perf_counter()
            req.done.set()
            return req
        req._need = need
        with self.cv:
            self.pending.append(req)
            self.cv.notify_all()
        return req

    def _dispatch(self):
        while True:
            slot = self.free_slots.get()          # blocks until a slot frees up
            with self.cv:
                while self.running and (not self.pending or
                                        self.pending[0]._need + self.in_use > self.budget):
                    self.cv.wait(timeout=0.05)
                if not self.running:
                    self.free_slots.put(slot)
                    return
                # the oldest request plus the waiting ones that can share its launch
                batch, self.in_use = take_batch(self.pending, self.in_use, self.budget,
                                                self.max_batch)
            threading.Thread(target=self._run, args=(slot, batch), daemon=True).start()

    def _run(self, slot: int, batch: list[Request]):
        torch = self.torch
        ctx, stream = self.slots[slot]
        t0 = time.perf_counter()
        for r in batch:
            r.t_start = t0
        try:
            head = batch[0]
            D = self.matrices[head.matrix_id]
            with torch.cuda.stream(stream):
                g = torch.from_numpy(np.stack([r.grouping for r in batch]).astype(np.int32)).to(
                    device=D.device, non_blocking=False)
                results = pm.permanova_test_batch(ctx.handle, D, D.shape[0], D.stride(0), g,
                                                  len(batch), head.n_groups, head.n_perms,
                                                  [r.seed for r in batch],
                                                  stream=stream.cuda_stream)
            for r, res in zip(batch, results):
                r.result = res
        except Exception as e:  # reported per request; the server keeps running
            for r in batch:
                r.error = str(e)
        finally:
            t1 = time.perf_counter()
            with self.cv:
                for r in batch:
                    r.t_done = t1
                    r.batch_size = len(batch)
                    self.in_use -= r._need
                    self.completed.append(r)
                self.cv.notify_all()
            self.free_slots.put(slot)
            for r in batch:
                r.done.set()

    def close(self):
        with self.cv:
            self.running = False
            self.cv.notify_all()
        self.dispatcher.join(timeout=5)
        for ctx, _ in self.slots:
            ctx.close()

    # -- reporting ----------------------------------------------------------
    @staticmethod
    def summarize(reqs: list[Request], wall_s: float) -> dict:
        lat = sorted(r.latency for r in reqs if r.error is None)
        if not lat:
            return {"tests": 0}

        def pct(q):
            return lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
        return {"tests": len(lat), "errors": sum(r.error is not None for r in reqs),
                "tests_per_s": len(lat) / wall_s, "p50_s": pct(0.50), "p99_s": pct(0.99),
                "wall_s": wall_s}
