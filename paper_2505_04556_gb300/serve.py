"""Continuous-batching PERMANOVA server on one GPU.

Requests (matrix id, one categorical factor, number of permutations, seed)
arrive at any time.  Distance matrices stay resident in HBM.  A request is
admitted as soon as an execution slot is free and its scratch fits the HBM
budget left by the requests already running; requests that arrive while
others run are admitted as slots and memory free up, so the GPU always holds
the work of several tests at once.  Each slot owns a permanova context (its
own scratch arena) and a CUDA stream, and runs ``permanova_test`` through
the C ABI; slots run concurrently, their kernels overlap on the device.

Results do not depend on the mix: every test's kernels are deterministic
(fixed-order reductions), so a test gives bit-identical s_W, F and p alone
and among other traffic.

Latency is measured from arrival (submit) to completion; the server reports
tests/s and p50/p99 latency.
"""
from __future__ import annotations

import collections
import queue
import threading
import time
from dataclasses import dataclass, field

import paper_2505_04556_gb300 as pm


@dataclass
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
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class Server:
    """``matrices``: dict id -> square fp32 CUDA tensor (resident)."""

    def __init__(self, matrices: dict, n_slots: int = 4, hbm_budget_bytes: int = 0,
                 device: int = 0):
        import torch
        self.torch = torch
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
            with self.cv:
                while self.running and (not self.pending or
                                        self.pending[0]._need + self.in_use > self.budget):
                    self.cv.wait(timeout=0.05)
                if not self.running:
                    return
                req = self.pending.popleft()
                self.in_use += req._need
            slot = self.free_slots.get()          # blocks until a slot frees up
            threading.Thread(target=self._run, args=(slot, req), daemon=True).start()

    def _run(self, slot: int, req: Request):
        torch = self.torch
        ctx, stream = self.slots[slot]
        try:
            req.t_start = time.perf_counter()
            D = self.matrices[req.matrix_id]
            with torch.cuda.stream(stream):
                g = torch.from_numpy(req.grouping).to(device=D.device, non_blocking=False)
                req.result = ctx.test(D, g, req.n_groups, req.n_perms, req.seed,
                                      stream=stream.cuda_stream)
        except Exception as e:  # reported per request; the server keeps running
            req.error = str(e)
        finally:
            req.t_done = time.perf_counter()
            with self.cv:
                self.in_use -= req._need
                self.completed.append(req)
                self.cv.notify_all()
            self.free_slots.put(slot)
            req.done.set()

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
