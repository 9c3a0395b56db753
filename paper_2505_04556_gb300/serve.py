"""Continuous-batching PERMANOVA server on one GPU.

Requests (matrix id, one categorical factor, number of permutations, seed)
arrive at any time.  Distance matrices stay resident in HBM.  A request is
admitted as soon as an execution slot is free and the batch's scratch fits
the HBM budget, counting the scratch every slot's context still holds from
earlier work (a context keeps its arena between calls; idle slots give theirs
back when the budget is short).  Requests that arrive while others run are
admitted as slots and memory free up, so the GPU always holds the work of
several tests at once.

When a slot frees up, the oldest waiting request is batched with the waiting
requests on the same matrix that run in the same kernel form (the form a lone
test of their sizes gets), whatever their number of groups and permutations:
one ``permanova_test_mixed`` call runs them all in one s_W pass over the
matrix (Sec. 1: many tests are typically run on one distance matrix).  For the
tensor-core form the pass works on the largest group count of the batch, so a
request joins only while that padding costs at most ``pad_cap`` times the
batch's unpadded work, unless the whole batch is small enough for launch
overheads to dominate.  Each slot owns a permanova context (its own scratch
arena) and a CUDA stream; slots run concurrently and their kernels overlap on
the device.

Results do not depend on the mix: every test's kernels are deterministic
(fixed-order reductions, per-row results independent of the other rows in a
launch and of the padded group count, the kernel form chosen by a single
test's sizes), so a test gives bit-identical s_W, F and p alone, batched and
among other traffic.

With ``prepare=True`` each resident matrix's tensor-core operands are made
once, on its first request, and shared by every slot (about 2 n^2 bytes per
matrix), so later requests skip that pass over the matrix.

Latency is measured from arrival (submit) to completion; the server reports
tests/s and p50/p99 latency.  With ``max_pending`` set, a request that finds
that many requests already waiting is refused at once ("server busy"), so
the latency of admitted requests stays bounded under overload.
"""
from __future__ import annotations

import collections
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

import paper_2505_04556_gb300 as pm

PAD_CAP = 1.25            # tensor-core form: padded work / unpadded work of a fused batch
SMALL_BATCH_EVALS = 2e10  # below this many pair-permutation evaluations a batch always fuses


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


def fusable(batch: list, r, pad_cap: float = PAD_CAP, small_evals: float = SMALL_BATCH_EVALS) -> bool:
    """Whether request ``r`` may join ``batch`` in one s_W pass: same matrix,
    same kernel form (``_form``), and for the tensor-core form a padding cost
    within ``pad_cap`` unless the batch stays small.  Requests carry
    ``_pairs`` (pairs of their matrix) and ``_form``."""
    head = batch[0]
    if r.matrix_id != head.matrix_id or r._form != head._form:
        return False
    if head._form != pm.FORM_GEMM:
        return True                       # the CUDA-core forms cost the same for any group count
    members = batch + [r]
    rows = sum(m.n_perms + 1 for m in members)
    kmax = max(m.n_groups for m in members)
    padded = kmax * rows
    exact = sum(m.n_groups * (m.n_perms + 1) for m in members)
    if padded <= pad_cap * exact:
        return True
    return head._pairs * rows <= small_evals


def take_batch(pending: "collections.deque[Request]", held_elsewhere: int, held_here: int,
               budget: int, max_batch: int, need_of=None) -> tuple[list[Request], int]:
    """Admission for one slot: the oldest waiting request, if the batch's
    scratch fits the budget, plus the waiting requests that can share its s_W
    pass (:func:`fusable`) and still fit, in arrival order, up to
    ``max_batch``.  The slot already holds ``held_here`` bytes (its arena) and
    the other slots ``held_elsewhere``; a batch needing B bytes is charged
    max(held_here, B).  ``need_of(batch)`` gives B (default: the sum of the
    requests' ``_need``).  Removes the batch from ``pending``; returns it
    (empty if the oldest does not fit) and the bytes charged to the slot."""
    need_of = need_of or (lambda b: sum(r._need for r in b))

    def charge(b):
        return max(held_here, need_of(b))

    if not pending or held_elsewhere + charge([pending[0]]) > budget:
        return [], 0
    batch = [pending.popleft()]
    for r in list(pending):
        if len(batch) >= max_batch:
            break
        if fusable(batch, r) and held_elsewhere + charge(batch + [r]) <= budget:
            pending.remove(r)
            batch.append(r)
    return batch, charge(batch)


class Server:
    """``matrices``: dict id -> square fp32 CUDA tensor (resident)."""

    def __init__(self, matrices: dict, n_slots: int = 4, hbm_budget_bytes: int = 0,
                 device: int = 0, max_batch: int = 16, reserve_per_slot: int = 0,
                 max_pending: int = 0, prepare: bool = False):
        import torch
        self.torch = torch
        self.max_batch = max_batch
        self.max_pending = max_pending    # 0: unbounded; else requests beyond it are refused
        self.device = device
        self.matrices = matrices
        free, _ = torch.cuda.mem_get_info(device)
        self.budget = hbm_budget_bytes or int(free * 0.8)
        self.cv = threading.Condition()
        self.pending: collections.deque[Request] = collections.deque()
        self.free_slots: queue.SimpleQueue = queue.SimpleQueue()
        self.slots = []
        for k in range(n_slots):
            ctx = pm.Context(device)
            stream = torch.cuda.Stream(device=device)
            self.slots.append((ctx, stream))
            self.free_slots.put(k)
        self.reserved = [0] * n_slots     # arena bytes each slot's context keeps
        if reserve_per_slot:
            # size every slot's arena up front, so requests do not pay its growth
            per = min(int(reserve_per_slot), self.budget // n_slots)
            for k, (ctx, _) in enumerate(self.slots):
                pm.permanova_reserve_scratch(ctx.handle, per)
                self.reserved[k] = pm.permanova_scratch_reserved(ctx.handle)
        # prepared matrices: the tensor-core operands of each resident matrix made
        # once (on its first request) and shared by every slot
        self.prepare = prepare
        self.prepared: dict = {}
        self.prep_lock = threading.Lock()
        self.charged = [0] * n_slots      # bytes charged to the batch running on a slot
        self.busy = [False] * n_slots
        self.completed: list[Request] = []
        self.running = True
        self.dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self.dispatcher.start()

    # -- admission ----------------------------------------------------------
    def batch_need(self, batch: list[Request]) -> int:
        """Scratch of one fused call: the s_W scratch of the padded pass plus
        the label rows, s_W values and per-test tables."""
        n = self.matrices[batch[0].matrix_id].shape[0]
        rows = sum(r.n_perms + 1 for r in batch)
        kmax = max(r.n_groups for r in batch)
        ctx = self.slots[0][0].handle
        sw = pm.permanova_scratch_bytes(ctx, batch[0]._form, n, kmax, rows)
        return sw + rows * n * (1 if kmax <= 256 else 2) + rows * 8 + (1 << 20)

    def submit(self, req: Request) -> Request:
        req.t_arrival = time.perf_counter()
        n = self.matrices[req.matrix_id].shape[0]
        req._pairs = n * (n - 1) / 2
        req._form = pm.permanova_plan_form(self.slots[0][0].handle, n, req.n_groups, req.n_perms + 1)
        need = self.batch_need([req])
        if need > self.budget:
            req.error = f"request needs {need} bytes, more than the HBM budget {self.budget}"
            req.t_done = time.perf_counter()
            req.done.set()
            return req
        req._need = need
        with self.cv:
            if self.max_pending and len(self.pending) >= self.max_pending:
                # back-pressure: the caller learns at once that the server is full
                req.error = f"server busy: {len(self.pending)} requests waiting (limit {self.max_pending})"
                req.t_done = time.perf_counter()
                req.done.set()
                return req
            self.pending.append(req)
            self.cv.notify_all()
        return req

    def _held(self, s: int) -> int:
        return max(self.reserved[s], self.charged[s])

    def _dispatch(self):
        while True:
            slot = self.free_slots.get()          # blocks until a slot frees up
            with self.cv:
                while True:
                    if not self.running:
                        self.free_slots.put(slot)
                        return
                    if self.pending:
                        elsewhere = sum(self._held(s) for s in range(len(self.slots)) if s != slot)
                        batch, charge = take_batch(self.pending, elsewhere, self.reserved[slot],
                                                   self.budget, self.max_batch, self.batch_need)
                        if batch:
                            break
                        # short of memory: idle slots give back the arenas they keep
                        idle = [s for s in range(len(self.slots))
                                if s != slot and not self.busy[s] and self.reserved[s] > 0]
                        if idle:
                            for s in idle:
                                pm.permanova_release_scratch(self.slots[s][0].handle)
                                self.reserved[s] = 0
                            continue
                    self.cv.wait(timeout=0.05)
                self.busy[slot] = True
                self.charged[slot] = charge
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
                args = ([r.n_groups for r in batch], [r.n_perms for r in batch], [r.seed for r in batch])
                prep = self._prepared(head.matrix_id, ctx, stream) if self.prepare else None
                if prep is not None:
                    results = pm.permanova_test_mixed_prepared(ctx.handle, prep, g, *args,
                                                               stream=stream.cuda_stream)
                else:
                    results = pm.permanova_test_mixed(ctx.handle, D, D.shape[0], D.stride(0), g, *args,
                                                      stream=stream.cuda_stream)
            for r, res in zip(batch, results):
                r.result = res
        except Exception as e:  # reported per request; the server keeps running
            for r in batch:
                r.error = str(e)
        finally:
            t1 = time.perf_counter()
            reserved = pm.permanova_scratch_reserved(ctx.handle)
            with self.cv:
                for r in batch:
                    r.t_done = t1
                    r.batch_size = len(batch)
                    self.completed.append(r)
                self.reserved[slot] = reserved
                self.charged[slot] = 0
                self.busy[slot] = False
                self.cv.notify_all()
            self.free_slots.put(slot)
            for r in batch:
                r.done.set()

    def _prepared(self, matrix_id: int, ctx, stream):
        """The prepared operands of a resident matrix, made on first use."""
        with self.prep_lock:
            prep = self.prepared.get(matrix_id)
            if prep is None:
                D = self.matrices[matrix_id]
                prep = pm.permanova_prepare(ctx.handle, D, D.shape[0], D.stride(0),
                                            stream=stream.cuda_stream)
                self.prepared[matrix_id] = prep
            return prep

    def close(self):
        with self.cv:
            self.running = False
            self.cv.notify_all()
        self.dispatcher.join(timeout=5)
        for prep in self.prepared.values():
            pm.permanova_prepared_destroy(prep)
        self.prepared.clear()
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
                "wall_s": wall_s, "mean_batch": float(np.mean([r.batch_size for r in reqs]))}
