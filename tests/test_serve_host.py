"""Host logic of the serving loop (CPU): admission and batching of waiting
requests (fusion across group and permutation counts within one kernel form,
the padding cap of the tensor-core form, budgets that count the scratch each
slot keeps), and the latency summary."""
import collections
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import paper_2505_04556_gb300 as pm  # noqa: E402
from paper_2505_04556_gb300.serve import Request, Server, fusable, take_batch  # noqa: E402

GEMM, PB = pm.FORM_GEMM, pm.FORM_PERMBLOCK


def _req(mid, K, P, need, tag, form=GEMM, pairs=1e6):
    r = Request(matrix_id=mid, grouping=np.zeros(4, np.int32), n_groups=K, n_perms=P, seed=tag)
    r._need, r._form, r._pairs = need, form, pairs
    return r


def test_oldest_request_first_with_fusable_followers_in_order():
    q = collections.deque([_req(0, 3, 999, 10, 1), _req(1, 3, 999, 10, 2),
                           _req(0, 3, 9999, 10, 3), _req(0, 4, 999, 10, 4, form=PB),
                           _req(0, 3, 999, 10, 5)])
    batch, charged = take_batch(q, 0, 0, 1000, 16)
    # same matrix and kernel form as the oldest, any permutation count
    assert [r.seed for r in batch] == [1, 3, 5]
    assert charged == 30
    assert [r.seed for r in q] == [2, 4]               # the rest keep their order


def test_tensor_core_padding_cap():
    big = 1e9                                          # pairs of a large matrix: no small-batch exemption
    head = _req(0, 4, 999, 1, 0, pairs=big)
    assert fusable([head], _req(0, 5, 999, 1, 1, pairs=big))       # 5*2000 <= 1.25*9000
    assert not fusable([head], _req(0, 12, 999, 1, 2, pairs=big))  # 12*2000 > 1.25*16000
    # the CUDA-core forms cost the same for every group count
    pb = _req(0, 40, 999, 1, 3, form=PB, pairs=big)
    assert fusable([pb], _req(0, 90, 99, 1, 4, form=PB, pairs=big))
    # small matrices fuse regardless (launch overheads dominate)
    small = _req(0, 2, 999, 1, 5, pairs=1e5)
    assert fusable([small], _req(0, 12, 999, 1, 6, pairs=1e5))
    assert not fusable([small], _req(1, 2, 999, 1, 7, pairs=1e5))  # other matrix


def test_budget_counts_the_scratch_slots_keep():
    q = collections.deque([_req(0, 3, 999, 40, k) for k in range(5)])
    batch, charged = take_batch(q, 0, 0, 100, 16)       # only two more fit after the head
    assert [r.seed for r in batch] == [0, 1] and charged == 80
    q = collections.deque([_req(0, 3, 999, 1, k) for k in range(5)])
    batch, _ = take_batch(q, 0, 0, 100, 3)
    assert [r.seed for r in batch] == [0, 1, 2] and len(q) == 2
    # this slot already keeps 70 bytes: a 10-byte batch is charged 70
    q = collections.deque([_req(0, 3, 999, 10, 0)])
    batch, charged = take_batch(q, 20, 70, 100, 16)
    assert len(batch) == 1 and charged == 70
    # other slots keep 50: the same request no longer fits next to a 70-byte arena
    q = collections.deque([_req(0, 3, 999, 10, 0)])
    assert take_batch(q, 50, 70, 100, 16) == ([], 0) and len(q) == 1


def test_oldest_that_does_not_fit_waits():
    q = collections.deque([_req(0, 3, 999, 60, 0), _req(0, 3, 999, 5, 1)])
    batch, charged = take_batch(q, 50, 0, 100, 16)      # 50 held elsewhere, the oldest needs 60
    assert batch == [] and charged == 0 and len(q) == 2
    assert take_batch(collections.deque(), 0, 0, 100, 16) == ([], 0)


def test_batch_need_callback():
    q = collections.deque([_req(0, 3, 999, 10, k) for k in range(4)])
    batch, charged = take_batch(q, 0, 0, 100, 16, need_of=lambda b: 25 + 5 * len(b))
    assert len(batch) == 4 and charged == 45


def test_summary_percentiles_ignore_failed_requests():
    reqs = []
    for k in range(100):
        r = _req(0, 3, 999, 1, k)
        r.t_arrival, r.t_done = 0.0, (k + 1) / 1000.0
        reqs.append(r)
    bad = _req(0, 3, 999, 1, 999)
    bad.error, bad.t_arrival, bad.t_done = "too big", 0.0, 5.0
    out = Server.summarize(reqs + [bad], wall_s=2.0)
    assert out["tests"] == 100 and out["errors"] == 1
    assert out["tests_per_s"] == 50.0
    assert abs(out["p50_s"] - 0.051) < 1e-12 and abs(out["p99_s"] - 0.099) < 1e-12
