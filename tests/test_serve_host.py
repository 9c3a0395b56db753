"""Host logic of the serving loop (CPU): admission and batching of waiting
requests, and the latency summary."""
import collections
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2505_04556_gb300.serve import Request, Server, take_batch  # noqa: E402


def _req(mid, K, P, need, tag):
    r = Request(matrix_id=mid, grouping=np.zeros(4, np.int32), n_groups=K, n_perms=P, seed=tag)
    r._need = need
    return r


def test_oldest_request_first_with_compatible_followers_in_order():
    q = collections.deque([_req(0, 3, 999, 10, 1), _req(1, 3, 999, 10, 2),
                           _req(0, 3, 999, 10, 3), _req(0, 4, 999, 10, 4),
                           _req(0, 3, 999, 10, 5)])
    batch, used = take_batch(q, 0, 1000, 16)
    assert [r.seed for r in batch] == [1, 3, 5]        # same matrix, K and P as the oldest
    assert used == 30
    assert [r.seed for r in q] == [2, 4]               # the rest keep their order


def test_budget_and_batch_size_limit_the_batch():
    q = collections.deque([_req(0, 3, 999, 40, k) for k in range(5)])
    batch, used = take_batch(q, 0, 100, 16)             # only two more fit after the head
    assert [r.seed for r in batch] == [0, 1]
    assert used == 80
    q = collections.deque([_req(0, 3, 999, 1, k) for k in range(5)])
    batch, used = take_batch(q, 0, 100, 3)
    assert [r.seed for r in batch] == [0, 1, 2] and len(q) == 2


def test_oldest_that_does_not_fit_waits():
    q = collections.deque([_req(0, 3, 999, 60, 0), _req(0, 3, 999, 5, 1)])
    batch, used = take_batch(q, 50, 100, 16)            # 50 in use, the oldest needs 60
    assert batch == [] and used == 50 and len(q) == 2
    assert take_batch(collections.deque(), 0, 100, 16) == ([], 0)


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
