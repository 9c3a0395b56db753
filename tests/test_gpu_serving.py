"""Serving loop: continuous admission, overlapping execution, and results that
do not depend on the traffic mix."""
import time

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def matrices():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_04556_gb300 as pm
    pm.build()
    rng = np.random.default_rng(11)
    mats, hosts = {}, {}
    for mid, n in enumerate((300, 777, 1500)):
        D = synth.euclidean_matrix(rng.standard_normal((n, 6)))
        hosts[mid] = D
        mats[mid] = torch.from_numpy(D).cuda()
    return mats, hosts


def _requests(hosts, seed):
    from paper_2505_04556_gb300.serve import Request
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(12):
        mid = k % len(hosts)
        n = hosts[mid].shape[0]
        K = int(rng.integers(2, 7))
        sizes = synth.largest_remainder_sizes(n, rng.dirichlet(np.ones(K) * 2), min_size=2)
        lab = synth.observed_labels(sizes, 100 + k)
        P = int(rng.choice([99, 499]))
        reqs.append(Request(mid, lab, K, P, seed=1000 + k))
    return reqs


def test_results_identical_alone_and_in_the_mix(matrices):
    from paper_2505_04556_gb300.serve import Server
    mats, hosts = matrices
    # alone: one slot, one request at a time
    alone = []
    srv = Server(mats, n_slots=1)
    try:
        for r in _requests(hosts, 5):
            srv.submit(r)
            assert r.done.wait(120)
            assert r.error is None, r.error
            alone.append(r.result)
    finally:
        srv.close()
    # mixed: four slots, everything submitted at once
    srv = Server(mats, n_slots=4)
    try:
        reqs = _requests(hosts, 5)
        for r in reqs:
            srv.submit(r)
        for r in reqs:
            assert r.done.wait(120)
            assert r.error is None, r.error
        overlap = any(a.t_start < b.t_done and b.t_start < a.t_done
                      for i, a in enumerate(reqs) for b in reqs[i + 1:])
        assert overlap, "no two tests were in flight together"
        for r, ref in zip(reqs, alone):
            for key in ("s_T", "s_W_obs", "F_obs", "p_value", "n_ge", "n_perms"):
                assert r.result[key] == ref[key], key
        summary = Server.summarize(reqs, max(r.t_done for r in reqs) - min(r.t_arrival for r in reqs))
        assert summary["tests"] == len(reqs) and summary["p99_s"] >= summary["p50_s"]
    finally:
        srv.close()


def test_batch_equals_single_tests(matrices):
    import paper_2505_04556_gb300 as pm
    mats, hosts = matrices
    n = hosts[1].shape[0]
    labs = [synth.observed_labels(synth.largest_remainder_sizes(n, [3, 2, 1 + k]), 40 + k)
            for k in range(5)]
    seeds = [7 + 3 * k for k in range(5)]
    with pm.Context(0) as ctx:
        single = [ctx.test(mats[1], torch.from_numpy(l).cuda(), 3, 199, s) for l, s in zip(labs, seeds)]
        g = torch.from_numpy(np.stack(labs)).cuda()
        out = torch.empty((5, 200), dtype=torch.float64, device="cuda")
        batch = pm.permanova_test_batch(ctx.handle, mats[1], n, n, g, 5, 3, 199, seeds, out)
    for a, b in zip(single, batch):
        assert a == b
    ref = oracle.permanova_test(hosts[1], labs[2], 3, 199, seeds[2])
    np.testing.assert_allclose(out[2].cpu().numpy(), ref["s_W"], rtol=1e-5)


def test_compatible_requests_are_batched(matrices):
    from paper_2505_04556_gb300.serve import Request, Server
    mats, hosts = matrices
    n = hosts[2].shape[0]

    def reqs():
        return [Request(2, synth.observed_labels([n // 2, n - n // 2], 60 + k), 2, 299, seed=500 + k)
                for k in range(10)]
    srv = Server(mats, n_slots=1)
    try:
        alone = []
        for r in reqs():
            srv.submit(r)
            assert r.done.wait(120) and r.error is None
            alone.append(r.result)
        mixed = reqs()
        for r in mixed:
            srv.submit(r)
        for r in mixed:
            assert r.done.wait(120) and r.error is None, r.error
    finally:
        srv.close()
    assert max(r.batch_size for r in mixed) > 1
    for r, ref in zip(mixed, alone):
        assert r.result == ref


def test_served_result_matches_oracle(matrices):
    from paper_2505_04556_gb300.serve import Request, Server
    mats, hosts = matrices
    lab = synth.observed_labels([300, 277, 200], 3)
    srv = Server(mats, n_slots=2)
    try:
        r = srv.submit(Request(1, lab, 3, 199, seed=77))
        assert r.done.wait(120) and r.error is None
    finally:
        srv.close()
    ref = oracle.permanova_test(hosts[1], lab, 3, 199, 77)
    assert abs(r.result["s_W_obs"] - ref["s_W"][0]) <= 1e-5 * ref["s_W"][0]
    band = np.abs(ref["s_W"][1:] - ref["s_W"][0]) <= 1e-5 * ref["s_W"][0]
    if not band.any():
        assert r.result["n_ge"] == ref["n_ge"]


def test_oversized_request_rejected_not_run(matrices):
    from paper_2505_04556_gb300.serve import Request, Server
    mats, hosts = matrices
    srv = Server(mats, n_slots=1, hbm_budget_bytes=1 << 20)
    try:
        r = srv.submit(Request(2, synth.observed_labels([750, 750], 1), 2, 999, seed=1))
        assert r.done.wait(5)
        assert r.error is not None and "budget" in r.error
    finally:
        srv.close()


def test_mixed_batch_equals_single_tests(matrices):
    """Tests on one matrix with different group counts and permutation counts,
    run through one permanova_test_mixed call (one s_W pass per kernel form:
    here the tensor-core form for K <= 24, the perm-block form for K = 40 and
    the brute force for 9 permutations), equal the same tests run one by one
    bit for bit, and their s_W rows land in caller order."""
    import paper_2505_04556_gb300 as pm
    mats, hosts = matrices
    n = hosts[1].shape[0]
    rng = np.random.default_rng(17)
    Ks = [2, 12, 5, 40, 3, 7]
    Ps = [199, 99, 499, 149, 9, 299]
    labs = [synth.observed_labels(synth.largest_remainder_sizes(n, rng.dirichlet(2 * np.ones(K)),
                                                                min_size=2), 70 + k)
            for k, K in enumerate(Ks)]
    seeds = [101 + 5 * k for k in range(len(Ks))]
    with pm.Context(0) as ctx:
        single, single_sw = [], []
        for lab, K, P, sd in zip(labs, Ks, Ps, seeds):
            o = torch.empty(P + 1, dtype=torch.float64, device="cuda")
            single.append(ctx.test(mats[1], torch.from_numpy(lab).cuda(), K, P, sd, out_sW=o))
            single_sw.append(o.cpu().numpy())
        forms = {pm.permanova_plan_form(ctx.handle, n, K, P + 1) for K, P in zip(Ks, Ps)}
        assert forms == {pm.FORM_GEMM, pm.FORM_PERMBLOCK, pm.FORM_BRUTE}
        g = torch.from_numpy(np.stack(labs)).cuda()
        out = torch.empty(sum(P + 1 for P in Ps), dtype=torch.float64, device="cuda")
        mixed = pm.permanova_test_mixed(ctx.handle, mats[1], n, n, g, Ks, Ps, seeds, out)
    off = 0
    for a, b, sw, P in zip(single, mixed, single_sw, Ps):
        assert a == b
        assert np.array_equal(out[off:off + P + 1].cpu().numpy(), sw)
        off += P + 1
    ref = oracle.permanova_test(hosts[1], labs[1], Ks[1], Ps[1], seeds[1])
    np.testing.assert_allclose(single_sw[1], ref["s_W"], rtol=1e-5)


def test_server_fuses_different_group_and_permutation_counts(matrices):
    """Requests on one matrix with different K and P are fused into one call
    by the server, and each result equals the request served alone."""
    from paper_2505_04556_gb300.serve import Request, Server
    mats, hosts = matrices
    n = hosts[0].shape[0]   # 300 objects: a small matrix, so the padding cap never splits

    def reqs():
        out = []
        for k in range(8):
            K = 2 + (k % 5)
            sizes = synth.largest_remainder_sizes(n, np.ones(K), min_size=2)
            out.append(Request(0, synth.observed_labels(sizes, 90 + k), K, (99, 199)[k % 2],
                               seed=900 + k))
        return out
    srv = Server(mats, n_slots=1)
    try:
        alone = []
        for r in reqs():
            srv.submit(r)
            assert r.done.wait(120) and r.error is None, r.error
            alone.append(r.result)
        mixed = reqs()
        for r in mixed:
            srv.submit(r)
        for r in mixed:
            assert r.done.wait(120) and r.error is None, r.error
    finally:
        srv.close()
    assert max(r.batch_size for r in mixed) > 1
    for r, ref in zip(mixed, alone):
        assert r.result == ref


def test_back_pressure_refuses_beyond_the_waiting_limit(matrices):
    """With max_pending set, requests that find the waiting queue full are
    refused at once with a "server busy" error; admitted ones complete."""
    from paper_2505_04556_gb300.serve import Request, Server
    mats, hosts = matrices
    n = hosts[2].shape[0]
    srv = Server(mats, n_slots=1, max_pending=2)
    try:
        reqs = [srv.submit(Request(2, synth.observed_labels([n // 2, n - n // 2], 80 + k), 2, 999,
                                   seed=700 + k)) for k in range(12)]
        for r in reqs:
            assert r.done.wait(120)
    finally:
        srv.close()
    busy = [r for r in reqs if r.error and "server busy" in r.error]
    served = [r for r in reqs if r.error is None]
    assert busy and served and len(busy) + len(served) == len(reqs)


def test_prepared_server_results_equal_unprepared(matrices):
    """A server that prepares its matrices gives the results of one that
    does not, request for request."""
    from paper_2505_04556_gb300.serve import Server
    mats, hosts = matrices
    out = []
    for prepare in (False, True):
        srv = Server(mats, n_slots=2, prepare=prepare)
        try:
            reqs = _requests(hosts, 9)
            for r in reqs:
                srv.submit(r)
            for r in reqs:
                assert r.done.wait(120) and r.error is None, r.error
            if prepare:
                assert srv.prepared
        finally:
            srv.close()
        out.append([r.result for r in reqs])
    assert out[0] == out[1]
