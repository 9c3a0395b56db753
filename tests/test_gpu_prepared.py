"""Prepared matrices: the tensor-core form's operands made once and reused.
Every call on a prepared matrix equals the same call on the matrix itself bit
for bit (and the FP64 oracle within tolerance), batch after batch, from
several contexts, for every kernel form."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2505_04556_gb300 as pm  # noqa: E402

RTOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pm.build()
    c = pm.Context(0)
    yield c
    c.close()


def _case(n, K, P, seed, ld=None):
    rng = np.random.default_rng(seed)
    D = synth.euclidean_matrix(rng.standard_normal((n, 6)))
    Dp = np.zeros((n, ld or n), dtype=np.float32)
    Dp[:, :n] = D
    sizes = synth.largest_remainder_sizes(n, rng.dirichlet(2 * np.ones(K)), min_size=2)
    obs = synth.observed_labels(sizes, seed + 1)
    rows = synth.shuffled_rows(obs, P, seed + 2)
    return D, torch.from_numpy(Dp).cuda(), rows, obs, synth.inv_sizes(obs, K)


@pytest.mark.parametrize("n,ld,K", [(1001, 1001, 4), (2177, 2180, 7), (300, 303, 30)])
def test_prepared_batches_equal_direct_calls(ctx, n, ld, K):
    D, Dd, rows, obs, w = _case(n, K, 600, n + K, ld)
    wd = torch.from_numpy(w).cuda()
    prep = pm.permanova_prepare(ctx.handle, Dd, n, ld)
    try:
        ref_all = oracle.sW_alg1(D, rows[::50], K, w.astype(np.float64))
        for b in range(3):   # three batches of 200 label rows on one preparation
            lab = torch.from_numpy(rows[200 * b:200 * (b + 1)].astype(np.uint8)).cuda()
            direct = torch.empty(200, dtype=torch.float64, device="cuda")
            pm.permanova_sW(ctx.handle, Dd, n, ld, lab, pm.LABEL_U8, K, 200, wd, direct)
            prepared = torch.full((200,), float("nan"), dtype=torch.float64, device="cuda")
            pm.permanova_sW_prepared(ctx.handle, prep, lab, pm.LABEL_U8, K, 200, wd, prepared)
            pm.permanova_sync(ctx.handle)
            assert np.array_equal(prepared.cpu().numpy(), direct.cpu().numpy())
            got = prepared.cpu().numpy()[::50]
            np.testing.assert_allclose(got, ref_all[4 * b:4 * (b + 1)], rtol=RTOL)
    finally:
        pm.permanova_prepared_destroy(prep)


@pytest.mark.parametrize("form", [pm.FORM_BRUTE, pm.FORM_PERMBLOCK, pm.FORM_GEMM])
def test_prepared_every_form(ctx, form):
    """A forced CUDA-core form reads the matrix itself; the GEMM form the
    prepared operands; all equal the direct call."""
    n, K, P = 777, 5, 70
    D, Dd, rows, obs, w = _case(n, K, P, 5)
    wd = torch.from_numpy(w).cuda()
    lab = torch.from_numpy(rows.astype(np.uint8)).cuda()
    prep = pm.permanova_prepare(ctx.handle, Dd, n, n)
    ctx.set_form(form)
    try:
        direct = ctx.sW(Dd, lab, K, wd)
        prepared = torch.empty(P, dtype=torch.float64, device="cuda")
        pm.permanova_sW_prepared(ctx.handle, prep, lab, pm.LABEL_U8, K, P, wd, prepared)
        pm.permanova_sync(ctx.handle)
    finally:
        ctx.set_form(pm.FORM_AUTO)
        pm.permanova_prepared_destroy(prep)
    assert np.array_equal(prepared.cpu().numpy(), direct.cpu().numpy())


def test_prepared_mixed_tests_from_two_contexts(ctx):
    """One prepared matrix serves permanova_test_mixed from two contexts, with
    the results of the unprepared call bit for bit."""
    n = 1500
    D, Dd, rows, obs, w = _case(n, 3, 10, 11)
    rng = np.random.default_rng(3)
    Ks, Ps = [2, 6, 40, 3], [199, 99, 149, 299]
    labs = [synth.observed_labels(synth.largest_remainder_sizes(n, rng.dirichlet(2 * np.ones(K)),
                                                                min_size=2), 60 + k)
            for k, K in enumerate(Ks)]
    seeds = [5, 6, 7, 8]
    g = torch.from_numpy(np.stack(labs)).cuda()
    direct = pm.permanova_test_mixed(ctx.handle, Dd, n, n, g, Ks, Ps, seeds)
    prep = pm.permanova_prepare(ctx.handle, Dd, n, n)
    try:
        with pm.Context(0) as other:
            for c in (ctx, other):
                out = pm.permanova_test_mixed_prepared(c.handle, prep, g, Ks, Ps, seeds)
                assert out == direct
    finally:
        pm.permanova_prepared_destroy(prep)
    ref = oracle.permanova_test(D, labs[0], Ks[0], Ps[0], seeds[0])
    assert abs(direct[0]["s_W_obs"] - ref["s_W"][0]) <= 1e-5 * ref["s_W"][0]


def test_prepare_rejects_bad_arguments(ctx):
    D, Dd, *_ = _case(64, 2, 4, 1)
    with pytest.raises(pm.PermanovaError) as ei:
        pm.permanova_prepare(ctx.handle, Dd, 64, 32)
    assert ei.value.status == pm.EINVAL
