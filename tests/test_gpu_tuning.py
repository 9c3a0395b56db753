"""Autotuner and CUDA-graph replay: the chosen plan and the replayed launch
sequence give the same s_W as direct launches."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2505_04556_gb300 as pm  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pm.build()
    c = pm.Context(0)
    yield c
    c.close()


def _case(n, K, P, seed):
    rng = np.random.default_rng(seed)
    D = synth.euclidean_matrix(rng.standard_normal((n, 6)))
    sizes = synth.largest_remainder_sizes(n, rng.dirichlet(2 * np.ones(K)), min_size=1)
    obs = synth.observed_labels(sizes, seed + 1)
    rows = synth.shuffled_rows(obs, P, seed + 2)
    return D, rows, synth.inv_sizes(obs, K)


def test_planner_boundary(ctx):
    """Without a tuned bucket the planner takes the GEMM form up to 24 groups
    and the perm-block form from 25 (measured crossover at n = 20k)."""
    assert pm.permanova_plan_form(ctx.handle, 20000, 24, 4000) == pm.FORM_GEMM
    assert pm.permanova_plan_form(ctx.handle, 20000, 25, 4000) == pm.FORM_PERMBLOCK


def test_autotune_then_auto_plan(ctx):
    n, K, P = 900, 4, 300
    D, rows, w = _case(n, K, P, 3)
    Dd, lab, wd = (torch.from_numpy(D).cuda(), torch.from_numpy(rows.astype(np.uint8)).cuda(),
                   torch.from_numpy(w).cuda())
    form = pm.permanova_autotune(ctx.handle, Dd, n, n, lab, pm.LABEL_U8, K, P, wd)
    assert form in (pm.FORM_BRUTE, pm.FORM_PERMBLOCK, pm.FORM_GEMM)
    assert pm.permanova_plan_form(ctx.handle, n, K, P) == form
    out = ctx.sW(Dd, lab, K, wd)
    pm.permanova_sync(ctx.handle)
    ref = oracle.sW_alg1(D, rows, K, w.astype(np.float64))
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-5)


def test_graph_replay_matches_direct_launches(ctx):
    n, K, P = 700, 3, 200
    D, rows, w = _case(n, K, P, 4)
    Dd, wd = torch.from_numpy(D).cuda(), torch.from_numpy(w).cuda()
    lab = torch.from_numpy(rows.astype(np.uint8)).cuda()
    stream = torch.cuda.Stream()
    direct = torch.empty(P, dtype=torch.float64, device="cuda")
    pm.permanova_sW(ctx.handle, Dd, n, n, lab, pm.LABEL_U8, K, P, wd, direct, stream)
    pm.permanova_sync(ctx.handle, stream)
    # kernels one direct call launches (the counter runs with profiling off)
    pm.permanova_profile_enable(ctx.handle, False)
    pm.permanova_sW(ctx.handle, Dd, n, n, lab, pm.LABEL_U8, K, P, wd, direct, stream)
    pm.permanova_sync(ctx.handle, stream)
    per_call = pm.permanova_profile_read(ctx.handle)["kernel_launches"]
    assert per_call >= 2
    pm.permanova_set_graphs(ctx.handle, True)
    try:
        out = torch.empty(P, dtype=torch.float64, device="cuda")
        for _ in range(3):   # capture once, then replay
            out.fill_(float("nan"))
            pm.permanova_sW(ctx.handle, Dd, n, n, lab, pm.LABEL_U8, K, P, wd, out, stream)
            pm.permanova_sync(ctx.handle, stream)
            assert torch.equal(out, direct)
        # replayed kernels are counted like launched ones
        assert pm.permanova_profile_read(ctx.handle)["kernel_launches"] == 3 * per_call
        # replays read the buffers at run time: new labels in the same buffer
        rows2 = synth.shuffled_rows(rows[0], P, 99)
        with torch.cuda.stream(stream):
            lab.copy_(torch.from_numpy(rows2.astype(np.uint8)))
        pm.permanova_sW(ctx.handle, Dd, n, n, lab, pm.LABEL_U8, K, P, wd, out, stream)
        pm.permanova_sync(ctx.handle, stream)
        ref2 = oracle.sW_alg1(D, rows2, K, w.astype(np.float64))
        np.testing.assert_allclose(out.cpu().numpy(), ref2, rtol=1e-5)
    finally:
        pm.permanova_set_graphs(ctx.handle, False)


@pytest.mark.parametrize("plan", [
    dict(form=pm.FORM_BRUTE, brute_chunk_mult=2),
    dict(form=pm.FORM_PERMBLOCK, permblock_variant=0),
    dict(form=pm.FORM_PERMBLOCK, permblock_variant=1),
    dict(form=pm.FORM_PERMBLOCK, permblock_variant=2),
    dict(form=pm.FORM_GEMM, gemm_rows_div=2, gemm_drain_kblocks=8),
    dict(form=pm.FORM_GEMM, gemm_rows_div=4, gemm_drain_kblocks=4),
    dict(form=pm.FORM_GEMM, gemm_rows_div=1, gemm_drain_kblocks=3),
], ids=["brute-x2", "pb-pair", "pb-f32", "pb-pair3", "gemm-half-8", "gemm-quarter-4", "gemm-full-3"])
@pytest.mark.parametrize("n,K,P", [(1001, 4, 300), (2500, 3, 257), (640, 40, 130)])
def test_every_plan_matches_oracle(ctx, plan, n, K, P):
    """Every knob setting the autotuner can pick gives s_W within the stated
    tolerance of the FP64 oracle (sizes with ragged tiles and label-row
    blocks; K = 40 exceeds the tensor-core form's usual range but runs)."""
    D, rows, w = _case(n, K, P, n + K)
    Dd, lab, wd = (torch.from_numpy(D).cuda(), torch.from_numpy(rows.astype(np.uint8)).cuda(),
                   torch.from_numpy(w).cuda())
    pm.permanova_set_plan(ctx.handle, **plan)
    try:
        desc = pm.permanova_plan_describe(ctx.handle, n, K, P)
        assert desc["source"] == "forced"
        out = ctx.sW(Dd, lab, K, wd)
        pm.permanova_sync(ctx.handle)
    finally:
        pm.permanova_set_plan(ctx.handle, pm.FORM_AUTO)
    ref = oracle.sW_alg1(D, rows, K, w.astype(np.float64))
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-5)


def test_plan_knob_limits(ctx):
    with pytest.raises(pm.PermanovaError) as ei:
        pm.permanova_set_plan(ctx.handle, pm.FORM_GEMM, gemm_drain_kblocks=16)
    assert ei.value.status == pm.EINVAL and "accuracy" in str(ei.value)
    with pytest.raises(pm.PermanovaError):
        pm.permanova_set_plan(ctx.handle, pm.FORM_PERMBLOCK, permblock_variant=3)
    pm.permanova_set_plan(ctx.handle, pm.FORM_AUTO)


def test_autotuned_plan_is_described_and_matches_oracle(ctx):
    """After permanova_autotune the bucket's plan (form and knobs) is the
    autotuned one, and calls in that bucket match the oracle."""
    n, K, P = 1500, 6, 600
    D, rows, w = _case(n, K, P, 9)
    Dd, lab, wd = (torch.from_numpy(D).cuda(), torch.from_numpy(rows.astype(np.uint8)).cuda(),
                   torch.from_numpy(w).cuda())
    form = pm.permanova_autotune(ctx.handle, Dd, n, n, lab, pm.LABEL_U8, K, P, wd)
    desc = pm.permanova_plan_describe(ctx.handle, n, K, P)
    assert desc["source"] == "autotuned" and desc["form"] == pm.FORM_NAMES[form]
    out = ctx.sW(Dd, lab, K, wd)
    pm.permanova_sync(ctx.handle)
    ref = oracle.sW_alg1(D, rows, K, w.astype(np.float64))
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-5)
