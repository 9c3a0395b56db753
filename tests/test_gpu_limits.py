"""Parity at the limits of the sizes the method is run at (Sec. 2: matrices of
1k^2 to 100k^2 elements, 1k to 1M permutations).

* One s_W call whose label rows hold more than 2^32 labels (rows * n > 2^32):
  every label, weight and partial offset must be 64-bit.  Rows on both sides
  of the 2^32 boundary, and the last rows, are compared with the FP64 oracle
  (Algorithm 1) in every kernel form.
* The permutation test at a million permutations (999,999 plus the observed
  row), exact: an integer matrix (entries 0..15) with two groups of 32, so
  every sum is exact on both sides, and s_W of all 10^6 rows, s_T, the
  exceedance count (with its exact ties: "greater or equal" counts them) and
  the p-value must match the oracle bit for bit in every form.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2505_04556_gb300 as pm  # noqa: E402

RTOL = 1e-5
FORMS = [pytest.param(pm.FORM_BRUTE, id="brute"), pytest.param(pm.FORM_PERMBLOCK, id="permblock"),
         pytest.param(pm.FORM_GEMM, id="gemm"), pytest.param(pm.FORM_AUTO, id="auto")]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pm.build()
    c = pm.Context(0)
    yield c
    c.close()


# ---------------------------------------------------------------------------
# more than 2^32 labels in one call
# ---------------------------------------------------------------------------
N_BIG = 2100
ROW_2_32 = (1 << 32) // N_BIG            # the label row that straddles flat index 2^32
P_BIG = ROW_2_32 + 200                   # rows * n exceeds 2^32 by 200 rows


@pytest.fixture(scope="module")
def big_rows(ctx):
    rng = np.random.default_rng(4242)
    X = rng.standard_normal((N_BIG, 8))
    D = synth.euclidean_matrix(X)
    sizes = synth.largest_remainder_sizes(N_BIG, [0.5, 0.3, 0.2], min_size=1)
    obs = synth.observed_labels(sizes, 4243)
    lab = synth.device_label_rows(obs, P_BIG, 4244, device="cuda", dtype=torch.uint8)
    assert lab.numel() > (1 << 32)
    idx = np.array([0, 1, 2, 777, 1_000_003, ROW_2_32 - 1, ROW_2_32, ROW_2_32 + 1, ROW_2_32 + 2,
                    P_BIG - 2, P_BIG - 1])
    assert ROW_2_32 * N_BIG < (1 << 32) < (ROW_2_32 + 1) * N_BIG
    rows = lab[torch.from_numpy(idx).cuda()].cpu().numpy().astype(np.int32)
    w = synth.inv_sizes(obs, 3)
    ref = oracle.sW_alg1(D, rows, 3, w.astype(np.float64))
    yield {"D": torch.from_numpy(D).cuda(), "lab": lab, "w": torch.from_numpy(w).cuda(), "idx": idx,
           "ref": ref}
    del lab
    torch.cuda.empty_cache()


@pytest.mark.parametrize("form", FORMS)
def test_label_index_beyond_32_bits(ctx, big_rows, form):
    b = big_rows
    out = torch.full((P_BIG,), float("nan"), dtype=torch.float64, device="cuda")
    ctx.set_form(form)
    try:
        pm.permanova_sW(ctx.handle, b["D"], N_BIG, N_BIG, b["lab"], pm.LABEL_U8, 3, P_BIG, b["w"], out)
        pm.permanova_sync(ctx.handle)
    finally:
        ctx.set_form(pm.FORM_AUTO)
        pm.permanova_release_scratch(ctx.handle)
    assert bool(torch.isfinite(out).all())
    got = out[torch.from_numpy(b["idx"]).cuda()].cpu().numpy()
    np.testing.assert_allclose(got, b["ref"], rtol=RTOL)


# ---------------------------------------------------------------------------
# the permutation test at a million permutations, exact
# ---------------------------------------------------------------------------
N_EXACT, P_MILLION, SEED = 64, 999_999, 2024


@pytest.fixture(scope="module")
def million(ctx):
    rng = np.random.default_rng(11)
    A = rng.integers(0, 16, (N_EXACT, N_EXACT)).astype(np.float32)
    D = np.triu(A, 1)
    D = D + D.T
    obs = synth.observed_labels([32, 32], 3)
    ref = oracle.permanova_test(D, obs, 2, P_MILLION, SEED)
    # exact ties with the observed statistic exist (integer sums), so the tie
    # rule is exercised
    assert int((ref["s_W"][1:] == ref["s_W"][0]).sum()) > 0
    return {"D": torch.from_numpy(D).cuda(), "obs": torch.from_numpy(obs.astype(np.int32)).cuda(),
            "ref": ref}


@pytest.mark.parametrize("form", FORMS)
def test_permutation_test_million_permutations_exact(ctx, million, form):
    m, ref = million, million["ref"]
    out = torch.empty(P_MILLION + 1, dtype=torch.float64, device="cuda")
    ctx.set_form(form)
    try:
        res = pm.permanova_test(ctx.handle, m["D"], N_EXACT, N_EXACT, m["obs"], 2, P_MILLION, SEED, out)
    finally:
        ctx.set_form(pm.FORM_AUTO)
    assert np.array_equal(out.cpu().numpy(), ref["s_W"])
    assert res["s_T"] == ref["s_T"]
    assert res["n_ge"] == ref["n_ge"]
    assert res["p_value"] == ref["p_value"]
    assert res["n_perms"] == P_MILLION
    assert abs(res["F_obs"] - ref["F"][0]) <= 1e-12 * abs(ref["F"][0])
