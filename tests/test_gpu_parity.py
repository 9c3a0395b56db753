"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Sizes span several 64/128-wide tiles and ragged tails; label types, group
counts, label-row counts and strides cover the cases the kernels branch on.
Tolerance: the stated 1e-5 relative for s_W and pseudo-F; integer-valued
matrices with power-of-two group sizes must match bit for bit; label
generation, exceedance counts and p-values are compared exactly.
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
         pytest.param(pm.FORM_GEMM, id="gemm")]
FORM_VALUES = [pm.FORM_BRUTE, pm.FORM_PERMBLOCK, pm.FORM_GEMM]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pm.build()
    c = pm.Context(0)
    yield c
    c.close()


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _label_tensor(rows, ltype):
    dt = {pm.LABEL_U8: torch.uint8, pm.LABEL_U16: torch.int16, pm.LABEL_I32: torch.int32}[ltype]
    npdt = {pm.LABEL_U8: np.uint8, pm.LABEL_U16: np.uint16, pm.LABEL_I32: np.int32}[ltype]
    a = np.ascontiguousarray(rows.astype(npdt))
    if ltype == pm.LABEL_U16:
        a = a.view(np.int16)
    return torch.from_numpy(a).cuda(), dt


def _run_sW(ctx, D, rows, K, w, form, ltype=pm.LABEL_I32, ld=None):
    n = D.shape[0]
    ld = ld or n
    Dp = np.zeros((n, ld), dtype=np.float32)
    Dp[:, :n] = D
    Dd = _dev(Dp)
    lab, _ = _label_tensor(rows, ltype)
    wd = _dev(np.asarray(w, dtype=np.float32))
    out = torch.empty(rows.shape[0], dtype=torch.float64, device="cuda")
    ctx.set_form(form)
    try:
        pm.permanova_sW(ctx.handle, Dd, n, ld, lab, ltype, K, rows.shape[0], wd, out)
        pm.permanova_sync(ctx.handle)
    finally:
        ctx.set_form(pm.FORM_AUTO)
    return out.cpu().numpy()


def _case(n, K, P, seed, kind="euclid"):
    rng = np.random.default_rng(seed)
    if kind == "euclid":
        X = rng.standard_normal((n, 8))
        D = synth.euclidean_matrix(X)
    else:
        C = synth.dirichlet_compositions(rng.integers(0, K, n), features=40, seed=seed)
        D = synth.braycurtis_matrix(C)
    sizes = synth.largest_remainder_sizes(n, rng.dirichlet(2 * np.ones(K)), min_size=1)
    obs = synth.observed_labels(sizes, seed + 1)
    rows = synth.shuffled_rows(obs, P, seed + 2)
    return D, rows, synth.inv_sizes(obs, K)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("n,K,P", [(2, 1, 1), (63, 2, 3), (130, 3, 129), (257, 5, 40),
                                   (300, 10, 131), (1001, 4, 17),
                                   # several accumulator chunks per band, ragged label-row
                                   # tiles of 128 (K = 2) and 85 (K = 3) rows, 36 rows (K = 7)
                                   (2500, 2, 300), (2500, 3, 200), (3000, 7, 150),
                                   # a large group count (7 label rows x 36)
                                   (700, 36, 50)])
def test_sW_matches_oracle(ctx, form, n, K, P):
    D, rows, w = _case(n, K, P, seed=n * 7 + K)
    ref = oracle.sW_alg1(D, rows, K, w.astype(np.float64))
    got = _run_sW(ctx, D, rows, K, w, form, pm.LABEL_U8)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=1e-12)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("ltype", [pm.LABEL_I32, pm.LABEL_U16, pm.LABEL_U8])
def test_label_types_and_padded_stride(ctx, form, ltype):
    D, rows, w = _case(200, 6, 70, seed=ltype + 11, kind="braycurtis")
    ref = oracle.sW_alg1(D, rows, 6, w.astype(np.float64))
    got = _run_sW(ctx, D, rows, 6, w, form, ltype, ld=203)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=1e-12)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("K,ltype", [(255, pm.LABEL_U8), (256, pm.LABEL_U8), (300, pm.LABEL_U16),
                                     (2048, pm.LABEL_U16), (2049, pm.LABEL_U16)])
def test_many_groups(ctx, form, K, ltype):
    if form == pm.FORM_GEMM and K > 256:
        pytest.skip("GEMM form holds at most 256 groups")
    rng = np.random.default_rng(K)
    n = 700
    D = synth.euclidean_matrix(rng.standard_normal((n, 4)))
    rows = rng.integers(0, K, size=(9, n)).astype(np.int32)
    w = rng.uniform(0.01, 1.0, K).astype(np.float32)
    ref = oracle.sW_alg1(D, rows, K, w.astype(np.float64))
    got = _run_sW(ctx, D, rows, K, w, form, ltype)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=1e-12)


@pytest.mark.parametrize("variant", [0, 1, 2])
@pytest.mark.parametrize("K", [257, 1000, 2048])
def test_permblock_uint16_codes(ctx, variant, K):
    """More than 256 groups: int32 labels become uint16 codes, which the paired
    perm-block kernel (variants 0 and 2, FP16 patterns 0x4000 + L) and the
    FP32 kernel (variant 1) both take; ragged tiles (n = 1,001) and a ragged
    last block of label rows (300 rows)."""
    rng = np.random.default_rng(K + variant)
    n, P = 1001, 300
    D = synth.euclidean_matrix(rng.standard_normal((n, 6)))
    rows = rng.integers(0, K, size=(P, n)).astype(np.int32)
    rows[0, :] = K - 1                       # the largest code in every column of one row
    w = rng.uniform(0.01, 1.0, K).astype(np.float32)
    ref = oracle.sW_alg1(D, rows, K, w.astype(np.float64))
    out = torch.empty(P, dtype=torch.float64, device="cuda")
    pm.permanova_set_plan(ctx.handle, form=pm.FORM_PERMBLOCK, permblock_variant=variant)
    try:
        pm.permanova_sW(ctx.handle, _dev(D), n, n, _dev(rows), pm.LABEL_I32, K, P, _dev(w), out)
        pm.permanova_sync(ctx.handle)
    finally:
        pm.permanova_set_plan(ctx.handle, pm.FORM_AUTO)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=RTOL, atol=1e-12)


@pytest.mark.parametrize("form", FORMS + [pytest.param(pm.FORM_AUTO, id="auto")])
@pytest.mark.parametrize("n,sizes", [(128, [64, 32, 32]), (1001, [512, 256, 128, 64, 41]),
                                     (4096, [2048, 1024, 1024])])
def test_integer_matrix_bit_exact(ctx, form, n, sizes):
    """Integer entries 0..15 with power-of-two weights: every sum of every form
    is exact, so every form equals the FP64 oracle bit for bit.  For the
    tensor-core form the bound is: d^2 <= 255 fits the BF16 hi plane exactly
    (the lo plane is 0), the band scale is a power of two, and the largest FP32
    sum it forms (32 rows x 2,048 columns of one label-row column before the
    FP64 hand-off) stays below 2^24 band units, so no FP32 step rounds."""
    D = synth.integer_matrix(n, 15, 5 + n)
    K = len(sizes)
    obs = synth.observed_labels(sizes, 6 + n)
    rows = synth.shuffled_rows(obs, 33, 7 + n)
    w = np.array([2.0 ** -(k + 3) for k in range(K)], dtype=np.float32)   # exact weights
    ref = oracle.sW_alg1(D, rows, K, w.astype(np.float64))
    got = _run_sW(ctx, D, rows, K, w, form, pm.LABEL_U8)
    assert np.array_equal(got, ref), np.max(np.abs(got - ref) / ref)


@pytest.mark.parametrize("form", FORMS)
def test_lower_triangle_never_read(ctx, form):
    D, rows, w = _case(190, 3, 20, seed=3)
    clean = _run_sW(ctx, D, rows, 3, w, form)
    dirty = _run_sW(ctx, synth.poison_lower(D), rows, 3, w, form)
    assert np.all(np.isfinite(dirty))
    assert np.array_equal(clean, dirty)


@pytest.mark.parametrize("form", FORMS)
def test_deterministic(ctx, form):
    D, rows, w = _case(333, 4, 300, seed=9)
    a = _run_sW(ctx, D, rows, 4, w, form)
    b = _run_sW(ctx, D, rows, 4, w, form)
    assert np.array_equal(a, b)


def test_forms_agree(ctx):
    D, rows, w = _case(500, 4, 200, seed=21)
    res = [_run_sW(ctx, D, rows, 4, w, f) for f in FORM_VALUES]
    for r in res[1:]:
        np.testing.assert_allclose(r, res[0], rtol=RTOL)


def test_single_group_closed_form(ctx):
    n = 517
    X = np.random.default_rng(4).standard_normal((n, 6))
    D = synth.euclidean_matrix(X)
    rows = np.zeros((3, n), dtype=np.int32)
    for form in FORM_VALUES:
        got = _run_sW(ctx, D, rows, 1, [1.0 / n], form)
        st = oracle.sT(D)
        np.testing.assert_allclose(got, st, rtol=RTOL)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("n,K", [(3000, 3), (2051, 1)])
@pytest.mark.parametrize("c", [0.7937, 1.0019550323486328, 2.989486])
def test_constant_matrix_closed_form(ctx, form, n, K, c):
    """Every term equal is the worst case for accumulation order: each FP32
    rounding (and the tensor core's truncating accumulation) errs the same way.
    For d_ij = c off the diagonal, s_W[p] = c^2 sum_g w_g n_g (n_g - 1) / 2,
    evaluated in FP64 from the label counts (s_W as Algorithm 1 defines it, Sec. 2).
    c = 1.0019550323486328 squares to 1 + 2^-8 + 2^-17, the worst value for a
    split of d^2 into two BF16 halves; c = 2.989486 was the worst constant for
    the tensor-core accumulation in a sweep of 60 values."""
    c = np.float32(c)
    D = np.full((n, n), c, dtype=np.float32)
    np.fill_diagonal(D, 0.0)
    rng = np.random.default_rng(77)
    rows = np.stack([rng.permutation(np.arange(n) % K) for _ in range(40)]).astype(np.int32)
    sizes = np.bincount(rows[0], minlength=K)
    w = (1.0 / sizes).astype(np.float32)
    want = float(c) ** 2 * sum(float(w[g]) * sizes[g] * (sizes[g] - 1) / 2 for g in range(K))
    got = _run_sW(ctx, D, rows, K, w, form)
    np.testing.assert_allclose(got, np.full(rows.shape[0], want), rtol=RTOL)


@pytest.mark.parametrize("form", FORMS)
def test_tight_clusters_far_apart(ctx, form):
    """Three clusters: every within-cluster distance is eps = 3.1e-5, the
    distances between clusters lie in [5, 12].  Each band's d^2 then spans
    ~2^37, and s_W of the observed labels (row 0) consists only of the equal
    tiny terms, so any rounding of them errs the same way for every pair:
    s_W = eps^2 sum_g w_g n_g (n_g - 1) / 2 exactly (Algorithm 1's sum, Sec. 2).
    The permuted rows are checked against the oracle."""
    rng = np.random.default_rng(31)
    n, K = 1500, 3
    lab = np.arange(n) % K
    eps = np.float32(3.1e-5)
    B = rng.uniform(5.0, 12.0, (n, n))
    D = np.triu(B, 1)
    D = (D + D.T).astype(np.float32)
    D[lab[:, None] == lab[None, :]] = eps
    np.fill_diagonal(D, 0.0)
    rows = np.stack([lab] + [rng.permutation(lab) for _ in range(39)]).astype(np.int32)
    w = synth.inv_sizes(lab, K)
    sizes = np.bincount(lab, minlength=K)
    want0 = float(eps) ** 2 * sum(float(np.float32(w[g])) * sizes[g] * (sizes[g] - 1) / 2 for g in range(K))
    ref = oracle.sW_alg1(D, rows[1:], K, np.asarray(w, dtype=np.float64))
    got = _run_sW(ctx, D, rows, K, w, form)
    np.testing.assert_allclose(got[0], want0, rtol=RTOL)
    np.testing.assert_allclose(got[1:], ref, rtol=RTOL)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("scale", [1e-15, 1e15])
def test_extreme_scales(ctx, form, scale):
    """D scaled by 1e-15 or 1e15 (d^2 from 1e-30 to 1e30, normal FP32): s_W
    scales by scale^2 exactly (Algorithm 1's sum is homogeneous of degree 2 in D)."""
    D, rows, w = _case(900, 4, 40, seed=41)
    ref = oracle.sW_alg1(D, rows, 4, np.asarray(w, dtype=np.float64))
    got = _run_sW(ctx, (D.astype(np.float64) * scale).astype(np.float32), rows, 4, w, form)
    np.testing.assert_allclose(got / scale ** 2, ref, rtol=RTOL)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("fill", [3e30, float("nan")])
def test_lower_triangle_never_read(ctx, form, fill):
    """Entries on and below the diagonal take no part (Algorithm 1 sums i < j
    only): huge or NaN values there change nothing, not even the tensor-core
    form's per-band scale, which comes from each band's largest d^2."""
    D, rows, w = _case(700, 3, 40, seed=43)
    Dg = D.copy()
    Dg[np.tril_indices(D.shape[0])] = fill
    ref = oracle.sW_alg1(D, rows, 3, np.asarray(w, dtype=np.float64))
    got = _run_sW(ctx, Dg, rows, 3, w, form)
    np.testing.assert_allclose(got, ref, rtol=RTOL)


@pytest.mark.parametrize("form", FORMS)
def test_all_zero_matrix(ctx, form):
    """d = 0 everywhere gives s_W = 0 exactly (every band's largest d^2 is 0:
    the tensor-core form's scale falls back to 1)."""
    n = 600
    rows = np.stack([np.random.default_rng(9).permutation(np.arange(n) % 4) for _ in range(33)])
    got = _run_sW(ctx, np.zeros((n, n), dtype=np.float32), rows.astype(np.int32), 4,
                  [0.25, 0.25, 0.25, 0.25], form)
    assert np.all(got == 0.0)


def test_permutations_bit_exact_with_oracle(ctx):
    obs = synth.observed_labels([37, 20, 13, 3], 12)
    n = obs.size
    for ltype, tdt in ((pm.LABEL_I32, torch.int32), (pm.LABEL_U8, torch.uint8),
                       (pm.LABEL_U16, torch.int16)):
        out = torch.empty((51, n), dtype=tdt, device="cuda")
        pm.permanova_permutations(ctx.handle, _dev(obs), n, 4, 50, 9013, out, ltype)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.int64) & (0xFFFF if ltype == pm.LABEL_U16 else -1)
        ref = oracle.permutations(obs, 50, 9013)
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 7, 8, 9, 16, 17, 1000, 5003, 50000, 60000])
def test_permutations_bit_exact_across_row_lengths(ctx, n):
    """Short and long rows (40 of them: a warp per row in shared memory, or
    in place in HBM when not one int32 row fits, n = 60,000): every row
    equals the oracle's Fisher-Yates shuffle.  At
    n >= 50,000 some draws need Lemire's rejection check (about 0.3 draws per
    row at 50,000, 0.4 at 60,000), which the shuffle takes one at a time."""
    K = 2 if n < 8 else 5
    obs = synth.observed_labels([n // K] * (K - 1) + [n - (K - 1) * (n // K)], 7)
    for ltype, tdt in ((pm.LABEL_U8, torch.uint8), (pm.LABEL_I32, torch.int32)):
        out = torch.empty((41, n), dtype=tdt, device="cuda")
        pm.permanova_permutations(ctx.handle, _dev(obs), n, K, 40, 77 + n, out, ltype)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().astype(np.int64), oracle.permutations(obs, 40, 77 + n))


@pytest.mark.parametrize("n,P,seed", [(1000, 4000, 5), (3000, 9999, 9), (4000, 9999, 10), (30000, 999, 6),
                                       (60000, 4000, 8), (100000, 80, 424242)])
def test_permutations_every_shuffle_path(ctx, n, P, seed):
    """Each way the shuffles run gives the oracle's rows bit for bit: in
    shared memory with one row to a warp (n = 1,000, 4,000 rows: 27 rows to a
    block; n = 30,000: 7 uint8 rows or 1 int32 row; n = 100,000 uint8: 1
    row), two rows to a warp (n = 4,000, 9,999 uint8 rows: 33 to a block) and
    four (n = 3,000, 9,999 uint8 rows: 66 to a block); in place in HBM (n =
    60,000 with 4,000 rows, more than eight times what shared memory holds at
    once; n = 100,000 int32, where not one row fits).  In the last case row
    80's stream has a rejection at draw 5,503, the last of a 128-draw refill
    of a row alone in its warp, whose second draw lies past the refill (found
    by a search over rows; the first draw is checked here)."""
    obs = synth.observed_labels([n // 3, n // 3, n - 2 * (n // 3)], seed)
    if seed == 424242:
        x = oracle.philox4x32_10([5503 // 4, 0, 80, 0], [seed & 0xFFFFFFFF, seed >> 32])[5503 % 4]
        rng = 94497                          # step i = 94,496 draws from [0, i]
        low = (int(x) * rng) & 0xFFFFFFFF
        assert low < (2**32 - rng) % rng     # Lemire rejects this draw
    ref = oracle.permutations(obs, P, seed)
    for ltype, tdt in ((pm.LABEL_U8, torch.uint8), (pm.LABEL_I32, torch.int32)):
        out = torch.empty((P + 1, n), dtype=tdt, device="cuda")
        pm.permanova_permutations(ctx.handle, _dev(obs), n, 3, P, seed, out, ltype)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().astype(np.int64), ref)


@pytest.mark.parametrize("n,K,P,seed", [(60, 2, 99, 1), (257, 3, 999, 2), (1000, 3, 999, 3)])
def test_permanova_test_matches_oracle(ctx, n, K, P, seed):
    cfg = synth.recipe("euclid-1k", n=n, P=P)
    X = synth.recipe_points(cfg)
    D = synth.euclidean_matrix(X)
    obs = cfg["labels"] if K == 3 else synth.observed_labels([n // 2, n - n // 2], seed)
    ref = oracle.permanova_test(D, obs, K, P, seed)
    out_sW = torch.empty(P + 1, dtype=torch.float64, device="cuda")
    res = pm.permanova_test(ctx.handle, _dev(D), n, n, _dev(obs), K, P, seed, out_sW)
    sW = out_sW.cpu().numpy()
    np.testing.assert_allclose(sW, ref["s_W"], rtol=RTOL)
    assert abs(res["s_T"] - ref["s_T"]) <= RTOL * ref["s_T"]
    # F = c (s_T - s_W) / s_W: a relative error e in s_W moves F by kappa * e with
    # kappa = s_T / (s_T - s_W) (>> 1 when groups barely differ), so F is held to
    # the s_W tolerance times its condition number.
    kappa = ref["s_T"] / (ref["s_T"] - ref["s_W"][0])
    assert abs(res["F_obs"] - ref["F"][0]) <= RTOL * max(1.0, kappa) * abs(ref["F"][0])
    # exceedance counts are exact outside the ambiguity band |s_W - s_W_obs| <= 1e-5 s_W_obs
    band = np.abs(ref["s_W"][1:] - ref["s_W"][0]) <= RTOL * ref["s_W"][0]
    if not band.any():
        assert res["n_ge"] == ref["n_ge"]
        assert res["p_value"] == ref["p_value"]
    assert res["n_perms"] == P


@pytest.mark.parametrize("form", FORMS[:2] + [pytest.param(pm.FORM_AUTO, id="auto")])
def test_permanova_test_many_groups(ctx, form):
    """The permutation test with more than 256 groups: the device permutations
    are uint16 codes and the s_W pass takes them (brute force, the paired
    perm-block kernel, the planner's choice); s_W of every row, s_T and the
    count against the oracle."""
    n, K, P, seed = 2003, 300, 199, 31
    rng = np.random.default_rng(seed)
    D = synth.euclidean_matrix(rng.standard_normal((n, 5)))
    obs = np.concatenate([np.arange(K), rng.integers(0, K, n - K)]).astype(np.int32)
    rng.shuffle(obs)
    ref = oracle.permanova_test(D, obs, K, P, seed)
    out_sW = torch.empty(P + 1, dtype=torch.float64, device="cuda")
    ctx.set_form(form)
    try:
        res = pm.permanova_test(ctx.handle, _dev(D), n, n, _dev(obs), K, P, seed, out_sW)
    finally:
        ctx.set_form(pm.FORM_AUTO)
    np.testing.assert_allclose(out_sW.cpu().numpy(), ref["s_W"], rtol=RTOL)
    assert abs(res["s_T"] - ref["s_T"]) <= RTOL * ref["s_T"]
    band = np.abs(ref["s_W"][1:] - ref["s_W"][0]) <= RTOL * ref["s_W"][0]
    if not band.any():
        assert res["n_ge"] == ref["n_ge"]
        assert res["p_value"] == ref["p_value"]


@pytest.mark.parametrize("form", FORMS + [pytest.param(pm.FORM_AUTO, id="auto")])
@pytest.mark.parametrize("n,P", [(3, 1), (4, 2), (5, 7)])
def test_permanova_test_smallest_cases(ctx, form, n, P):
    """The smallest tests the method allows (n = 3 objects in two groups, one
    permutation; then 4 and 5 objects): s_W of every row and s_T against the
    oracle, and the exceedance count within the bounds the 1e-5 band around
    the observed s_W allows."""
    rng = np.random.default_rng(n * 10 + P)
    A = rng.integers(1, 9, (n, n)).astype(np.float32)
    D = np.triu(A, 1)
    D = D + D.T
    obs = np.array([0, 1] * n, dtype=np.int32)[:n]
    ref = oracle.permanova_test(D, obs, 2, P, 77)
    out_sW = torch.empty(P + 1, dtype=torch.float64, device="cuda")
    ctx.set_form(form)
    try:
        res = pm.permanova_test(ctx.handle, _dev(D), n, n, _dev(obs), 2, P, 77, out_sW)
    finally:
        ctx.set_form(pm.FORM_AUTO)
    np.testing.assert_allclose(out_sW.cpu().numpy(), ref["s_W"], rtol=RTOL)
    assert abs(res["s_T"] - ref["s_T"]) <= 1e-12 * ref["s_T"]
    obs_sW, perm_sW = ref["s_W"][0], ref["s_W"][1:]
    lo = int(np.sum(perm_sW < obs_sW * (1 - RTOL)))
    hi = int(np.sum(perm_sW <= obs_sW * (1 + RTOL)))
    assert lo <= res["n_ge"] <= hi
    assert res["n_perms"] == P


def test_invalid_label_reported(ctx):
    D, rows, w = _case(100, 3, 5, seed=1)
    rows = rows.copy()
    rows[2, 17] = 3
    for form in FORM_VALUES:
        with pytest.raises(pm.PermanovaError) as ei:
            _run_sW(ctx, D, rows, 3, w, form)
        assert ei.value.status == pm.EINVAL
    # the context stays usable
    ok = _run_sW(ctx, D, rows % 3, 3, w, pm.FORM_BRUTE)
    assert np.all(np.isfinite(ok))


def test_argument_errors(ctx):
    Dd = torch.zeros((10, 10), device="cuda")
    lab = torch.zeros((1, 10), dtype=torch.uint8, device="cuda")
    w = torch.ones(2, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    h = ctx.handle
    cases = [
        dict(n=1, ld=10, K=2, P=1, lt=pm.LABEL_U8),
        dict(n=10, ld=9, K=2, P=1, lt=pm.LABEL_U8),
        dict(n=10, ld=10, K=0, P=1, lt=pm.LABEL_U8),
        dict(n=10, ld=10, K=2, P=0, lt=pm.LABEL_U8),
        dict(n=10, ld=10, K=257, P=1, lt=pm.LABEL_U8),
        dict(n=10, ld=10, K=2, P=1, lt=7),
    ]
    for c in cases:
        with pytest.raises(pm.PermanovaError) as ei:
            pm.permanova_sW(h, Dd, c["n"], c["ld"], lab, c["lt"], c["K"], c["P"], w, out)
        assert ei.value.status == pm.EINVAL
    with pytest.raises(pm.PermanovaError) as ei:
        pm.permanova_sW(h, None, 10, 10, lab, pm.LABEL_U8, 2, 1, w, out)
    assert ei.value.status == pm.EINVAL
    g = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(pm.PermanovaError) as ei:   # K < 2
        pm.permanova_test(h, Dd, 10, 10, g, 1, 10, 1)
    assert ei.value.status == pm.EINVAL
    with pytest.raises(pm.PermanovaError) as ei:   # empty group 1
        pm.permanova_test(h, Dd, 10, 10, g, 2, 10, 1)
    assert ei.value.status == pm.EINVAL


def test_budget_enforced():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    small = pm.Context(0, hbm_budget_bytes=4096)
    try:
        D, rows, w = _case(400, 3, 300, seed=2)
        with pytest.raises(pm.PermanovaError) as ei:
            _run_sW(small, D, rows, 3, w, pm.FORM_PERMBLOCK)
        assert ei.value.status == pm.ENOMEM
    finally:
        small.close()


def test_gemm_rejects_too_many_groups(ctx):
    D, rows, w = _case(100, 3, 5, seed=1)
    with pytest.raises(pm.PermanovaError) as ei:
        _run_sW(ctx, D, rows, 300, np.ones(300, np.float32), pm.FORM_GEMM, pm.LABEL_U16)
    assert ei.value.status == pm.EUNSUPPORTED


def test_host_entry_point(ctx):
    D, rows, w = _case(321, 4, 50, seed=31)
    ref = oracle.sW_alg1(D, rows, 4, w.astype(np.float64))
    out = np.zeros(50, dtype=np.float64)
    lab = np.ascontiguousarray(rows.astype(np.uint8))
    pm.permanova_sW_host(ctx.handle, np.ascontiguousarray(D), 321, 321, lab, pm.LABEL_U8, 4, 50,
                         np.ascontiguousarray(w), out)
    np.testing.assert_allclose(out, ref, rtol=RTOL)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("n,ld", [(1000, 1003), (2177, 2177)])
def test_host_entry_segments(ctx, form, n, ld):
    """The host entry point copies D with flat copies (each band's host range
    with the tensor-core form, which runs band segments as they land through
    three staging slots; the whole matrix otherwise) and never reads the
    lower triangle: results equal the device entry point's bit for bit (on a
    device copy with the caller's row stride: the brute-force kernel's
    summation order depends on whether rows are 16-byte aligned) and the
    oracle's within tolerance."""
    K, P = 5, 70
    D, rows, w = _case(n, K, P, seed=37)
    Dp = np.full((n, ld), np.nan, dtype=np.float32)
    Dp[:, :n] = D
    Dp[np.tril_indices(n)] = np.nan
    lab = np.ascontiguousarray(rows.astype(np.uint8))
    out = np.zeros(P, dtype=np.float64)
    ctx.set_form(form)
    try:
        pm.permanova_sW_host(ctx.handle, Dp, n, ld, lab, pm.LABEL_U8, K, P,
                             np.ascontiguousarray(w, dtype=np.float32), out)
    finally:
        ctx.set_form(pm.FORM_AUTO)
    dev = _run_sW(ctx, D, rows, K, w, form, pm.LABEL_U8, ld=ld)
    np.testing.assert_array_equal(out, dev)
    idx = np.arange(0, P, 7)
    ref = oracle.sW_alg1(D, rows[idx], K, w.astype(np.float64))
    np.testing.assert_allclose(out[idx], ref, rtol=RTOL)


def test_host_entry_profile(ctx):
    """With profiling on, the host entry point records one call, the bytes it
    copied (each band's flat host range, the labels and the weights) and an
    ordered device timeline: first segment <= last segment <= end, and per
    segment the time it landed and the time its kernel had run."""
    n, ld, K, P = 1000, 1003, 5, 70
    D, rows, w = _case(n, K, P, seed=41)
    Dp = np.zeros((n, ld), dtype=np.float32)
    Dp[:, :n] = D
    lab = np.ascontiguousarray(rows.astype(np.uint8))
    out = np.zeros(P, dtype=np.float64)
    ctx.set_form(pm.FORM_GEMM)
    try:
        pm.permanova_profile_enable(ctx.handle, True)
        pm.permanova_sW_host(ctx.handle, Dp, n, ld, lab, pm.LABEL_U8, K, P,
                             np.ascontiguousarray(w, dtype=np.float32), out)
        prof = pm.permanova_profile_read(ctx.handle)
    finally:
        pm.permanova_profile_enable(ctx.handle, False)
        ctx.set_form(pm.FORM_AUTO)
    # each band's flat host range, from (128 I, 128 I) to the end of its last
    # row, or for a band whose rows span under half the width its trapezoid
    bands = sum((min(128, n - r0) * (n - r0) if 2 * (n - r0) < n
                 else (min(128, n - r0) - 1) * ld + n - r0) * 4 for r0 in range(0, n, 128))
    assert prof["host_calls"] == 1
    assert prof["host_h2d_bytes"] == bands + n * P + 4 * K
    assert 0.0 < prof["host_first_segment_ms"] <= prof["host_copy_ms"] <= prof["host_total_ms"]
    # per segment (8 bands, one segment each): landed in copy order, each
    # segment's kernel after its copy and before the end of the call
    landed, done = prof["host_seg_landed_ms"], prof["host_seg_done_ms"]
    assert prof["host_segments"] == len(landed) == len(done) == 8
    assert landed == sorted(landed)
    assert all(0.0 < a <= b <= prof["host_total_ms"] for a, b in zip(landed, done))
    assert landed[0] <= prof["host_first_segment_ms"] and landed[-1] <= prof["host_copy_ms"]
    ref = oracle.sW_alg1(D, rows, K, w.astype(np.float64))
    np.testing.assert_allclose(out, ref, rtol=RTOL)
