"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each test ties an oracle function to something it cannot produce by itself:
closed forms (single group, constant distances, Huygens' identity for
Euclidean distances, the one-way MANOVA trace statistic), exact rational brute
force on tiny inputs, invariances, and the cuRAND host library's own
Philox4x32-10 stream.  Runs on the CPU only.
"""
import ctypes
import ctypes.util
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


def _random_case(n, K, seed, integer=False):
    rng = np.random.default_rng(seed)
    if integer:
        D = synth.integer_matrix(n, 15, seed)
    else:
        X = rng.standard_normal((n, 3))
        D = synth.euclidean_matrix(X)
    lab = rng.integers(0, K, size=n).astype(np.int32)
    lab[:K] = np.arange(K)  # every group non-empty
    return D, lab


def _exact_sW(D, lab, w_frac):
    """Exact rational value of the pair sum: group by group, every unordered
    pair {i, j} of members counted once, d^2 times the group weight."""
    n = len(lab)
    members = {}
    for i in range(n):
        members.setdefault(int(lab[i]), []).append(i)
    total = Fraction(0)
    for g, idx in members.items():
        for a, b in itertools.combinations(idx, 2):
            i, j = min(a, b), max(a, b)
            v = Fraction(float(D[i, j]))
            total += v * v * w_frac[g]
    return total


@pytest.mark.parametrize("n,K,seed", [(2, 1, 1), (5, 2, 2), (9, 3, 3), (12, 4, 4), (12, 12, 5)])
def test_alg1_equals_exact_groupwise_pair_sum(n, K, seed):
    D, lab = _random_case(n, K, seed)
    rng = np.random.default_rng(seed + 100)
    w = rng.uniform(0.1, 2.0, size=K)
    got = oracle.sW_alg1(D, lab[None, :], K, w)[0]
    exact = _exact_sW(D, lab, [Fraction(float(x)) for x in w])
    assert abs(got - float(exact)) <= 1e-13 * max(1.0, abs(float(exact)))


@pytest.mark.parametrize("n,K,P,seed", [(40, 1, 3, 1), (57, 3, 5, 2), (130, 10, 4, 3)])
def test_alg1_equals_one_hot_contraction(n, K, P, seed):
    """The tensor-core form's algebra, written out in FP64 with numpy: with M
    the strict upper triangle of D o D and X_p the one-hot (n x K) indicator
    of row p, Z_p = M X_p and s_W[p] = sum_i w[g_p(i)] Z_p[i, g_p(i)]."""
    D, lab = _random_case(n, K, seed)
    rng = np.random.default_rng(seed + 7)
    rows = np.stack([rng.permutation(lab) for _ in range(P)]).astype(np.int32)
    w = rng.uniform(0.1, 2.0, size=K)
    M = np.triu(D.astype(np.float64) ** 2, k=1)
    ref = []
    for g in rows:
        X = np.zeros((n, K))
        X[np.arange(n), g] = 1.0
        Z = M @ X
        ref.append(float(np.sum(w[g] * Z[np.arange(n), g])))
    got = oracle.sW_alg1(D, rows, K, w)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)


def _bf16_rne(x):
    """float32 -> the nearest bfloat16 (ties to even), returned as float32:
    keep the top 16 bits of the rounded bit pattern."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _band_scale(x_max):
    """Power of two S with S * x_max in [2^23, 2^24) (S = 1 for a zero maximum)."""
    if x_max == 0.0:
        return 1.0
    e = int(np.floor(np.log2(np.float64(x_max))))
    return 2.0 ** min(100, max(-100, 23 - e))


def _band_is_wide(x):
    """The band's smallest nonzero d^2 below 2^-28 of its largest: too wide for
    an FP16 lo plane."""
    nz = x[x > 0]
    return nz.size > 0 and float(nz.min()) < float(x.max()) * 2.0 ** -28


def _split(x, S, wide=False):
    """The GEMM form's split of d^2 = x (FP32) in a band with scale S:
    y = S x, h = bf16(y), hi plane = bf16(2^7 h), lo plane = fp16(y - h), or
    bf16(2^7 (y - h)) in a band too wide for FP16.  Returns y, h and the lo
    plane's value (divided by 2^7 for the BF16 plane)."""
    y = (np.float32(S) * x).astype(np.float32)
    h = _bf16_rne(y)
    hi = _bf16_rne((h * np.float32(128.0)).astype(np.float32))
    assert np.array_equal(hi.astype(np.float64), 128.0 * h.astype(np.float64))
    r = (y - h).astype(np.float32)
    if wide:
        lo = _bf16_rne((r * np.float32(128.0)).astype(np.float32)).astype(np.float64) / 128.0
    else:
        lo16 = r.astype(np.float16)
        assert np.all(np.isfinite(lo16)) and np.max(np.abs(lo16.astype(np.float64))) <= 2.0 ** 15
        lo = lo16.astype(np.float64)
    return y, h, lo


def test_gemm_split_error_bound():
    """hi (BF16) + lo (FP16) carry 19 significant bits of S x: relative error
    <= 2^-20 for every term of a band whose smallest nonzero d^2 is at least
    2^-28 of its largest (and the lo plane never overflows FP16); a wider band
    uses a BF16 lo plane, 16 bits, <= 2^-17 at any magnitude.  Checked on
    log-uniform magnitudes, random distances, the value 1 + 2^-8 + 2^-17 (the
    worst case of a BF16 + BF16 split), and bands spanning 2^40 and 2^120."""
    rng = np.random.default_rng(11)
    narrow = [np.exp(rng.uniform(-9.0, 9.0, 100000)),
              rng.uniform(0.05, 3.0, 100000) ** 2,
              np.exp(rng.uniform(-8.0, 8.0, 100000)) * 1e6,
              np.full(1000, 1 + 2.0 ** -8 + 2.0 ** -17)]
    wide = [np.exp(rng.uniform(-14.0, 14.0, 100000)),
            np.exp(rng.uniform(-40.0, 40.0, 100000))]
    worst = {False: 0.0, True: 0.0}
    for bands, is_wide in ((narrow, False), (wide, True)):
        for v in bands:
            x = v.astype(np.float32)
            assert _band_is_wide(x) == is_wide
            S = _band_scale(float(x.max()))
            assert 2.0 ** 23 <= S * float(x.max()) < 2.0 ** 24
            y, h, lo = _split(x, S, is_wide)
            rel = np.abs(h.astype(np.float64) + lo - y.astype(np.float64)) / y.astype(np.float64)
            bound = 2.0 ** -17 if is_wide else 2.0 ** -20
            assert np.all(rel <= bound)
            worst[is_wide] = max(worst[is_wide], float(rel.max()))
    # the bounds are nearly reached: 19 and 16 bits, not more
    assert worst[False] > 2.0 ** -22 and worst[True] > 2.0 ** -19
    # the old BF16 + BF16 worst case is now far inside the narrow bound
    x = np.float32(1 + 2.0 ** -8 + 2.0 ** -17)
    lo16 = _bf16_rne((x - _bf16_rne(x)).astype(np.float32))
    assert abs(float(_bf16_rne(x)) + float(lo16) - float(x)) / float(x) > 2.0 ** -18


def test_alg1_exact_on_integer_matrix_power_of_two_groups():
    # integer d in [0, 15], groups of 8/4/4 -> every partial sum is exact in FP64
    n = 16
    D = synth.integer_matrix(n, 15, 7)
    lab = np.array([0] * 8 + [1] * 4 + [2] * 4, dtype=np.int32)
    np.random.default_rng(8).shuffle(lab)
    w = synth.inv_sizes(lab, 3)
    got = oracle.sW_alg1(D, lab[None, :], 3, w)[0]
    exact = _exact_sW(D, lab, [Fraction(1, 8), Fraction(1, 4), Fraction(1, 4)])
    assert Fraction(got) == exact


def test_alg2_f32_close_to_fp64():
    """The FP32 Algorithm 2 (the paper's CPU method, timed for context only)
    agrees with the FP64 oracle to FP32 summation accuracy."""
    D, lab = _random_case(300, 4, 23)
    rows = synth.shuffled_rows(lab, 8, 24)
    w = synth.inv_sizes(lab, 4)
    ref = oracle.sW_alg1(D, rows, 4, w)
    got = oracle.sW_alg2_f32(D, rows, 4, w, 64)
    np.testing.assert_allclose(got.astype(np.float64), ref, rtol=1e-4)
    assert not np.array_equal(got.astype(np.float64), ref)   # it is FP32, not FP64


@pytest.mark.parametrize("tile", [1, 3, 7, 16, 64, 97])
def test_alg1_equals_alg2(tile):
    D, lab = _random_case(97, 5, 11)
    rows = synth.shuffled_rows(lab, 6, 12)
    w = synth.inv_sizes(lab, 5)
    a1 = oracle.sW_alg1(D, rows, 5, w)
    a2 = oracle.sW_alg2(D, rows, 5, w, tile)
    np.testing.assert_allclose(a2, a1, rtol=1e-12, atol=0)


def test_single_group_closed_form():
    # K = 1 and w = 1/n: s_W = s_T = (1/n) sum_{i<j} d_ij^2
    n = 40
    X = np.random.default_rng(3).standard_normal((n, 5))
    D = synth.euclidean_matrix(X)
    lab = np.zeros(n, dtype=np.int32)
    got = oracle.sW_alg1(D, lab[None, :], 1, np.array([1.0 / n]))[0]
    iu = np.triu_indices(n, 1)
    closed = float(np.sum(D[iu].astype(np.float64) ** 2)) / n
    assert abs(got - closed) <= 1e-13 * closed
    assert abs(oracle.sT(D) - closed) <= 1e-13 * closed


@pytest.mark.parametrize("sizes", [[4, 4, 8], [3, 5, 7, 1], [10, 10]])
def test_constant_matrix_closed_form(sizes):
    # d_ij = c off the diagonal: s_W = c^2 (n - K) / 2 for every labelling
    c = 3.0
    n = sum(sizes)
    K = len(sizes)
    D = np.full((n, n), c, dtype=np.float32)
    np.fill_diagonal(D, 0)
    lab = np.repeat(np.arange(K, dtype=np.int32), sizes)
    rows = synth.shuffled_rows(lab, 5, 21)
    w = 1.0 / np.asarray(sizes, dtype=np.float64)
    got = oracle.sW_alg1(D, rows, K, w)
    np.testing.assert_allclose(got, c * c * (n - K) / 2.0, rtol=1e-14)
    assert abs(oracle.sT(D) - c * c * (n - 1) / 2.0) < 1e-12


def test_euclidean_huygens_identity():
    # sum_{i<j in g} |x_i - x_j|^2 / n_g = sum_{i in g} |x_i - mu_g|^2
    cfg = synth.recipe("euclid-1k", n=300, P=8)
    X = synth.recipe_points(cfg)
    D = synth.euclidean_matrix(X)
    rows = synth.shuffled_rows(cfg["labels"], 8, 5)
    got = oracle.sW_alg1(D, rows, cfg["K"], cfg["w"].astype(np.float64))
    for r in range(rows.shape[0]):
        closed = 0.0
        for g in range(cfg["K"]):
            Xg = X[rows[r] == g]
            closed += float(np.sum((Xg - Xg.mean(axis=0)) ** 2))
        # D is stored in fp32 and w = 1/n_g in fp32: agreement to ~1e-6
        assert abs(got[r] - closed) <= 2e-6 * closed


def test_relabel_invariance_bit_identical():
    D, lab = _random_case(60, 4, 31)
    w = synth.inv_sizes(lab, 4).astype(np.float64)
    perm = np.array([2, 0, 3, 1])
    lab2 = perm[lab].astype(np.int32)
    w2 = np.empty_like(w)
    w2[perm] = w
    a = oracle.sW_alg1(D, lab[None, :], 4, w)[0]
    b = oracle.sW_alg1(D, lab2[None, :], 4, w2)[0]
    assert a == b


def test_object_permutation_invariance():
    D, lab = _random_case(50, 3, 41)
    w = synth.inv_sizes(lab, 3).astype(np.float64)
    sigma = np.random.default_rng(42).permutation(50)
    D2 = D[np.ix_(sigma, sigma)]
    a = oracle.sW_alg1(D, lab[None, :], 3, w)[0]
    b = oracle.sW_alg1(D2, lab[sigma][None, :], 3, w)[0]
    assert abs(a - b) <= 1e-12 * a


def test_lower_triangle_and_diagonal_never_read():
    D, lab = _random_case(33, 3, 51)
    w = synth.inv_sizes(lab, 3).astype(np.float64)
    E = synth.poison_lower(D)
    rows = synth.shuffled_rows(lab, 4, 52)
    a = oracle.sW_alg1(D, rows, 3, w)
    b = oracle.sW_alg1(E, rows, 3, w)
    c = oracle.sW_alg2(E, rows, 3, w, 5)
    assert np.all(np.isfinite(b)) and np.array_equal(a, b)
    np.testing.assert_allclose(c, a, rtol=1e-12)
    assert np.isfinite(oracle.sT(E))


def test_invalid_labels_rejected():
    D, lab = _random_case(10, 2, 61)
    bad = lab.copy()
    bad[3] = 2
    with pytest.raises(ValueError):
        oracle.sW_alg1(D, bad[None, :], 2, [0.5, 0.5])
    bad[3] = -1
    with pytest.raises(ValueError):
        oracle.sW_alg1(D, bad[None, :], 2, [0.5, 0.5])


# ---------------------------------------------------------------------------
# Permutation generator: Philox4x32-10 against the cuRAND host library.
# ---------------------------------------------------------------------------

def _curand():
    cands = [ctypes.util.find_library("curand"), "/usr/local/cuda/lib64/libcurand.so",
             "libcurand.so.10", "libcurand.so"]
    for c in cands:
        if not c:
            continue
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    return None


def _curand_host_philox(seed, n_words):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    PHILOX = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), PHILOX) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(n_words, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(n_words)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


# The cuRAND host Philox generator emits 65,536 interleaved subsequences:
# output block b is Philox4x32-10 of counter (b // 65536, 0, b % 65536, 0)
# under key (seed_lo, seed_hi).
_SUBSEQ = 65536


@pytest.mark.parametrize("seed", [0, 9013, 0x1234567890ABCDEF])
def test_philox_matches_curand_host_generator(seed):
    T = 3
    words = _curand_host_philox(seed, 4 * _SUBSEQ * T)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for t in range(T):
        for sub in (0, 1, 2, 777, 4095, 65535):
            b = t * _SUBSEQ + sub
            ref = words[4 * b: 4 * b + 4]
            got = oracle.philox4x32_10([t, 0, sub, 0], key)
            assert np.array_equal(got, ref), (seed, t, sub)


def test_draw_stream_order_matches_curand_subsequence():
    # range 2^31 has no rejection: each draw is the raw 32-bit word >> 1, so
    # the stream of permutation p is cuRAND's subsequence p in order.
    seed = 9012
    T = 4
    words = _curand_host_philox(seed, 4 * _SUBSEQ * T)
    for p in (1, 2, 99):
        ref = np.concatenate([words[4 * (t * _SUBSEQ + p): 4 * (t * _SUBSEQ + p) + 4]
                              for t in range(T)]) >> 1
        got = oracle.bounded_draws(seed, p, 1 << 31, 4 * T)
        assert np.array_equal(got, ref)


def test_bounded_draw_is_unbiased_for_awkward_range():
    # range 3*2^30: without the rejection step residues mod 3 would get
    # probabilities 1/2, 1/4, 1/4; with it they are uniform.
    r = 3 * (1 << 30)
    d = oracle.bounded_draws(5, 1, r, 60000)
    assert d.max() < r
    frac = np.bincount(d % 3, minlength=3) / d.size
    assert np.all(np.abs(frac - 1 / 3) < 0.02)
    # small range: chi-square over 7 values
    d7 = oracle.bounded_draws(6, 2, 7, 70000)
    cnt = np.bincount(d7, minlength=7)
    chi2 = float(np.sum((cnt - 10000.0) ** 2 / 10000.0))
    assert chi2 < 30.0  # 6 dof, p ~ 4e-5


def test_permutations_preserve_multiset_and_row0():
    lab = np.array([0, 0, 0, 1, 1, 2, 3, 3, 3, 3], dtype=np.int32)
    out = oracle.permutations(lab, 200, 77)
    assert np.array_equal(out[0], lab)
    for r in out[1:]:
        assert np.array_equal(np.sort(r), np.sort(lab))
    # rows differ from each other (not a fixed permutation)
    assert len({tuple(r) for r in out[1:]}) > 150


def test_permutation_rows_independent_of_batch_size():
    lab = synth.observed_labels([30, 20, 10], 3)
    a = oracle.permutations(lab, 10, 1234)
    b = oracle.permutations(lab, 50, 1234)
    assert np.array_equal(a, b[:11])


def test_fisher_yates_uniform_over_all_orders():
    # n = 4 distinct labels: all 24 orders equally likely (Sattolo's or an
    # off-by-one variant would reach only some of them).
    lab = np.arange(4, dtype=np.int32)
    P = 48000
    out = oracle.permutations(lab, P, 99)[1:]
    codes = out @ np.array([64, 16, 4, 1])
    cnt = np.bincount(codes, minlength=256)
    used = cnt[cnt > 0]
    assert used.size == 24
    exp = P / 24.0
    chi2 = float(np.sum((used - exp) ** 2 / exp))
    assert chi2 < 60.0  # 23 dof, p ~ 4e-5


# ---------------------------------------------------------------------------
# Test wrapper: s_T, pseudo-F, p-value.
# ---------------------------------------------------------------------------

def test_pseudo_F_equals_manova_trace_statistic():
    # For Euclidean D, PERMANOVA's pseudo-F is the one-way MANOVA trace ratio
    # (tr B / (K-1)) / (tr W / (n-K)) computed from the points themselves.
    cfg = synth.recipe("euclid-1k", n=240, P=5)
    X = synth.recipe_points(cfg)
    D = synth.euclidean_matrix(X)
    lab = cfg["labels"]
    K, n = cfg["K"], len(lab)
    res = oracle.permanova_test(D, lab, K, 5, seed=1)
    mu = X.mean(axis=0)
    trW = sum(float(np.sum((X[lab == g] - X[lab == g].mean(axis=0)) ** 2)) for g in range(K))
    trB = sum(float((lab == g).sum()) * float(np.sum((X[lab == g].mean(axis=0) - mu) ** 2))
              for g in range(K))
    trT = float(np.sum((X - mu) ** 2))
    F_manova = (trB / (K - 1)) / (trW / (n - K))
    assert abs(res["s_T"] - trT) <= 1e-6 * trT
    assert abs(res["s_W"][0] - trW) <= 1e-6 * trW
    assert abs(res["F"][0] - F_manova) <= 1e-5 * F_manova


def test_count_on_F_equals_count_on_sW():
    D, lab = _random_case(40, 3, 71)
    res = oracle.permanova_test(D, lab, 3, 300, seed=72)
    by_F = int(np.sum(res["F"][1:] >= res["F"][0]))
    by_sW = int(np.sum(res["s_W"][1:] <= res["s_W"][0]))
    assert res["n_ge"] == by_F == by_sW
    assert res["p_value"] == (1 + by_F) / 301


def test_constant_matrix_gives_F_one_p_one():
    n, K = 16, 2
    D = np.full((n, n), 2.0, dtype=np.float32)
    np.fill_diagonal(D, 0)
    lab = np.array([0] * 8 + [1] * 8, dtype=np.int32)
    res = oracle.permanova_test(D, lab, K, 50, seed=3)
    np.testing.assert_allclose(res["F"], 1.0, rtol=1e-14)
    assert res["p_value"] == 1.0


def test_p_value_matches_exact_enumeration():
    # n = 8, two groups of 4: 70 distinct labelings.  The Monte Carlo p with
    # many permutations lands within 4 sigma of the exact permutation p.
    rng = np.random.default_rng(81)
    X = rng.standard_normal((8, 2))
    X[:4] += 0.7
    D = synth.euclidean_matrix(X)
    lab = np.array([0] * 4 + [1] * 4, dtype=np.int32)
    w = np.array([0.25, 0.25])
    obs = oracle.sW_alg1(D, lab[None, :], 2, w)[0]
    labs = []
    for comb in itertools.combinations(range(8), 4):
        r = np.ones(8, dtype=np.int32)
        r[list(comb)] = 0
        labs.append(r)
    all_sW = oracle.sW_alg1(D, np.array(labs), 2, w)
    p_exact = float(np.mean(all_sW <= obs * (1 + 1e-12)))
    P = 20000
    res = oracle.permanova_test(D, lab, 2, P, seed=82)
    sigma = math.sqrt(p_exact * (1 - p_exact) / P)
    assert abs(res["p_value"] - p_exact) < 4 * sigma + 2.0 / P


def test_null_p_values_roughly_uniform():
    from scipy import stats
    ps = []
    for s in range(150):
        rng = np.random.default_rng(1000 + s)
        X = rng.standard_normal((24, 3))
        D = synth.euclidean_matrix(X)
        lab = np.repeat(np.arange(3, dtype=np.int32), 8)
        ps.append(oracle.permanova_test(D, lab, 3, 199, seed=s)["p_value"])
    # discrete p on a grid of 1/200: KS against U(0,1) at a loose level
    assert stats.kstest(ps, "uniform").pvalue > 1e-3


def test_shift_gives_smallest_p():
    cfg = synth.recipe("euclid-1k", n=300, P=99)
    X = synth.recipe_points(cfg)
    X[np.arange(300), cfg["labels"]] += 1.0  # strong effect on top of the 0.3 shift
    D = synth.euclidean_matrix(X)
    res = oracle.permanova_test(D, cfg["labels"], cfg["K"], 99, seed=5)
    assert res["n_ge"] == 0 and res["p_value"] == 1 / 100


def test_test_wrapper_rejects_degenerate_inputs():
    D, lab = _random_case(10, 2, 91)
    with pytest.raises(ValueError):
        oracle.permanova_test(D, np.zeros(10, np.int32), 1, 10, 1)   # K < 2
    lab3 = lab.copy()
    lab3[:] = 0
    with pytest.raises(ValueError):
        oracle.permanova_test(D, lab3, 2, 10, 1)                     # empty group
