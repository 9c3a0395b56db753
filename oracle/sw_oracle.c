/*
 * PERMANOVA s_W oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of what the paper's hot path computes
 * ("Comparing CPU and GPU compute of PERMANOVA on MI300A", Sfiligoi 2025).
 * Only the test suite, the package smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code, header or constant
 * generator with the CUDA library; the two meet only through seeded inputs.
 *
 * What each function follows:
 *   oracle_sW_alg1   the statistic of Algorithm 1 (Sec. 2) from its
 *                    definition: d_ij^2 * w_{g(i)} summed over the pairs
 *                    i < j in one group, pairs taken in row-major order;
 *                    one label row per permutation, the label of object i
 *                    in row p at groupings[p*n + i].  FP64 throughout.
 *   oracle_sW_alg2   the blocked evaluation of Algorithm 2 (Sec. 2): row
 *                    blocks and column blocks of TILE, the column blocks of
 *                    a row block starting one column right of its first
 *                    row, each row segment summed without weights and then
 *                    weighted once.  FP64 throughout.
 *   oracle_sW_alg2_f32
 *                    Algorithm 2 with the listing's FP32 value types (float
 *                    accumulators and weights): the paper's CPU method, timed
 *                    by the benchmark for context only; never a parity
 *                    reference.
 *   oracle_sT        total sum of squares s_T = (1/n) sum_{i<j} d_ij^2, the
 *                    textbook PERMANOVA quantity (Sec. 1 refers to the method
 *                    [1-2]; Sec. 2 leaves these steps out of its listings as
 *                    cheap ones around s_W).
 *   oracle_philox4x32_10, oracle_permutations
 *                    the permutation test of Sec. 1 (the objects' group
 *                    labels reassigned at random): permutation p >= 1 is an
 *                    independent Fisher-Yates shuffle of the observed labels
 *                    driven by Philox4x32-10 (Salmon et al., SC'11) keyed by
 *                    the seed with counter (block, 0, p, 0), bounded draws by
 *                    Lemire's multiply-shift with rejection (ACM TOMACS 2019).
 *                    Row 0 is the observed grouping.
 *   oracle_permanova_test
 *                    s_T, s_W, pseudo-F = ((s_T-s_W)/(K-1)) / (s_W/(n-K)) and
 *                    p = (1 + #{p>=1 : F_p >= F_obs}) / (1 + P).
 *
 * All indices are 64-bit: the listings' 32-bit products (row*n_dims with
 * uint32, p*n_dims with int) overflow at n = 100,000 and are read as listing
 * slips, not as part of the method.
 */
#include <stdint.h>
#include <stdlib.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1

static int set_threads(int n_threads) {
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
    return omp_get_max_threads();
#else
    (void)n_threads;
    return 1;
#endif
}

int oracle_max_threads(void) { return set_threads(0); }

/* s_W of one labelling, written as its definition (Sec. 2, Algorithm 1's
 * statistic): the sum of d_ij^2 * w_{g(i)} over every pair i < j whose two
 * objects share a group.  The strict upper triangle is walked as a single
 * sequence of pairs, ordered by first index and then by second index, and
 * each qualifying pair's term is added to one FP64 accumulator in that
 * order (the accumulation order of Algorithm 1). */
static double within_ss_pairwise(const float *D, uint64_t n, uint64_t ld,
                                 const int32_t *lab, const double *w) {
    double acc = 0.0;
    if (n < 2) return acc;
    const uint64_t n_pairs = n * (n - 1) / 2;
    uint64_t i = 0, j = 1;                 /* current pair (i, j), i < j */
    for (uint64_t k = 0; k < n_pairs; ++k) {
        const int32_t gi = lab[i];
        if (lab[j] == gi) {
            const double d = (double)D[i * ld + j];
            acc += d * d * w[gi];
        }
        if (++j == n) {                    /* next first index */
            ++i;
            j = i + 1;
        }
    }
    return acc;
}

/* Sum of d_ij^2 over the columns j in [lo, hi) of row i whose label equals
 * g (no weight): one row segment of the blocked evaluation below. */
static double row_segment(const float *D, uint64_t ld, const int32_t *lab, uint64_t i,
                          uint64_t lo, uint64_t hi, int32_t g) {
    double part = 0.0;
    const float *Di = D + i * ld;
    for (uint64_t j = lo; j < hi; ++j)
        if (lab[j] == g) part += (double)Di[j] * (double)Di[j];
    return part;
}

/* s_W of one labelling evaluated in blocks, as Algorithm 2 (Sec. 2)
 * describes it: the rows are cut into blocks of `tile` rows; the columns a
 * row block meets are cut into blocks of `tile` columns, the first starting
 * one column right of the block's first row; in each (row block, column
 * block) every row contributes the part of its segment that lies right of
 * the diagonal, summed without weights, and the segment's sum is then
 * multiplied once by the weight of the row's group. */
static double within_ss_blocked(const float *D, uint64_t n, uint64_t ld,
                                const int32_t *lab, const double *w, uint64_t tile) {
    double acc = 0.0;
    if (n < 2) return acc;
    const uint64_t last_row = n - 1;       /* rows 0 .. n-2 own pairs */
    for (uint64_t rb = 0; rb < last_row; rb += tile) {
        const uint64_t rb_end = rb + tile < last_row ? rb + tile : last_row;
        for (uint64_t cb = rb + 1; cb < n; cb += tile) {
            const uint64_t cb_end = cb + tile < n ? cb + tile : n;
            for (uint64_t i = rb; i < rb_end; ++i) {
                const uint64_t lo = cb > i + 1 ? cb : i + 1;
                if (lo >= cb_end) continue;    /* segment empty: adds 0 */
                const int32_t g = lab[i];
                acc += row_segment(D, ld, lab, i, lo, cb_end, g) * w[g];
            }
        }
    }
    return acc;
}

static int labels_valid(const int32_t *groupings, uint64_t n, uint64_t n_perms, uint32_t n_groups) {
    for (uint64_t k = 0; k < n * n_perms; ++k)
        if (groupings[k] < 0 || (uint32_t)groupings[k] >= n_groups) return 0;
    return 1;
}

/* Driver of Algorithm 1: one s_W per label row (perm-major labels). */
int oracle_sW_alg1(const float *mat, uint64_t n, uint64_t ld, const int32_t *groupings,
                   uint64_t n_perms, uint32_t n_groups, const double *inv_group_sizes,
                   double *group_sWs, int n_threads) {
    if (!mat || !groupings || !inv_group_sizes || !group_sWs || ld < n || n_groups == 0)
        return ORACLE_EINVAL;
    if (!labels_valid(groupings, n, n_perms, n_groups)) return ORACLE_EINVAL;
    set_threads(n_threads);
    int64_t np = (int64_t)n_perms;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < np; ++p)
        group_sWs[p] = within_ss_pairwise(mat, n, ld, groupings + (uint64_t)p * n, inv_group_sizes);
    return ORACLE_OK;
}

/* Driver of Algorithm 2. */
int oracle_sW_alg2(const float *mat, uint64_t n, uint64_t ld, const int32_t *groupings,
                   uint64_t n_perms, uint32_t n_groups, const double *inv_group_sizes,
                   uint64_t tile, double *group_sWs, int n_threads) {
    if (!mat || !groupings || !inv_group_sizes || !group_sWs || ld < n || n_groups == 0 || tile == 0)
        return ORACLE_EINVAL;
    if (!labels_valid(groupings, n, n_perms, n_groups)) return ORACLE_EINVAL;
    set_threads(n_threads);
    int64_t np = (int64_t)n_perms;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < np; ++p)
        group_sWs[p] = within_ss_blocked(mat, n, ld, groupings + (uint64_t)p * n, inv_group_sizes, tile);
    return ORACLE_OK;
}

/* The blocked evaluation above with FP32 value types throughout (float
 * accumulators, float weights), the precision the paper's CPU code uses;
 * timing context only. */
static float within_ss_blocked_f32(const float *D, uint64_t n, uint64_t ld,
                                   const int32_t *lab, const float *w, uint64_t tile) {
    float acc = 0.0f;
    if (n < 2) return acc;
    const uint64_t last_row = n - 1;
    for (uint64_t rb = 0; rb < last_row; rb += tile) {
        const uint64_t rb_end = rb + tile < last_row ? rb + tile : last_row;
        for (uint64_t cb = rb + 1; cb < n; cb += tile) {
            const uint64_t cb_end = cb + tile < n ? cb + tile : n;
            for (uint64_t i = rb; i < rb_end; ++i) {
                const uint64_t lo = cb > i + 1 ? cb : i + 1;
                if (lo >= cb_end) continue;
                const int32_t g = lab[i];
                const float *Di = D + i * ld;
                float part = 0.0f;
                for (uint64_t j = lo; j < cb_end; ++j)
                    if (lab[j] == g) part += Di[j] * Di[j];
                acc += part * w[g];
            }
        }
    }
    return acc;
}

/* Driver of Algorithm 2 in FP32 (timing context only). */
int oracle_sW_alg2_f32(const float *mat, uint64_t n, uint64_t ld, const int32_t *groupings,
                       uint64_t n_perms, uint32_t n_groups, const float *inv_group_sizes,
                       uint64_t tile, float *group_sWs, int n_threads) {
    if (!mat || !groupings || !inv_group_sizes || !group_sWs || ld < n || n_groups == 0 || tile == 0)
        return ORACLE_EINVAL;
    if (!labels_valid(groupings, n, n_perms, n_groups)) return ORACLE_EINVAL;
    set_threads(n_threads);
    int64_t np = (int64_t)n_perms;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < np; ++p)
        group_sWs[p] = within_ss_blocked_f32(mat, n, ld, groupings + (uint64_t)p * n, inv_group_sizes, tile);
    return ORACLE_OK;
}

/* s_T = (1/n) * sum_{i<j} d_ij^2 in FP64. */
double oracle_sT(const float *mat, uint64_t n, uint64_t ld) {
    double s = 0.0;
    for (uint64_t row = 0; row + 1 < n; ++row)
        for (uint64_t col = row + 1; col < n; ++col) {
            double val = (double)mat[row * ld + col];
            s += val * val;
        }
    return s / (double)n;
}

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ------------------ */
/* Round: multiply words 0 and 2 by the two round constants, cross the
 * high halves into the other lanes XORed with the odd words and the key,
 * keep the low halves; the key is bumped by the two Weyl constants between
 * rounds. */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * x0;
        uint64_t p1 = (uint64_t)M1 * x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0; k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

typedef struct {
    uint32_t key[2];
    uint32_t perm;
    uint32_t block;
    uint32_t buf[4];
    int used;
} draw_stream;

static uint32_t stream_next(draw_stream *s) {
    if (s->used == 4) {
        uint32_t ctr[4] = {s->block, 0u, s->perm, 0u};
        oracle_philox4x32_10(ctr, s->key, s->buf);
        s->block += 1;
        s->used = 0;
    }
    return s->buf[s->used++];
}

/* Uniform integer in [0, range), range >= 1: Lemire's nearly-divisionless
 * method -- the high word of x*range, rejecting low words below
 * (2^32 - range) mod range. */
static uint32_t stream_bounded(draw_stream *s, uint32_t range) {
    uint64_t m = (uint64_t)stream_next(s) * (uint64_t)range;
    uint32_t low = (uint32_t)m;
    if (low < range) {
        uint32_t threshold = (uint32_t)(-range) % range;
        while (low < threshold) {
            m = (uint64_t)stream_next(s) * (uint64_t)range;
            low = (uint32_t)m;
        }
    }
    return (uint32_t)(m >> 32);
}

/* Exposed for the tests: ``count`` bounded draws in [0, range) from stream
 * (seed, perm), the same draw sequence the shuffle consumes. */
int oracle_bounded_draws(uint64_t seed, uint32_t perm, uint32_t range, uint64_t count, uint32_t *out) {
    if (!out || range == 0) return ORACLE_EINVAL;
    draw_stream s;
    s.key[0] = (uint32_t)seed;
    s.key[1] = (uint32_t)(seed >> 32);
    s.perm = perm;
    s.block = 0;
    s.used = 4;
    for (uint64_t k = 0; k < count; ++k) out[k] = stream_bounded(&s, range);
    return ORACLE_OK;
}

/* out: (n_perms + 1) x n int32, row 0 = grouping, row p = Fisher-Yates shuffle
 * of grouping driven by stream (seed, p). */
int oracle_permutations(const int32_t *grouping, uint64_t n, uint64_t n_perms, uint64_t seed,
                        int32_t *out, int n_threads) {
    if (!grouping || !out || n == 0 || n > 0xFFFFFFFFull || n_perms >= 0xFFFFFFFFull)
        return ORACLE_EINVAL;
    set_threads(n_threads);
    for (uint64_t i = 0; i < n; ++i) out[i] = grouping[i];
    int64_t np = (int64_t)n_perms;
#pragma omp parallel for schedule(static)
    for (int64_t pp = 1; pp <= np; ++pp) {
        int32_t *a = out + (uint64_t)pp * n;
        for (uint64_t i = 0; i < n; ++i) a[i] = grouping[i];
        draw_stream s;
        s.key[0] = (uint32_t)seed;
        s.key[1] = (uint32_t)(seed >> 32);
        s.perm = (uint32_t)pp;
        s.block = 0;
        s.used = 4;
        for (uint64_t i = n - 1; i >= 1; --i) {
            uint32_t j = stream_bounded(&s, (uint32_t)(i + 1));
            int32_t t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
    return ORACLE_OK;
}

/* Full permutation test.  sW_out and F_out hold n_perms + 1 values (index 0 =
 * observed).  Returns EINVAL when a label is outside [0, K), a group is empty,
 * K < 2 or n <= K (pseudo-F undefined). */
int oracle_permanova_test(const float *mat, uint64_t n, uint64_t ld, const int32_t *grouping,
                          uint32_t n_groups, uint64_t n_perms, uint64_t seed,
                          double *s_T_out, double *sW_out, double *F_out,
                          double *p_value_out, uint64_t *n_ge_out, int n_threads) {
    if (!mat || !grouping || !sW_out || !F_out || !s_T_out || !p_value_out || !n_ge_out)
        return ORACLE_EINVAL;
    if (n_groups < 2 || n <= n_groups || ld < n || n_perms == 0) return ORACLE_EINVAL;
    uint64_t *sizes = (uint64_t *)calloc(n_groups, sizeof(uint64_t));
    double *w = (double *)calloc(n_groups, sizeof(double));
    int32_t *labels = (int32_t *)malloc(sizeof(int32_t) * n * (n_perms + 1));
    int rc = ORACLE_OK;
    if (!sizes || !w || !labels) { rc = ORACLE_EINVAL; goto done; }
    for (uint64_t i = 0; i < n; ++i) {
        if (grouping[i] < 0 || (uint32_t)grouping[i] >= n_groups) { rc = ORACLE_EINVAL; goto done; }
        sizes[grouping[i]] += 1;
    }
    for (uint32_t g = 0; g < n_groups; ++g) {
        if (sizes[g] == 0) { rc = ORACLE_EINVAL; goto done; }
        w[g] = 1.0 / (double)sizes[g];
    }
    rc = oracle_permutations(grouping, n, n_perms, seed, labels, n_threads);
    if (rc) goto done;
    rc = oracle_sW_alg1(mat, n, ld, labels, n_perms + 1, n_groups, w, sW_out, n_threads);
    if (rc) goto done;
    double s_T = oracle_sT(mat, n, ld);
    double dfb = (double)(n_groups - 1), dfw = (double)(n - n_groups);
    for (uint64_t p = 0; p <= n_perms; ++p) {
        double s_W = sW_out[p];
        F_out[p] = ((s_T - s_W) / dfb) / (s_W / dfw);
    }
    uint64_t n_ge = 0;
    for (uint64_t p = 1; p <= n_perms; ++p)
        if (F_out[p] >= F_out[0]) n_ge += 1;
    *s_T_out = s_T;
    *n_ge_out = n_ge;
    *p_value_out = (double)(1 + n_ge) / (double)(1 + n_perms);
done:
    free(sizes);
    free(w);
    free(labels);
    return rc;
}
