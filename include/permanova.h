/*
 * permanova.h -- C ABI of libpermanova.so, PERMANOVA's within-group statistic
 * s_W on one NVIDIA GB300 (sm_103a).
 *
 * The operation is the one the paper calls permanova_f_stat_sW ("Comparing CPU
 * and GPU compute of PERMANOVA on MI300A", Sec. 2, Algorithms 1-3): for each
 * label row p of a batch of groupings,
 *
 *     s_W[p] = sum over 0 <= i < j < n with g_p(i) == g_p(j) of
 *              mat[i*ld + j]^2 * inv_group_sizes[g_p(i)]
 *
 * over a dense distance matrix of which only the strict upper triangle
 * (column > row) is read; the diagonal and the lower triangle may hold
 * anything, NaN included.  Around it, permanova_test adds the steps that the
 * paper leaves around s_W (Sec. 2) for the permutation test of Sec. 1:
 * group sizes, permutations of the observed grouping, the total sum of squares
 * s_T, the pseudo-F statistic and the permutation p-value.
 *
 * Conventions for every call:
 *  - Every function returns a permanova_status (0 = success).  On failure a
 *    message is available from permanova_last_error(ctx) until the next call
 *    on the same context from the same thread.
 *  - "DEVICE" pointers are CUDA device (or managed) memory on the context's
 *    device; "HOST" pointers are ordinary host memory.  The caller owns every
 *    buffer it passes; the library never frees or retains them after the call.
 *  - Scratch memory (partial sums, packed labels, the split D^2 planes of the
 *    tensor-core form, permutation labels) belongs to the context, is reused
 *    across calls and is bounded by the context's HBM budget: a call whose
 *    scratch would exceed the budget returns PERMANOVA_ENOMEM before
 *    allocating anything.
 *  - stream is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Asynchronous calls only enqueue work on it.
 *  - Calls on one context are serialised by an internal lock; separate
 *    contexts are independent.
 *  - Device kernels never trap.  A label found outside [0, n_groups) or a
 *    device-side wait that ran out of time sets a device error word; the next
 *    call that synchronises (permanova_sync, permanova_test, the _host
 *    variants) returns PERMANOVA_EINVAL / PERMANOVA_ETIMEOUT and clears it.
 *    The outputs of the failed batch are unspecified.
 */
#ifndef PERMANOVA_H
#define PERMANOVA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PERMANOVA_OK = 0,
    PERMANOVA_EINVAL = 1,       /* bad argument, or a label >= n_groups found on the device */
    PERMANOVA_ENOMEM = 2,       /* scratch would exceed the HBM budget, or cudaMalloc failed */
    PERMANOVA_ECUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
    PERMANOVA_ETIMEOUT = 4,     /* a bounded device-side wait ran out */
    PERMANOVA_EUNSUPPORTED = 5  /* form not available for these sizes (e.g. GEMM with K > 256) */
} permanova_status;

/* Element type of the label rows ("groupings").  The paper's listings use
 * int; the packed types cut label traffic 4x / 2x. */
typedef enum {
    PERMANOVA_LABEL_I32 = 0,
    PERMANOVA_LABEL_U16 = 1,
    PERMANOVA_LABEL_U8 = 2
} permanova_label_t;

/* Kernel form used for s_W.
 *   BRUTE      Algorithm 3's brute force: the triangle is streamed from HBM
 *              once per label row (HBM-bound).
 *   PERMBLOCK  a triangle tile of D^2 is held in shared memory and reused by
 *              a block of 256 label rows, two per thread compared at once
 *              with packed FP16 equality (uint8 codes, and uint16 codes up to
 *              2,048 groups; beyond that 128 rows with FP32 compares),
 *              CUDA-core and issue-bound; the row
 *              weight is applied once per row segment as in Algorithm 2.
 *   GEMM       the dense-contraction form Z_p = (D o D) X_p with one-hot
 *              indicator columns X_p, on the tcgen05 tensor cores: D^2, scaled
 *              by a power of two per 128-row band, split into a BF16 hi and an
 *              FP16 lo part (BF16 where a band spans more than 2^28), FP32
 *              accumulation in tensor memory drained every 512 columns, FP64
 *              partial sums.  Needs n_groups <= 256.
 *   AUTO       the planner's choice for (n, K, P): a bucket timed by
 *              permanova_autotune if there is one, else GEMM for K <= 24,
 *              n >= 256 and P >= 32, else PERMBLOCK for P >= 16, else BRUTE.
 * Accuracy of s_W against an FP64 evaluation of the definition: the CUDA-core
 * forms (BRUTE, PERMBLOCK) sum in FP32 per row segment and FP64 beyond, about
 * 1e-9 relative on typical data and at most a few 1e-7 on adversarial ones;
 * the GEMM form stays within 1e-5 relative (measured about 5e-7 on typical
 * data and at most 5.2e-6 on adversarial ones: constant, two-valued and
 * narrowly spread matrices, where every rounding errs the same way). */
typedef enum {
    PERMANOVA_FORM_AUTO = 0,
    PERMANOVA_FORM_BRUTE = 1,
    PERMANOVA_FORM_PERMBLOCK = 2,
    PERMANOVA_FORM_GEMM = 3
} permanova_form_t;

typedef struct permanova_ctx permanova_ctx;

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * context's scratch (0 = 90% of the device's free memory at creation).
 * *out receives the context; NULL on failure.  Returns EINVAL for a bad
 * device or NULL out, ECUDA if the device cannot be initialised. */
int permanova_create(int device, size_t hbm_budget_bytes, permanova_ctx **out);

/* Synchronise the context's device, free its scratch and destroy it.  NULL is
 * a no-op. */
void permanova_destroy(permanova_ctx *ctx);

/* Message describing the last failure on this thread for ctx ("" if none).
 * The pointer stays valid until the next call on ctx from this thread. */
const char *permanova_last_error(const permanova_ctx *ctx);

/* Force a kernel form for subsequent calls (PERMANOVA_FORM_AUTO restores the
 * planner).  Returns EINVAL for an unknown form. */
int permanova_set_form(permanova_ctx *ctx, int form);

/* A kernel plan: the form and its knobs (0 = the default of a knob). */
typedef struct {
    int form;                     /* permanova_form_t; AUTO restores the planner */
    int permblock_variant;        /* 0: paired FP16-compare kernel for uint8 codes and uint16
                                     codes up to 2,048 groups (3 blocks/SM), 2: the same at
                                     4 blocks/SM, 1: FP32 compare-and-set */
    uint32_t gemm_rows_div;       /* tensor-core form: label rows per tile divided by 1, 2 or 4 */
    uint32_t gemm_drain_kblocks;  /* tensor-core form: k-blocks between FP64 drains, 1 .. 8 (default 8) */
    uint32_t brute_chunk_mult;    /* brute force: chunks per label row multiplied by 1 .. 16 */
} permanova_plan_t;

/* Force a plan (form and knobs) for subsequent calls; NULL or form AUTO
 * restores the planner.  EINVAL for a knob out of range (a drain interval
 * above 8 k-blocks is refused: it breaks the 1e-5 accuracy target). */
int permanova_set_plan(permanova_ctx *ctx, const permanova_plan_t *plan);

/* Form the planner would use (or the forced one) for these sizes. */
int permanova_plan_form(permanova_ctx *ctx, uint32_t n_dims, uint32_t n_groups, uint64_t n_perms);

/* The plan (form and knobs) a permanova_sW call of these sizes would use, as
 * a one-line JSON object written to `out` (HOST, `cap` bytes), with its
 * source: "forced", "autotuned" or "rule".  EINVAL if it does not fit. */
int permanova_plan_describe(permanova_ctx *ctx, uint32_t n_dims, uint32_t n_groups, uint64_t n_perms,
                            char *out, size_t cap);

/* Autotuner: times candidate plans on a sample of the given label rows (about
 * 4e12 pair evaluations, 64 to 4,096 rows) and makes the fastest the
 * planner's choice for calls with the same log2 buckets of n_dims and n_perms
 * and the same n_groups.  The candidates cover every form that can run these
 * sizes and each form's knobs: the brute force's chunks per label row (x1,
 * x2), the perm-block kernel's variant (paired FP16 compares at 3 or 4
 * blocks per SM, or FP32 compare-and-set), the tensor-core form's label rows per tile (full or
 * half width) and drain interval (8 or 4 k-blocks: never longer, the accuracy
 * limit of the 1e-5 target).  Arguments as permanova_sW (no output buffer:
 * the sample's results go to scratch).  *out_form (optional, HOST) receives
 * the chosen permanova_form_t.  Synchronises `stream`; errors as
 * permanova_sW. */
int permanova_autotune(permanova_ctx *ctx, const float *mat, uint32_t n_dims, uint64_t ld,
                       const void *groupings, int label_type, uint32_t n_groups, uint64_t n_perms,
                       const float *inv_group_sizes, int *out_form, void *stream);

/* CUDA graphs (1 = on, 0 = off, the default): with graphs on, a
 * permanova_sW call on a non-default stream whose arguments and chosen form
 * repeat an earlier call's replays the captured graph of its launches instead
 * of launching each kernel.  Graphs are dropped when the scratch arena grows
 * and when graphs are turned off; calls on a stream that is already being
 * captured, and profiled calls, launch directly. */
int permanova_set_graphs(permanova_ctx *ctx, int enable);

/* Failure-detection self-test (not a paper operation): launches, on
 * `stream`, a kernel whose one thread waits on a device barrier that nothing
 * ever completes, using the same bounded wait as the tensor-core kernel.
 * After limit_us microseconds (1 .. 10,000,000) the wait gives up, records
 * the timeout in the context's device error word and the kernel returns; the
 * next permanova_sync reports PERMANOVA_ETIMEOUT and the context stays
 * usable.  Asynchronous; EINVAL for a limit out of range. */
int permanova_selftest_wait(permanova_ctx *ctx, uint32_t limit_us, void *stream);

/* Bytes of context scratch a permanova_sW call of these sizes needs under
 * `form` (AUTO = the planner's form).  0 on invalid sizes. */
size_t permanova_scratch_bytes(permanova_ctx *ctx, int form, uint32_t n_dims, uint32_t n_groups,
                               uint64_t n_perms);

/* Bytes of device scratch the context holds now (its arena only grows while
 * calls need more, up to the budget, and is kept between calls). */
size_t permanova_scratch_reserved(permanova_ctx *ctx);

/* Grow the context's scratch arena to at least `bytes` now (so later calls
 * need no allocation of their own).  ENOMEM beyond the budget. */
int permanova_reserve_scratch(permanova_ctx *ctx, size_t bytes);

/* Wait for the context's device, then free the context's scratch arena (the
 * next call allocates again).  Lets a server that keeps several contexts
 * return the memory an idle one holds. */
int permanova_release_scratch(permanova_ctx *ctx);

/* The paper's permanova_f_stat_sW_T (Sec. 2, Algorithm 1's driver): s_W for
 * n_perms label rows.  Asynchronous on `stream`.
 *   mat              DEVICE, fp32, row-major, n_dims rows of stride ld
 *                    elements (ld >= n_dims); only column > row is read.
 *   groupings        DEVICE, n_perms rows of n_dims labels, perm-major: label
 *                    of object i in row p at groupings[p*n_dims + i], element
 *                    type label_type; every label must be < n_groups.
 *   inv_group_sizes  DEVICE, n_groups fp32 weights (the paper's
 *                    inv_group_sizes; normally 1/n_g, any value accepted).
 *   out_sW           DEVICE, n_perms doubles, written in full.
 * Errors: EINVAL for NULL pointers, n_dims < 2, ld < n_dims, n_groups == 0,
 * n_groups > 256 with U8 or > 65536 with U16, n_perms == 0; ENOMEM if the
 * scratch exceeds the budget; EUNSUPPORTED if a forced form cannot run these
 * sizes; ECUDA on a launch failure.  Labels >= n_groups are reported by the
 * next synchronising call. */
int permanova_sW(permanova_ctx *ctx, const float *mat, uint32_t n_dims, uint64_t ld,
                 const void *groupings, int label_type, uint32_t n_groups, uint64_t n_perms,
                 const float *inv_group_sizes, double *out_sW, void *stream);

/* Same as permanova_sW with HOST buffers: mat (n_dims x ld fp32),
 * groupings, inv_group_sizes and out_sW live in host memory (pinned memory
 * gives full copy speed).  The call copies the inputs to the device, runs
 * s_W, copies the n_perms results back and synchronises `stream`.  With the
 * tensor-core form each 128-row band b is copied as the flat host range from
 * element (128 b, 128 b) to the end of the band's last row, or, when the
 * band's rows span under half the width (n - 128 b < n / 2), as one
 * two-dimensional copy of its trapezoid alone, in up to 16 segments (band
 * counts ramping up 1 : 2 : 4 :
 * 8 : 8 : ..., so the kernels start after a short first copy) through three
 * device staging slots sized for the largest segment, and each segment's
 * kernels start as soon as it has landed, so the copies overlap the
 * computation; segments
 * alternate between `stream` and a second stream of the context (joined back
 * into `stream` before the final reduction), so one segment's last wave of
 * blocks overlaps the next segment's first.  The CUDA-core forms copy the
 * whole matrix first.  The copies run on a stream of the context, ordered
 * after the work already queued on `stream`.  Errors as permanova_sW, plus
 * any error the device reported (the call synchronises). */
int permanova_sW_host(permanova_ctx *ctx, const float *mat, uint32_t n_dims, uint64_t ld,
                      const void *groupings, int label_type, uint32_t n_groups, uint64_t n_perms,
                      const float *inv_group_sizes, double *out_sW, void *stream);

/* permanova_sW for callers that cannot allocate device memory.  The paper has
 * no counterpart: this is a deployment variant.  Callers that cannot call
 * cudaMalloc include plugins whose host framework owns every device
 * allocation (and forbids others), and processes confined to a fixed device
 * memory pool with no headroom, where a new allocation would fail or evict
 * the host framework's own buffers.
 * It needs no context and allocates nothing: it runs the perm-block kernel
 * (when the labels are uint8 or uint16 codes whose rows start on 16-byte
 * boundaries and its partials, one row of n_perms doubles per 64-row band,
 * fit) or else the brute-force kernel, with their scratch (FP64 partial
 * sums, FP64 weights, the device error word) in one fixed 8 MiB device array
 * that the library keeps resident on every GPU that loads it, until the
 * process exits.
 *   Arguments as permanova_sW (DEVICE mat, groupings, inv_group_sizes,
 *   out_sW; the current CUDA device is used).
 *   Limits: n_perms * 8 bytes must fit in the array after the error word and
 *   the weights (1,048,512 label rows with n_groups <= 32); larger calls
 *   return PERMANOVA_EINVAL with a message, before any work is queued.
 *   Set-up: the first call on a device (and the first after the device's
 *   context was replaced, e.g. by cudaDeviceReset) looks up the array's
 *   device address; make that call before any stream capture on the device.
 *   The call synchronises `stream` and reports a label >= n_groups as
 *   PERMANOVA_EINVAL.  All calls on a device share the array, and it keeps
 *   the last call's contents (each call clears the error word and overwrites
 *   the weights and partials it reads): calls whose work overlaps on the GPU
 *   (other streams, other host threads) race, so callers must serialise
 *   them.  Error text: permanova_last_error(NULL). */
int permanova_sW_noalloc(const float *mat, uint32_t n_dims, uint64_t ld, const void *groupings,
                         int label_type, uint32_t n_groups, uint64_t n_perms,
                         const float *inv_group_sizes, double *out_sW, void *stream);

/* Wait for `stream`, then report (and clear) any device error word raised by
 * earlier asynchronous calls on this context.  Returns OK, EINVAL (invalid
 * label), ETIMEOUT or ECUDA. */
int permanova_sync(permanova_ctx *ctx, void *stream);

/* Permutation labels for the permutation test of Sec. 1 (the objects' group
 * labels reassigned at random), generated on the device:
 *   grouping   DEVICE, n_dims int32 observed labels in [0, n_groups).
 *   out        DEVICE, (n_perms + 1) rows of n_dims labels of label_type;
 *              row 0 = grouping, row p >= 1 = an independent Fisher-Yates
 *              shuffle of grouping driven by Philox4x32-10 (Salmon et al.,
 *              SC'11) under key (seed mod 2^32, seed / 2^32) and counter
 *              (block, 0, p, 0), words taken in order, bounded draws by
 *              Lemire's multiply-shift with rejection.
 * Asynchronous.  EINVAL for NULL pointers, n_dims < 2, n_perms == 0 or
 * n_perms >= 2^32 - 1, n_dims >= 2^32, a label type too narrow for
 * n_groups. */
int permanova_permutations(permanova_ctx *ctx, const int32_t *grouping, uint32_t n_dims,
                           uint32_t n_groups, uint64_t n_perms, uint64_t seed, void *out,
                           int label_type, void *stream);

/* Profiling counters of a context (not a paper operation; measurement
 * support).  While enabled, every s_W call on device buffers records CUDA
 * events on its stream around its dominant kernel (the brute-force, perm-block
 * or GEMM kernel), every kernel the library launches is counted, and every
 * permanova_sW_host call records events at its start, when each segment of
 * the matrix has landed on the device, when each segment's dominant kernel
 * has run, and at its end (the results copied back). */
typedef struct {
    double main_kernel_ms;          /* summed event time of the dominant kernels */
    uint64_t main_kernel_launches;  /* dominant-kernel launches recorded */
    uint64_t kernel_launches;       /* all kernels launched by the library */
    int last_form;                  /* permanova_form_t of the last s_W call */
    uint64_t host_calls;            /* permanova_sW_host calls recorded */
    double host_total_ms;           /* summed device time, call start to results copied back */
    double host_first_segment_ms;   /* summed time until the first matrix segment landed */
    double host_copy_ms;            /* summed time until the last matrix segment landed */
    uint64_t host_h2d_bytes;        /* bytes those calls copied host to device */
    uint32_t host_segments;         /* matrix segments of the last recorded call (<= 16;
                                       1 for the CUDA-core forms, which copy D whole) */
    double host_seg_landed_ms[16];  /* per segment k: summed time, call start to segment
                                       k landed (calls with fewer segments add nothing) */
    double host_seg_done_ms[16];    /* per segment k: summed time, call start to segment
                                       k's dominant kernel done */
} permanova_profile_t;

/* Enable (1) or disable (0) profiling; enabling clears the counters. */
int permanova_profile_enable(permanova_ctx *ctx, int enable);

/* Synchronise the context's device, sum the recorded events into *out
 * (HOST) and clear the counters. */
int permanova_profile_read(permanova_ctx *ctx, permanova_profile_t *out);

typedef struct {
    double s_T;        /* (1/n) sum_{i<j} d_ij^2 */
    double s_W_obs;    /* s_W of the observed grouping */
    double F_obs;      /* ((s_T - s_W)/(K-1)) / (s_W/(n-K)) */
    double p_value;    /* (1 + n_ge) / (1 + n_perms) */
    uint64_t n_ge;     /* #{p >= 1 : F_p >= F_obs}, counted as s_W[p] <= s_W_obs */
    uint64_t n_perms;  /* permutations drawn */
} permanova_result;

/* One PERMANOVA test (Sec. 1; s_W as in Sec. 2).
 *   mat        DEVICE distance matrix as in permanova_sW.
 *   grouping   DEVICE, n_dims int32 labels in [0, n_groups), every group
 *              non-empty.
 *   n_perms    permutations (>= 1); their labels come from
 *              permanova_permutations with `seed`.
 *   out_host   HOST, receives the result.
 *   out_sW     optional DEVICE buffer of n_perms + 1 doubles (NULL = none):
 *              s_W of the observed grouping (index 0) and of every
 *              permutation.
 * Synchronises `stream`.  EINVAL for NULL mat/grouping/out_host, n_groups < 2,
 * n_dims <= n_groups (pseudo-F undefined), an empty group or a label outside
 * [0, n_groups); plus the errors of permanova_sW. */
int permanova_test(permanova_ctx *ctx, const float *mat, uint32_t n_dims, uint64_t ld,
                   const int32_t *grouping, uint32_t n_groups, uint64_t n_perms, uint64_t seed,
                   permanova_result *out_host, double *out_sW, void *stream);

/* n_tests permutation tests on one matrix with the same n_groups and n_perms
 * in one pass (permanova_test_mixed with equal counts).
 *   groupings  DEVICE, n_tests rows of n_dims int32 observed labels (row t =
 *              test t), each in [0, n_groups) with every group non-empty.
 *   seeds      HOST, n_tests permutation seeds.
 *   out_host   HOST, n_tests results.
 *   out_sW     optional DEVICE buffer of n_tests x (n_perms + 1) doubles.
 * All tests' label rows go through one s_W launch, each test weighted by its
 * own 1/n_g; the kernel form is the one a single test of these sizes gets,
 * so every result equals the corresponding permanova_test call bit for bit.
 * Synchronises `stream`; errors as permanova_test (the message names the
 * test). */
int permanova_test_batch(permanova_ctx *ctx, const float *mat, uint32_t n_dims, uint64_t ld,
                         const int32_t *groupings, uint32_t n_tests, uint32_t n_groups,
                         uint64_t n_perms, const uint64_t *seeds, permanova_result *out_host,
                         double *out_sW, void *stream);

/* Several permutation tests on one matrix with their own group counts and
 * permutation counts, in as few s_W passes as possible (the fusion a server
 * applies to the requests waiting on one matrix; Sec. 1 notes that many
 * tests are typically run on one distance matrix).
 *   groupings  DEVICE, n_tests rows of n_dims int32 observed labels; row t in
 *              [0, n_groups[t]) with every group non-empty.
 *   n_groups   HOST, n_tests group counts (each >= 2 and < n_dims).
 *   n_perms    HOST, n_tests permutation counts (each >= 1).
 *   seeds      HOST, n_tests permutation seeds.
 *   out_host   HOST, n_tests results.
 *   out_sW     optional DEVICE buffer of sum_t (n_perms[t] + 1) doubles: test
 *              t's s_W (observed first) after those of tests 0 .. t-1.
 * Every test runs in the kernel form a lone test of its sizes gets; the tests
 * of one form share one s_W launch over all their label rows, with the
 * largest group count among them (each test weighted by its own 1/n_g,
 * groups it lacks weighted 0).  Each result equals the corresponding
 * permanova_test call bit for bit.  Synchronises `stream`; errors as
 * permanova_test (the message names the test). */
int permanova_test_mixed(permanova_ctx *ctx, const float *mat, uint32_t n_dims, uint64_t ld,
                         const int32_t *groupings, uint32_t n_tests, const uint32_t *n_groups,
                         const uint64_t *n_perms, const uint64_t *seeds, permanova_result *out_host,
                         double *out_sW, void *stream);

/* A prepared matrix: the tensor-core form's operands (D^2 of every band
 * trapezoid, scaled per band and split into the BF16 hi and FP16/BF16 lo
 * tiles, with the band words) made once and reused by every call that names
 * it, so a run of many batches (the 13 batches of a 99,999-permutation test
 * at n = 100,000) or the many tests of a served matrix pay for them once.
 * Not a paper operation: the paper recomputes nothing between permutations
 * because its kernel reads D directly.
 *   permanova_prepare   mat (DEVICE, as in permanova_sW) is read once, on
 *                       `stream`, into a new device allocation of about
 *                       2 n^2 bytes owned by the handle (not counted in any
 *                       context's budget); synchronises `stream`.  The
 *                       caller keeps mat alive and unchanged while the handle
 *                       exists (calls whose plan is a CUDA-core form read it).
 *                       *out is NULL on failure (EINVAL, ENOMEM, ECUDA).
 *   permanova_prepared_destroy   waits for the device and frees the handle.
 * The handle is read-only after preparation: contexts on its device may use
 * it concurrently. */
typedef struct permanova_prepared permanova_prepared;
int permanova_prepare(permanova_ctx *ctx, const float *mat, uint32_t n_dims, uint64_t ld,
                      permanova_prepared **out, void *stream);
void permanova_prepared_destroy(permanova_prepared *prepared);

/* permanova_sW on a prepared matrix: the same arguments after the handle,
 * the same results bit for bit; with the tensor-core form the operand
 * preparation is skipped (and its scratch not needed). */
int permanova_sW_prepared(permanova_ctx *ctx, const permanova_prepared *prepared, const void *groupings,
                          int label_type, uint32_t n_groups, uint64_t n_perms,
                          const float *inv_group_sizes, double *out_sW, void *stream);

/* permanova_test_mixed on a prepared matrix (same results bit for bit). */
int permanova_test_mixed_prepared(permanova_ctx *ctx, const permanova_prepared *prepared,
                                  const int32_t *groupings, uint32_t n_tests, const uint32_t *n_groups,
                                  const uint64_t *n_perms, const uint64_t *seeds,
                                  permanova_result *out_host, double *out_sW, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PERMANOVA_H */
