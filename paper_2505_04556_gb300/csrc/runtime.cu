// Host runtime behind the C ABI of libpermanova (include/permanova.h):
// argument checks, the kernel-form planner, the context's scratch arena, and
// the orchestration of the s_W path and the permutation test.
#include "../../include/permanova.h"
#include "common.cuh"

#include <algorithm>
#include <array>
#include <functional>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <map>
#include <tuple>
#include <vector>

using namespace pmn;

namespace {
// (log2 bucket of n, n_groups, log2 bucket of n_perms) -> tuned plan
using TuneKey = std::tuple<int, uint32_t, int>;
// every argument of a permanova_sW call plus the form and the scratch arena
using GraphKey = std::tuple<const void*, uint32_t, uint64_t, const void*, int, uint32_t, uint64_t,
                            const void*, void*, void*, int, void*>;
int log2_bucket(uint64_t x) {
    int b = 0;
    while ((1ull << b) < x && b < 63) ++b;
    return b;
}
}  // namespace

// A kernel plan: the form and the knobs of that form.
struct Plan {
    int form = PERMANOVA_FORM_BRUTE;
    int pb_variant = 0;          // perm-block: 0 paired FP16 compares (uint8 codes, 3 CTAs/SM), 2 the
                                 // same at 4 CTAs/SM, 1 FP32 compare-and-set
    uint32_t gemm_ppt_div = 1;   // tensor-core form: label rows per tile divided by this
    uint32_t gemm_drain = 0;     // tensor-core form: k-blocks between FP64 drains (0 = default, 8)
    uint32_t brute_mult = 1;     // brute force: chunks per label row multiplied by this
    bool tuned = false;
    bool prepared = false;       // GEMM operands come from a prepared matrix (no scratch for them)
    bool operator==(const Plan& o) const {
        return form == o.form && pb_variant == o.pb_variant && gemm_ppt_div == o.gemm_ppt_div &&
               gemm_drain == o.gemm_drain && brute_mult == o.brute_mult;
    }
};

struct permanova_ctx {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0;
    int forced_form = PERMANOVA_FORM_AUTO;
    Plan forced_plan;                           // knobs of a forced plan (permanova_set_plan)
    std::map<TuneKey, Plan> tuned;              // autotuner results
    bool graphs = false;                        // replay captured launch sequences
    struct CachedGraph {
        cudaGraphExec_t exec;
        uint64_t kernels;   // kernels the captured sequence launches (counted on every replay)
    };
    std::map<GraphKey, CachedGraph> graph_cache;
    std::mutex mu;
    void* arena = nullptr;
    size_t arena_size = 0;
    DevStatus* status = nullptr;        // device error word
    DevStatus* status_host = nullptr;   // pinned mirror
    // profiling
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    uint64_t launch_mark = 0;
    int last_form = 0;
    // host entry point (profiling): per call, timing events at its start, when
    // the first and the last matrix segment have landed, and at its end
    std::vector<std::array<cudaEvent_t, 4>> host_events;
    // per host-entry call (same index as host_events): segment k landed for
    // k < m, then segment k's dominant kernel done, m segments
    std::vector<std::vector<cudaEvent_t>> host_seg_events;
    uint64_t host_h2d_bytes = 0;
    // host entry point: copies run on their own stream, ordered by events;
    // matrix segments alternate between the caller's stream and seg_stream so
    // that one segment's last wave overlaps the next segment's first
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> copy_events;
    cudaStream_t seg_stream = nullptr;
    cudaEvent_t seg_fork = nullptr, seg_join = nullptr;
};

// A matrix whose tensor-core operands (the split D^2 tiles and band words)
// were made once and are reused by every call that names it.
struct permanova_prepared {
    int device = 0;
    const float* mat = nullptr;   // the caller's matrix (the CUDA-core forms still read it)
    uint32_t n = 0;
    uint64_t ld = 0;
    void* ops = nullptr;
    size_t bytes = 0;
};

namespace {

thread_local std::string tl_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    tl_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();  // clear a sticky-free error so later calls can proceed
    return fail(e == cudaErrorMemoryAllocation ? PERMANOVA_ENOMEM : PERMANOVA_ECUDA, "%s: %s (%s)",
                what, cudaGetErrorString(e), cudaGetErrorName(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

constexpr size_t kAlign = 256;
constexpr uint32_t kHostSegments = 16;   // band segments of the host entry point's copy pipeline
constexpr uint32_t kHostSlots = 3;       // staging slots of the tensor-core form's band segments
size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }

// Scratch carve-up for one s_W call.
struct SWLayout {
    int form = 0;
    Plan plan;
    uint32_t part_rows = 0;     // rows of the FP64 partials table
    size_t part_off = 0;
    bool repack = false;        // labels re-laid out as codes
    int code_type = LABEL_U8;
    uint64_t lstride = 0;
    size_t lab_off = 0;
    size_t gemm_off = 0;        // prepared operands (GEMM form; unused when prepared elsewhere)
    size_t counter_off = 0;     // GEMM work counters
    size_t w_off = 0;           // n_groups FP64 weights
    size_t total = 0;
};

int label_bytes(int t) { return t == LABEL_U8 ? 1 : t == LABEL_U16 ? 2 : 4; }

Plan plan_for(const permanova_ctx* ctx, uint32_t n, uint32_t K, uint64_t P) {
    Plan pl;
    if (ctx->forced_form != PERMANOVA_FORM_AUTO) return ctx->forced_plan;
    auto it = ctx->tuned.find(TuneKey{log2_bucket(n), K, log2_bucket(P)});
    if (it != ctx->tuned.end()) return it->second;
    // The tensor-core form costs 4K flops per pair and label row (two 16-bit
    // planes, K one-hot columns); the paired perm-block kernel about 1.6
    // instructions per pair and label row whatever K is.  Measured on a GB300
    // at n = 20,000 with 4,000 label rows: GEMM / perm-block = 1.62 at K = 16,
    // 1.22 at 20, 1.10 at 22, 1.01 at 24, 0.90 at 26, 0.78 at 32.
    if (gemm_available() && K <= 24 && n >= 256 && P >= 32) pl.form = PERMANOVA_FORM_GEMM;
    else if (P >= 16 && K <= 65536) pl.form = PERMANOVA_FORM_PERMBLOCK;
    else pl.form = PERMANOVA_FORM_BRUTE;
    return pl;
}

Plan plan_of_form(int form) {
    Plan pl;
    pl.form = form;
    return pl;
}

int plan_form(const permanova_ctx* ctx, uint32_t n, uint32_t K, uint64_t P) {
    return plan_for(ctx, n, K, P).form;
}

int layout_for(const permanova_ctx* ctx, const Plan& plan_in, uint32_t n, uint64_t ld, const void* labels,
               int label_type, uint32_t K, uint64_t P, SWLayout* L) {
    const Plan plan = plan_in;   // a copy: plan_in may be L->plan, reset on the next line
    *L = SWLayout{};
    const int form = plan.form;
    L->form = form;
    L->plan = plan;
    size_t off = 0;
    if (form == PERMANOVA_FORM_BRUTE) {
        L->part_rows = brute_chunks(n, ctx->sm_count, plan.brute_mult);
    } else if (form == PERMANOVA_FORM_PERMBLOCK) {
        if (K > 65536)
            return fail(PERMANOVA_EUNSUPPORTED, "perm-block form needs n_groups <= 65536 (got %u)", K);
        L->part_rows = permblock_bands(n);
        L->code_type = K <= 256 ? LABEL_U8 : LABEL_U16;
        const bool direct = labels != nullptr && (label_type == L->code_type) &&
                            ((uint64_t)n * label_bytes(label_type)) % 16 == 0 &&
                            ((uintptr_t)labels % 16 == 0);
        L->repack = !direct;
        L->lstride = direct ? n : (uint64_t)align_up(n, 64);
    } else if (form == PERMANOVA_FORM_GEMM) {
        if (!gemm_available()) return fail(PERMANOVA_EUNSUPPORTED, "GEMM form not built");
        if (K > 256) return fail(PERMANOVA_EUNSUPPORTED, "GEMM form needs n_groups <= 256 (got %u)", K);
        if (n < 2) return fail(PERMANOVA_EINVAL, "n_dims < 2");
        const GemmPlan gp = gemm_plan(n, K, P, plan.gemm_ppt_div);
        L->part_rows = gp.n_bands;
        L->code_type = LABEL_U8;
        L->repack = true;  // the GEMM form reads 16-byte aligned, zero-padded uint8 rows
        L->lstride = gp.n_pad;
    } else {
        return fail(PERMANOVA_EINVAL, "unknown form %d", form);
    }
    (void)ld;
    L->part_off = off;
    off = align_up(off + (size_t)L->part_rows * P * sizeof(double));
    if (L->repack) {
        L->lab_off = off;
        const size_t lab = form == PERMANOVA_FORM_GEMM
                               ? gemm_label_bytes(gemm_plan(n, K, P, plan.gemm_ppt_div))
                               : (size_t)L->lstride * P * label_bytes(L->code_type);
        off = align_up(off + lab);
    }
    if (form == PERMANOVA_FORM_GEMM) {
        const GemmPlan gp = gemm_plan(n, K, P, plan.gemm_ppt_div);
        L->counter_off = off;
        off = align_up(off + kGemmWorkCounters * sizeof(unsigned long long));
        L->gemm_off = off;
        if (!plan.prepared) off = align_up(off + gemm_scratch_bytes(gp, P));
    }
    L->w_off = off;   // K doubles
    off = align_up(off + (size_t)K * sizeof(double));
    L->total = off;
    return PERMANOVA_OK;
}

// Make the arena at least `bytes`.  Growing waits for all device work (the
// old arena may still be in use) before it is replaced.
int ensure_arena(permanova_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->arena_size) return PERMANOVA_OK;
    if (bytes > ctx->budget)
        return fail(PERMANOVA_ENOMEM, "scratch of %zu bytes exceeds the context budget of %zu bytes",
                    bytes, ctx->budget);
    size_t want = std::min(ctx->budget, std::max(bytes, ctx->arena_size + ctx->arena_size / 4));
    CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    // captured graphs point into the old arena
    for (auto& kv : ctx->graph_cache) cudaGraphExecDestroy(kv.second.exec);
    ctx->graph_cache.clear();
    if (ctx->arena) {
        cudaFree(ctx->arena);
        ctx->arena = nullptr;
        ctx->arena_size = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess && want > bytes) {
        cudaGetLastError();
        want = bytes;
        e = cudaMalloc(&p, want);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(scratch)");
    ctx->arena = p;
    ctx->arena_size = want;
    return PERMANOVA_OK;
}

int check_sW_args(const float* mat, uint32_t n, uint64_t ld, const void* labels, int label_type,
                  uint32_t K, uint64_t P, const float* w, const double* out) {
    if (!mat || !labels || !w || !out) return fail(PERMANOVA_EINVAL, "NULL pointer argument");
    if (n < 2) return fail(PERMANOVA_EINVAL, "n_dims must be >= 2 (got %u)", n);
    if (ld < n) return fail(PERMANOVA_EINVAL, "ld (%llu) < n_dims (%u)", (unsigned long long)ld, n);
    if (K == 0) return fail(PERMANOVA_EINVAL, "n_groups must be >= 1");
    if (P == 0) return fail(PERMANOVA_EINVAL, "n_perms must be >= 1");
    if (label_type != LABEL_I32 && label_type != LABEL_U16 && label_type != LABEL_U8)
        return fail(PERMANOVA_EINVAL, "unknown label type %d", label_type);
    if (label_type == LABEL_U8 && K > 256)
        return fail(PERMANOVA_EINVAL, "uint8 labels hold at most 256 groups (n_groups = %u)", K);
    if (label_type == LABEL_U16 && K > 65536)
        return fail(PERMANOVA_EINVAL, "uint16 labels hold at most 65536 groups (n_groups = %u)", K);
    return PERMANOVA_OK;
}

// Events around the dominant kernel of an s_W call (profiling only).
int profile_begin(permanova_ctx* ctx, cudaStream_t s) {
    if (!ctx->profiling) return PERMANOVA_OK;
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a), "cudaEventCreate");
    CK(cudaEventCreate(&b), "cudaEventCreate");
    ctx->events.emplace_back(a, b);
    CK(cudaEventRecord(a, s), "cudaEventRecord");
    return PERMANOVA_OK;
}

int profile_end(permanova_ctx* ctx, cudaStream_t s) {
    if (!ctx->profiling || ctx->events.empty()) return PERMANOVA_OK;
    CK(cudaEventRecord(ctx->events.back().second, s), "cudaEventRecord");
    return PERMANOVA_OK;
}

void profile_clear(permanova_ctx* ctx) {
    for (auto& e : ctx->events) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    ctx->events.clear();
    for (auto& h : ctx->host_events)
        for (cudaEvent_t e : h) cudaEventDestroy(e);
    ctx->host_events.clear();
    for (auto& v : ctx->host_seg_events)
        for (cudaEvent_t e : v) cudaEventDestroy(e);
    ctx->host_seg_events.clear();
    ctx->host_h2d_bytes = 0;
    ctx->launch_mark = kernel_launch_count();
}

// Inputs that arrive on the device while the path runs (host entry point):
// segment k covers the 128-row bands [band[k], band[k+1]) of D and is on the
// device once seg_ready[k] has fired; labels and weights once lab_ready has.
// With the tensor-core form, issue_copy(k) queues segment k's copies (called
// just before the segment's kernels are queued, so it can wait for the
// preparation that last read its staging slot, prep_done[k - slots]), and
// segment k sits in the band-flat layout at slot_mat[k % slots].
struct Arrival {
    cudaEvent_t lab_ready = nullptr;
    std::vector<uint32_t> band;
    std::vector<cudaEvent_t> seg_ready;
    cudaStream_t s2 = nullptr;                 // second stream for odd segments
    cudaEvent_t fork = nullptr, join = nullptr;
    std::function<cudaError_t(size_t)> issue_copy;
    std::vector<const float*> slot_mat;
    std::vector<cudaEvent_t> prep_done;
    // timing events (profiling only, else empty): segment k landed, and its
    // dominant kernel done
    std::vector<cudaEvent_t> t_landed, t_done;
};

// The s_W path on device buffers; the arena is already large enough.
// `wf` (device fp32 inv_group_sizes) is widened into the layout's FP64 slot;
// with wf == NULL, pr.w (FP64, possibly several weight sets) is used, or the
// layout's slot when pr.w is NULL.  With `arr`, each step waits for the inputs
// it reads; the GEMM form then prepares and runs band segment k as soon as
// segment k has arrived, so the copies of later segments overlap the tensor-core
// work on earlier ones.
int run_sW(permanova_ctx* ctx, const SWLayout& L, SWProblem pr, const float* wf, cudaStream_t s,
           const Arrival* arr = nullptr, const void* prepared_ops = nullptr) {
    char* base = static_cast<char*>(ctx->arena);
    if (arr) CK(cudaStreamWaitEvent(s, arr->lab_ready, 0), "wait for labels");
    // all of D: the CUDA-core forms read every band in one launch
    auto wait_all_rows = [&]() -> cudaError_t {
        return arr ? cudaStreamWaitEvent(s, arr->seg_ready.back(), 0) : cudaSuccess;
    };
    double* partials = reinterpret_cast<double*>(base + L.part_off);
    double* wd = reinterpret_cast<double*>(base + L.w_off);
    if (wf) {
        CK(launch_widen(wf, pr.K, wd, s), "widen weights");
        pr.w = wd;
    } else if (!pr.w) {
        pr.w = wd;
    }
    SWProblem q = pr;
    if (L.form == PERMANOVA_FORM_BRUTE) {
        CK(launch_validate_labels(pr.labels, pr.label_type, (uint64_t)pr.n * pr.P, pr.K, ctx->status, s),
           "validate labels");
        CK(wait_all_rows(), "wait for the matrix");
        int rc = profile_begin(ctx, s);
        if (rc) return rc;
        CK(launch_brute(pr, L.part_rows, partials, ctx->status, s), "brute-force kernel");
        rc = profile_end(ctx, s);
        if (rc) return rc;
        if (arr && !arr->t_done.empty()) CK(cudaEventRecord(arr->t_done[0], s), "record kernel done");
    } else {
        if (L.repack) {
            void* codes = base + L.lab_off;
            if (L.form == PERMANOVA_FORM_GEMM)
                CK(launch_repack_gemm(pr.labels, pr.label_type, pr.n, pr.P, pr.K,
                                      gemm_plan(pr.n, pr.K, pr.P, L.plan.gemm_ppt_div),
                                      codes, ctx->status, s),
                   "repack labels");
            else
                CK(launch_repack_labels(pr.labels, pr.label_type, pr.n, pr.P, pr.K, codes, L.code_type,
                                        L.lstride, ctx->status, s),
                   "repack labels");
            q.labels = codes;
            q.label_type = L.code_type;
        } else {
            CK(launch_validate_labels(pr.labels, pr.label_type, (uint64_t)pr.n * pr.P, pr.K,
                                      ctx->status, s),
               "validate labels");
        }
        if (L.form == PERMANOVA_FORM_PERMBLOCK) {
            CK(wait_all_rows(), "wait for the matrix");
            int rc = profile_begin(ctx, s);
            if (rc) return rc;
            CK(launch_permblock_internal(q, L.lstride, partials, ctx->status, s, L.plan.pb_variant),
               "perm-block kernel");
            rc = profile_end(ctx, s);
            if (rc) return rc;
            if (arr && !arr->t_done.empty()) CK(cudaEventRecord(arr->t_done[0], s), "record kernel done");
        } else {
            const GemmPlan gp = gemm_plan(pr.n, pr.K, pr.P, L.plan.gemm_ppt_div);
            // the operands: prepared once for this matrix, or made now in the scratch
            void* gs = prepared_ops ? const_cast<void*>(prepared_ops) : base + L.gemm_off;
            unsigned long long* counters = reinterpret_cast<unsigned long long*>(base + L.counter_off);
            if (!arr) {
                if (!prepared_ops) CK(launch_gemm_prep(q, gp, gs, s), "GEMM operand preparation");
                CK(cudaMemsetAsync(counters, 0, sizeof(unsigned long long), s), "reset the work counter");
                int rc = profile_begin(ctx, s);
                if (rc) return rc;
                CK(launch_gemm_main(q, gp, gs, partials, ctx->status, ctx->sm_count, s, 0, 0xFFFFFFFFu,
                                    L.plan.gemm_drain, counters),
                   "GEMM kernel");
                rc = profile_end(ctx, s);
                if (rc) return rc;
            } else {
                // segments alternate between s and s2 (disjoint bands: disjoint tiles,
                // band words and partial rows), so a segment's last wave overlaps the
                // next segment's first; s2 starts after everything queued on s so far
                // and s continues after all of s2's work
                // one work counter per segment launch, all zeroed before the fork
                if (arr->band.size() - 1 > kGemmWorkCounters) return fail(PERMANOVA_EINVAL, "too many segments");
                CK(cudaMemsetAsync(counters, 0, (arr->band.size() - 1) * sizeof(unsigned long long), s),
                   "reset the work counters");
                CK(cudaEventRecord(arr->fork, s), "fork segment streams");
                CK(cudaStreamWaitEvent(arr->s2, arr->fork, 0), "fork segment streams");
                for (size_t k = 0; k + 1 < arr->band.size(); ++k) {
                    cudaStream_t sk = (k & 1) ? arr->s2 : s;
                    if (arr->issue_copy) CK(arr->issue_copy(k), "copy a matrix segment");
                    CK(cudaStreamWaitEvent(sk, arr->seg_ready[k], 0), "wait for a matrix segment");
                    SWProblem qk = q;   // segment k's bands, in its staging slot
                    if (!arr->slot_mat.empty()) {
                        qk.mat = arr->slot_mat[k % arr->slot_mat.size()];
                        qk.banded = 1;
                        qk.band0 = arr->band[k];
                    }
                    CK(launch_gemm_prep(qk, gp, gs, sk, arr->band[k], arr->band[k + 1]),
                       "GEMM operand preparation");
                    if (!arr->prep_done.empty())
                        CK(cudaEventRecord(arr->prep_done[k], sk), "record a segment's preparation");
                    CK(launch_gemm_main(q, gp, gs, partials, ctx->status, ctx->sm_count, sk, arr->band[k],
                                        arr->band[k + 1], L.plan.gemm_drain, counters + k),
                       "GEMM kernel");
                    if (!arr->t_done.empty()) CK(cudaEventRecord(arr->t_done[k], sk), "record kernel done");
                }
                CK(cudaEventRecord(arr->join, arr->s2), "join segment streams");
                CK(cudaStreamWaitEvent(s, arr->join, 0), "join segment streams");
            }
        }
    }
    CK(launch_reduce_rows(partials, L.part_rows, pr.P, pr.out, s), "reduce partials");
    ctx->last_form = L.form;
    return PERMANOVA_OK;
}

int read_status(permanova_ctx* ctx, cudaStream_t s) {
    CK(cudaMemcpyAsync(ctx->status_host, ctx->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s),
       "read device status");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    DevStatus h = *ctx->status_host;
    if (h.code == DEV_OK) return PERMANOVA_OK;
    CK(cudaMemsetAsync(ctx->status, 0, sizeof(DevStatus), s), "reset device status");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (h.code == DEV_BAD_LABEL)
        return fail(PERMANOVA_EINVAL, "label >= n_groups at flat index %llu", h.info);
    if (h.code == DEV_TIMEOUT)
        return fail(PERMANOVA_ETIMEOUT, "device wait timed out (kernel stage %u, detail %llu)", h.where,
                    h.info);
    return fail(PERMANOVA_ECUDA, "device error code %u", h.code);
}

}  // namespace

void pmn::set_last_error(const char* msg) { tl_err = msg; }

extern "C" {

int permanova_create(int device, size_t hbm_budget_bytes, permanova_ctx** out) {
    if (!out) return fail(PERMANOVA_EINVAL, "out is NULL");
    *out = nullptr;
    int count = 0;
    CK(cudaGetDeviceCount(&count), "cudaGetDeviceCount");
    if (device < 0 || device >= count)
        return fail(PERMANOVA_EINVAL, "device %d out of range (%d devices)", device, count);
    DeviceGuard g(device);
    if (!g.ok) return fail(PERMANOVA_ECUDA, "cannot select device %d", device);
    auto* ctx = new permanova_ctx();
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : fr / 10 * 9;
    cudaError_t e = cudaMalloc(&ctx->status, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->status_host, sizeof(DevStatus));
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "context allocation");
        permanova_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return PERMANOVA_OK;
}

void permanova_destroy(permanova_ctx* ctx) {
    if (!ctx) return;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        profile_clear(ctx);
        for (auto& kv : ctx->graph_cache) cudaGraphExecDestroy(kv.second.exec);
        ctx->graph_cache.clear();
        if (ctx->arena) cudaFree(ctx->arena);
        for (cudaEvent_t e : ctx->copy_events) cudaEventDestroy(e);
        if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
        if (ctx->seg_fork) cudaEventDestroy(ctx->seg_fork);
        if (ctx->seg_join) cudaEventDestroy(ctx->seg_join);
        if (ctx->seg_stream) cudaStreamDestroy(ctx->seg_stream);
        if (ctx->status) cudaFree(ctx->status);
        if (ctx->status_host) cudaFreeHost(ctx->status_host);
    }
    delete ctx;
}

const char* permanova_last_error(const permanova_ctx*) { return tl_err.c_str(); }

int permanova_set_form(permanova_ctx* ctx, int form) {
    if (!ctx) return fail(PERMANOVA_EINVAL, "ctx is NULL");
    if (form < PERMANOVA_FORM_AUTO || form > PERMANOVA_FORM_GEMM)
        return fail(PERMANOVA_EINVAL, "unknown form %d", form);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->forced_form = form;
    ctx->forced_plan = plan_of_form(form);
    return PERMANOVA_OK;
}

int permanova_set_plan(permanova_ctx* ctx, const permanova_plan_t* plan) {
    if (!ctx) return fail(PERMANOVA_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!plan || plan->form == PERMANOVA_FORM_AUTO) {
        ctx->forced_form = PERMANOVA_FORM_AUTO;
        ctx->forced_plan = Plan{};
        return PERMANOVA_OK;
    }
    if (plan->form < PERMANOVA_FORM_BRUTE || plan->form > PERMANOVA_FORM_GEMM)
        return fail(PERMANOVA_EINVAL, "unknown form %d", plan->form);
    if (plan->permblock_variant < 0 || plan->permblock_variant > 2)
        return fail(PERMANOVA_EINVAL, "perm-block variant must be 0, 1 or 2");
    if (plan->gemm_rows_div != 0 && plan->gemm_rows_div != 1 && plan->gemm_rows_div != 2 &&
        plan->gemm_rows_div != 4)
        return fail(PERMANOVA_EINVAL, "gemm_rows_div must be 1, 2 or 4");
    if (plan->gemm_drain_kblocks > 8)
        return fail(PERMANOVA_EINVAL, "gemm_drain_kblocks above 8 breaks the 1e-5 accuracy target");
    if (plan->brute_chunk_mult > 16) return fail(PERMANOVA_EINVAL, "brute_chunk_mult must be <= 16");
    Plan pl = plan_of_form(plan->form);
    pl.pb_variant = plan->permblock_variant;
    pl.gemm_ppt_div = plan->gemm_rows_div ? plan->gemm_rows_div : 1;
    pl.gemm_drain = plan->gemm_drain_kblocks;
    pl.brute_mult = plan->brute_chunk_mult ? plan->brute_chunk_mult : 1;
    ctx->forced_form = plan->form;
    ctx->forced_plan = pl;
    return PERMANOVA_OK;
}

int permanova_plan_form(permanova_ctx* ctx, uint32_t n, uint32_t K, uint64_t P) {
    if (!ctx) return fail(PERMANOVA_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    return plan_form(ctx, n, K, P);
}

size_t permanova_scratch_bytes(permanova_ctx* ctx, int form, uint32_t n, uint32_t K, uint64_t P) {
    if (!ctx || n < 2 || K == 0 || P == 0) return 0;
    std::lock_guard<std::mutex> lk(ctx->mu);
    const Plan pl = form == PERMANOVA_FORM_AUTO ? plan_for(ctx, n, K, P) : plan_of_form(form);
    SWLayout L;
    // worst case: labels need a repack
    if (layout_for(ctx, pl, n, n, nullptr, LABEL_I32, K, P, &L) != PERMANOVA_OK) return 0;
    return L.total;
}

size_t permanova_scratch_reserved(permanova_ctx* ctx) {
    if (!ctx) return 0;
    std::lock_guard<std::mutex> lk(ctx->mu);
    return ctx->arena_size;
}

int permanova_reserve_scratch(permanova_ctx* ctx, size_t bytes) {
    if (!ctx) return fail(PERMANOVA_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    return ensure_arena(ctx, bytes);
}

int permanova_release_scratch(permanova_ctx* ctx) {
    if (!ctx) return fail(PERMANOVA_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    for (auto& kv : ctx->graph_cache) cudaGraphExecDestroy(kv.second.exec);
    ctx->graph_cache.clear();
    if (ctx->arena) CK(cudaFree(ctx->arena), "cudaFree(scratch)");
    ctx->arena = nullptr;
    ctx->arena_size = 0;
    return PERMANOVA_OK;
}

int permanova_sW(permanova_ctx* ctx, const float* mat, uint32_t n, uint64_t ld, const void* groupings,
                 int label_type, uint32_t K, uint64_t P, const float* w, double* out, void* stream) {
    if (!ctx) return fail(PERMANOVA_EINVAL, "ctx is NULL");
    int rc = check_sW_args(mat, n, ld, groupings, label_type, K, P, w, out);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SWLayout L;
    rc = layout_for(ctx, plan_for(ctx, n, K, P), n, ld, groupings, label_type, K, P, &L);
    if (rc) return rc;
    rc = ensure_arena(ctx, L.total);
    if (rc) return rc;
    SWProblem pr{mat, n, ld, groupings, label_type, K, P, nullptr, out};
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const bool use_graph = ctx->graphs && !ctx->profiling && s != nullptr &&
                           cudaStreamIsCapturing(s, &cap) == cudaSuccess &&
                           cap == cudaStreamCaptureStatusNone;
    if (!use_graph) return run_sW(ctx, L, pr, w, s);
    // replay the launch sequence of an identical earlier call, or capture it now
    const int plan_code = L.form + 8 * (L.plan.pb_variant + 2 * ((int)L.plan.gemm_ppt_div +
                                                          16 * ((int)L.plan.gemm_drain + 64 * (int)L.plan.brute_mult)));
    const GraphKey key{mat, n, ld, groupings, label_type, K, P, w, out, ctx->arena, plan_code, nullptr};
    auto it = ctx->graph_cache.find(key);
    bool fresh = false;
    if (it == ctx->graph_cache.end()) {
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        const uint64_t before = kernel_launch_count();
        rc = run_sW(ctx, L, pr, w, s);
        const uint64_t captured = kernel_launch_count() - before;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        it = ctx->graph_cache.emplace(key, permanova_ctx::CachedGraph{exec, captured}).first;
        fresh = true;
    }
    CK(cudaGraphLaunch(it->second.exec, s), "cudaGraphLaunch");
    // the capture counted its kernels once (for this first launch); replays count them again
    if (!fresh) note_launches((unsigned)it->second.kernels);
    return PERMANOVA_OK;
}

int permanova_selftest_wait(permanova_ctx* ctx, uint32_t limit_us, void* stream) {
    if (!ctx) return fail(PERMANOVA_EINVAL, "ctx is NULL");
    if (limit_us == 0 || limit_us > 10000000u) return fail(PERMANOVA_EINVAL, "limit_us out of range");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    int khz = 0;
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device);
    const long long cycles = (long long)limit_us * (khz > 0 ? khz : 2000000) / 1000;
    CK(launch_wait_selftest(ctx->status, cycles, static_cast<cudaStream_t>(stream)), "wait self-test");
    return PERMANOVA_OK;
}

int permanova_set_graphs(permanova_ctx* ctx, int enable) {
    if (!ctx) return fail(PERMANOVA_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    ctx->graphs = enable != 0;
    if (!ctx->graphs) {
        CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
        for (auto& kv : ctx->graph_cache) cudaGraphExecDestroy(kv.second.exec);
        ctx->graph_cache.clear();
    }
    return PERMANOVA_OK;
}

int permanova_autotune(permanova_ctx* ctx, const float* mat, uint32_t n, uint64_t ld,
                       const void* groupings, int label_type, uint32_t K, uint64_t P, const float* w,
                       int* out_form, void* stream) {
    if (!ctx) return fail(PERMANOVA_EINVAL, "ctx is NULL");
    const double no_output = 0.0;   // the sample's results go to scratch
    int rc = check_sW_args(mat, n, ld, groupings, label_type, K, P, w, &no_output);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // a sample of the caller's label rows sized to ~4e12 pair evaluations
    // (about 0.1 s of the tensor-core form), at least 64 rows, at most 4,096
    const double pairs = (double)n * (n - 1) / 2.0;
    uint64_t Ps = (uint64_t)std::max(64.0, 4e12 / std::max(pairs, 1.0));
    Ps = std::min<uint64_t>(Ps, std::min<uint64_t>(P, 4096));
    // candidate plans: every form with its knobs.  The drain interval of the
    // tensor-core form stays at 8 k-blocks or fewer, the accuracy limit of the
    // 1e-5 target (the worst case measured at 8 is 5.2e-6).
    std::vector<Plan> cands;
    for (uint32_t mult : {1u, 2u}) {
        Plan pl = plan_of_form(PERMANOVA_FORM_BRUTE);
        pl.brute_mult = mult;
        cands.push_back(pl);
    }
    for (int var : {0, 2, 1}) {
        if (var != 1 && K > 2048) continue;   // the paired kernel holds up to 2,048 weights
        Plan pl = plan_of_form(PERMANOVA_FORM_PERMBLOCK);
        pl.pb_variant = var;
        cands.push_back(pl);
    }
    for (uint32_t div : {1u, 2u})
        for (uint32_t drain : {8u, 4u}) {
            Plan pl = plan_of_form(PERMANOVA_FORM_GEMM);
            pl.gemm_ppt_div = div;
            pl.gemm_drain = drain;
            cands.push_back(pl);
        }
    double best_t = 1e300;
    Plan best = plan_of_form(PERMANOVA_FORM_BRUTE);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0), "cudaEventCreate");
    if (cudaError_t e = cudaEventCreate(&e1); e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(e, "cudaEventCreate");
    }
    for (const Plan& pl : cands) {
        // the brute force re-reads D per label row: skip it where it cannot win
        if (pl.form == PERMANOVA_FORM_BRUTE && Ps > 64 && pairs * Ps > 4e11) continue;
        SWLayout L;
        if (layout_for(ctx, pl, n, ld, groupings, label_type, K, Ps, &L) != PERMANOVA_OK) continue;
        const size_t out_off = align_up(L.total);
        if (ensure_arena(ctx, out_off + (size_t)Ps * sizeof(double)) != PERMANOVA_OK) continue;
        double* out = reinterpret_cast<double*>(static_cast<char*>(ctx->arena) + out_off);
        SWProblem pr{mat, n, ld, groupings, label_type, K, Ps, nullptr, out};
        float ms = 0.f;
        bool ok = run_sW(ctx, L, pr, w, s) == PERMANOVA_OK;   // warm-up
        ok = ok && cudaEventRecord(e0, s) == cudaSuccess;
        ok = ok && run_sW(ctx, L, pr, w, s) == PERMANOVA_OK;
        ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
             cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (ok && ms < best_t) {
            best_t = ms;
            best = pl;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    rc = read_status(ctx, s);
    if (rc) return rc;
    best.tuned = true;
    ctx->tuned[TuneKey{log2_bucket(n), K, log2_bucket(P)}] = best;
    if (out_form) *out_form = best.form;
    return PERMANOVA_OK;
}

int permanova_plan_describe(permanova_ctx* ctx, uint32_t n, uint32_t K, uint64_t P, char* out, size_t cap) {
    if (!ctx || !out || cap == 0) return fail(PERMANOVA_EINVAL, "NULL argument");
    if (n < 2 || K == 0 || P == 0) return fail(PERMANOVA_EINVAL, "invalid sizes");
    std::lock_guard<std::mutex> lk(ctx->mu);
    const Plan pl = plan_for(ctx, n, K, P);
    const char* src = ctx->forced_form != PERMANOVA_FORM_AUTO ? "forced" : pl.tuned ? "autotuned" : "rule";
    int m = 0;
    if (pl.form == PERMANOVA_FORM_GEMM) {
        const GemmPlan gp = gemm_plan(n, K, P, pl.gemm_ppt_div);
        m = snprintf(out, cap,
                     "{\"form\": \"gemm\", \"source\": \"%s\", \"label_rows_per_tile\": %u, "
                     "\"mma_n\": %u, \"drain_kblocks\": %u, \"band_rows\": 128, \"kblock_cols\": 64}",
                     src, gp.perms_per_tile, (gp.perms_per_tile * K + 15) / 16 * 16,
                     pl.gemm_drain ? pl.gemm_drain : 8u);
    } else if (pl.form == PERMANOVA_FORM_PERMBLOCK) {
        const bool pair = pl.pb_variant != 1 && K <= 256;
        m = snprintf(out, cap,
                     "{\"form\": \"permblock\", \"source\": \"%s\", \"variant\": \"%s\", "
                     "\"label_rows_per_block\": %u, \"tile\": 64}",
                     src, !pair ? "f32 compare-and-set" : pl.pb_variant == 2 ? "paired f16x2 compare, 4 CTAs/SM"
                                                                          : "paired f16x2 compare, 3 CTAs/SM",
                     pair ? 256u : 128u);
    } else {
        m = snprintf(out, cap, "{\"form\": \"brute\", \"source\": \"%s\", \"chunks_per_row\": %u}", src,
                     brute_chunks(n, ctx->sm_count, pl.brute_mult));
    }
    if (m < 0 || (size_t)m >= cap) return fail(PERMANOVA_EINVAL, "buffer too small");
    return PERMANOVA_OK;
}

int permanova_profile_enable(permanova_ctx* ctx, int enable) {
    if (!ctx) return fail(PERMANOVA_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    profile_clear(ctx);
    ctx->profiling = enable != 0;
    return PERMANOVA_OK;
}

int permanova_profile_read(permanova_ctx* ctx, permanova_profile_t* out) {
    if (!ctx || !out) return fail(PERMANOVA_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    double ms = 0.0;
    for (auto& e : ctx->events) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e.first, e.second), "cudaEventElapsedTime");
        ms += t;
    }
    out->main_kernel_ms = ms;
    out->main_kernel_launches = ctx->events.size();
    out->host_calls = ctx->host_events.size();
    out->host_total_ms = out->host_first_segment_ms = out->host_copy_ms = 0.0;
    for (auto& h : ctx->host_events) {
        float a = 0.f, b = 0.f, c = 0.f;
        CK(cudaEventElapsedTime(&a, h[0], h[1]), "cudaEventElapsedTime");
        CK(cudaEventElapsedTime(&b, h[0], h[2]), "cudaEventElapsedTime");
        CK(cudaEventElapsedTime(&c, h[0], h[3]), "cudaEventElapsedTime");
        out->host_first_segment_ms += a;
        out->host_copy_ms += b;
        out->host_total_ms += c;
    }
    out->host_segments = 0;
    for (int k = 0; k < 16; ++k) out->host_seg_landed_ms[k] = out->host_seg_done_ms[k] = 0.0;
    for (size_t c = 0; c < ctx->host_seg_events.size() && c < ctx->host_events.size(); ++c) {
        const auto& v = ctx->host_seg_events[c];
        const size_t m = v.size() / 2;
        out->host_segments = (uint32_t)m;
        for (size_t k = 0; k < m && k < 16; ++k) {
            float a = 0.f, b = 0.f;
            CK(cudaEventElapsedTime(&a, ctx->host_events[c][0], v[k]), "cudaEventElapsedTime");
            CK(cudaEventElapsedTime(&b, ctx->host_events[c][0], v[m + k]), "cudaEventElapsedTime");
            out->host_seg_landed_ms[k] += a;
            out->host_seg_done_ms[k] += b;
        }
    }
    out->host_h2d_bytes = ctx->host_h2d_bytes;
    out->kernel_launches = kernel_launch_count() - ctx->launch_mark;
    out->last_form = ctx->last_form;
    profile_clear(ctx);
    return PERMANOVA_OK;
}

int permanova_sync(permanova_ctx* ctx, void* stream) {
    if (!ctx) return fail(PERMANOVA_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    return read_status(ctx, static_cast<cudaStream_t>(stream));
}

// Whether the host entry copies band I of an n-object matrix as a
// two-dimensional copy of its trapezoid (rows 128 I .., columns 128 I .. n-1)
// rather than as its flat host range: when the trapezoid's rows are under half
// the matrix width.
static bool host_band_2d(uint64_t n, uint64_t I) { return 2 * (n - 128 * I) < n; }

int permanova_sW_host(permanova_ctx* ctx, const float* mat, uint32_t n, uint64_t ld,
                      const void* groupings, int label_type, uint32_t K, uint64_t P, const float* w,
                      double* out, void* stream) {
    if (!ctx) return fail(PERMANOVA_EINVAL, "ctx is NULL");
    int rc = check_sW_args(mat, n, ld, groupings, label_type, K, P, w, out);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SWLayout L;
    rc = layout_for(ctx, plan_for(ctx, n, K, P), n, ld, nullptr, label_type, K, P, &L);
    if (rc) return rc;
    // Staging for the inputs and the output after the s_W scratch.  The
    // tensor-core form reads D only through its band trapezoids and gets them
    // in the band-flat layout (band I = the host range from element (128 I,
    // 128 I) to the end of its last row, row stride ld) in one of kHostSlots
    // staging slots; the prep kernel of its segment reads it there, so the
    // device holds kHostSlots segments of D, not all of it.  A band whose
    // trapezoid is at least half its flat range comes in one flat copy (the
    // rows' lower-left parts come along); a later band, whose rows are mostly
    // left of the diagonal, comes in one two-dimensional copy of its
    // trapezoid into the same layout (two-dimensional copies out of
    // page-locked host memory ran at about 120 against 210 GB/s for flat
    // ones, so they pay only where they move under half the bytes).  The
    // CUDA-core forms get the whole matrix in one flat copy (row stride ld).
    const bool gemm = L.form == PERMANOVA_FORM_GEMM;
    const uint32_t n_bands = (n + 127) / 128;
    const uint32_t n_seg = gemm ? std::min<uint32_t>(kHostSegments, n_bands) : 1u;
    // segment boundaries: the first segments small (band counts in the ratio
    // 1 : 2 : 4 : 8 : 8 : ...), so the kernels start after a short copy and each
    // early segment's kernels cover the next one's copy; the copies move about
    // the same bytes per band
    std::vector<uint32_t> seg_band(n_seg + 1, 0);
    {
        std::vector<uint64_t> cum(n_seg + 1, 0);
        for (uint32_t k = 0; k < n_seg; ++k) cum[k + 1] = cum[k] + (k < 3 ? (1ull << k) : 8ull);
        for (uint32_t k = 1; k <= n_seg; ++k) {
            uint32_t b = (uint32_t)((n_bands * cum[k] + cum[n_seg] / 2) / cum[n_seg]);
            b = std::max(b, seg_band[k - 1] + 1);                // every segment has a band
            seg_band[k] = std::min(b, n_bands - (n_seg - k));    // and leaves one for each after it
        }
    }
    auto seg_floats = [&](uint32_t k) -> uint64_t {   // floats of segment k's bands, band-flat
        const uint32_t last = seg_band[k + 1] - 1;
        return band_flat_offset(last, ld, n) - band_flat_offset(seg_band[k], ld, n) + band_flat_floats(last, ld, n);
    };
    uint64_t slot_floats = 0;
    if (gemm)
        for (uint32_t k = 0; k < n_seg; ++k) slot_floats = std::max(slot_floats, seg_floats(k));
    const uint32_t n_slots = gemm ? std::min<uint32_t>(kHostSlots, n_seg) : 1u;
    const size_t slot_bytes = align_up((gemm ? slot_floats : (uint64_t)(n - 1) * ld + n) * sizeof(float));
    const size_t lab_bytes = (size_t)n * P * label_bytes(label_type);
    size_t off = L.total;
    const size_t mat_off = off;
    off = align_up(off + slot_bytes * n_slots);
    const size_t lab_off = off;
    off = align_up(off + lab_bytes);
    const size_t w_off = off;
    off = align_up(off + (size_t)K * sizeof(float));
    const size_t out_off = off;
    off = align_up(off + (size_t)P * sizeof(double));
    rc = ensure_arena(ctx, off);
    if (rc) return rc;
    char* base = static_cast<char*>(ctx->arena);

    if (!ctx->copy_stream)
        CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking), "create copy stream");
    if (!ctx->seg_stream)
        CK(cudaStreamCreateWithFlags(&ctx->seg_stream, cudaStreamNonBlocking), "create segment stream");
    if (!ctx->seg_fork) CK(cudaEventCreateWithFlags(&ctx->seg_fork, cudaEventDisableTiming), "create event");
    if (!ctx->seg_join) CK(cudaEventCreateWithFlags(&ctx->seg_join, cudaEventDisableTiming), "create event");
    while (ctx->copy_events.size() < 2 * kHostSegments + 2) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "create copy event");
        ctx->copy_events.push_back(e);
    }
    // profiling: timing events at the start, first segment, last segment and end,
    // and per segment when it landed and when its dominant kernel had run
    std::array<cudaEvent_t, 4> tev{};
    if (ctx->profiling) {
        for (auto& e : tev) {
            if (cudaError_t ce = cudaEventCreate(&e); ce != cudaSuccess) {
                for (cudaEvent_t x : tev)
                    if (x) cudaEventDestroy(x);
                return cuda_fail(ce, "cudaEventCreate");
            }
        }
        ctx->host_events.push_back(tev);
        std::vector<cudaEvent_t> sev(2 * (size_t)n_seg, nullptr);
        for (auto& e : sev) {
            if (cudaError_t ce = cudaEventCreate(&e); ce != cudaSuccess) {
                for (cudaEvent_t x : sev)
                    if (x) cudaEventDestroy(x);
                ctx->host_seg_events.emplace_back();   // keeps the two lists aligned
                return cuda_fail(ce, "cudaEventCreate");
            }
        }
        ctx->host_seg_events.push_back(sev);
        ctx->host_h2d_bytes += lab_bytes + (size_t)K * sizeof(float);
        CK(cudaEventRecord(tev[0], s), "record start");
    }
    cudaStream_t cs = ctx->copy_stream;
    Arrival arr;
    arr.lab_ready = ctx->copy_events[0];
    arr.s2 = ctx->seg_stream;
    arr.fork = ctx->seg_fork;
    arr.join = ctx->seg_join;
    cudaEvent_t start = ctx->copy_events[1];
    CK(cudaEventRecord(start, s), "record start");
    CK(cudaStreamWaitEvent(cs, start, 0), "order copies after earlier work");
    CK(cudaMemcpyAsync(base + lab_off, groupings, lab_bytes, cudaMemcpyHostToDevice, cs), "copy labels");
    CK(cudaMemcpyAsync(base + w_off, w, (size_t)K * sizeof(float), cudaMemcpyHostToDevice, cs),
       "copy weights");
    CK(cudaEventRecord(arr.lab_ready, cs), "record labels");
    float* dmat = reinterpret_cast<float*>(base + mat_off);
    arr.band = seg_band;
    for (uint32_t k = 0; k < n_seg; ++k) arr.seg_ready.push_back(ctx->copy_events[2 + k]);
    if (ctx->profiling) {
        const auto& sev = ctx->host_seg_events.back();
        arr.t_landed.assign(sev.begin(), sev.begin() + n_seg);
        arr.t_done.assign(sev.begin() + n_seg, sev.end());
    }
    if (gemm) {
        for (uint32_t k = 0; k < n_slots; ++k)
            arr.slot_mat.push_back(reinterpret_cast<const float*>(base + mat_off + (size_t)k * slot_bytes));
        for (uint32_t k = 0; k < n_seg; ++k) arr.prep_done.push_back(ctx->copy_events[2 + kHostSegments + k]);
        // segment k's copies, queued as its kernels are (after the preparation that
        // last read its slot)
        arr.issue_copy = [&, n_seg, n_slots](size_t k) -> cudaError_t {
            cudaError_t e = cudaSuccess;
            if (k >= n_slots) e = cudaStreamWaitEvent(cs, arr.prep_done[k - n_slots], 0);
            float* slot = dmat + (k % n_slots) * (slot_bytes / sizeof(float));
            const uint64_t o0 = band_flat_offset(seg_band[k], ld, n);
            for (uint32_t I = seg_band[k]; I < seg_band[k + 1] && e == cudaSuccess; ++I) {
                const uint64_t r0 = 128ull * I;
                const uint64_t rows = std::min<uint64_t>(128, n - r0), width = n - r0;
                float* dst = slot + (band_flat_offset(I, ld, n) - o0);
                size_t bytes;
                if (host_band_2d(n, I)) {
                    bytes = rows * width * sizeof(float);
                    e = cudaMemcpy2DAsync(dst, ld * sizeof(float), mat + r0 * ld + r0, ld * sizeof(float),
                                          width * sizeof(float), rows, cudaMemcpyHostToDevice, cs);
                } else {
                    bytes = band_flat_floats(I, ld, n) * sizeof(float);
                    e = cudaMemcpyAsync(dst, mat + r0 * ld + r0, bytes, cudaMemcpyHostToDevice, cs);
                }
                if (ctx->profiling) ctx->host_h2d_bytes += bytes;
            }
            if (e == cudaSuccess) e = cudaEventRecord(arr.seg_ready[k], cs);
            if (e == cudaSuccess && !arr.t_landed.empty()) e = cudaEventRecord(arr.t_landed[k], cs);
            if (e == cudaSuccess && ctx->profiling && k == 0) e = cudaEventRecord(tev[1], cs);
            if (e == cudaSuccess && ctx->profiling && k + 1 == n_seg) e = cudaEventRecord(tev[2], cs);
            return e;
        };
    } else {
        const size_t bytes = ((uint64_t)(n - 1) * ld + n) * sizeof(float);
        CK(cudaMemcpyAsync(dmat, mat, bytes, cudaMemcpyHostToDevice, cs), "copy matrix");
        if (ctx->profiling) ctx->host_h2d_bytes += bytes;
        CK(cudaEventRecord(arr.seg_ready[0], cs), "record matrix");
        if (ctx->profiling) {
            CK(cudaEventRecord(arr.t_landed[0], cs), "record segment landed");
            CK(cudaEventRecord(tev[1], cs), "record first segment");
            CK(cudaEventRecord(tev[2], cs), "record last segment");
        }
    }
    // the staged label buffer is 256-byte aligned: re-plan so the direct path can be taken
    rc = layout_for(ctx, L.plan, n, ld, base + lab_off, label_type, K, P, &L);
    if (rc) return rc;
    SWProblem pr{reinterpret_cast<const float*>(dmat), n, ld, base + lab_off, label_type, K,
                 P, nullptr, reinterpret_cast<double*>(base + out_off)};
    rc = run_sW(ctx, L, pr, reinterpret_cast<const float*>(base + w_off), s, &arr);
    if (rc) return rc;
    CK(cudaMemcpyAsync(out, base + out_off, (size_t)P * sizeof(double), cudaMemcpyDeviceToHost, s),
       "copy results");
    if (ctx->profiling) CK(cudaEventRecord(tev[3], s), "record end");
    return read_status(ctx, s);
}

int permanova_permutations(permanova_ctx* ctx, const int32_t* grouping, uint32_t n, uint32_t K,
                           uint64_t n_perms, uint64_t seed, void* out, int label_type, void* stream) {
    if (!ctx) return fail(PERMANOVA_EINVAL, "ctx is NULL");
    if (!grouping || !out) return fail(PERMANOVA_EINVAL, "NULL pointer argument");
    if (n < 2) return fail(PERMANOVA_EINVAL, "n_dims must be >= 2");
    if (n_perms == 0 || n_perms >= 0xFFFFFFFFull) return fail(PERMANOVA_EINVAL, "n_perms out of range");
    if (label_type != LABEL_I32 && label_type != LABEL_U16 && label_type != LABEL_U8)
        return fail(PERMANOVA_EINVAL, "unknown label type %d", label_type);
    if ((label_type == LABEL_U8 && K > 256) || (label_type == LABEL_U16 && K > 65536))
        return fail(PERMANOVA_EINVAL, "label type too narrow for %u groups", K);
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    CK(launch_permutations(grouping, n, n_perms, seed, out, label_type, static_cast<cudaStream_t>(stream)),
       "permutation kernels");
    return PERMANOVA_OK;
}

int permanova_test(permanova_ctx* ctx, const float* mat, uint32_t n, uint64_t ld,
                   const int32_t* grouping, uint32_t K, uint64_t P, uint64_t seed,
                   permanova_result* out_host, double* out_sW, void* stream) {
    return permanova_test_mixed(ctx, mat, n, ld, grouping, 1, &K, &P, &seed, out_host, out_sW, stream);
}

int permanova_test_batch(permanova_ctx* ctx, const float* mat, uint32_t n, uint64_t ld,
                         const int32_t* groupings, uint32_t T, uint32_t K, uint64_t P,
                         const uint64_t* seeds, permanova_result* out_host, double* out_sW,
                         void* stream) {
    if (T == 0) return fail(PERMANOVA_EINVAL, "n_tests must be >= 1");
    std::vector<uint32_t> Ks(T, K);
    std::vector<uint64_t> Ps(T, P);
    return permanova_test_mixed(ctx, mat, n, ld, groupings, T, Ks.data(), Ps.data(), seeds, out_host,
                                out_sW, stream);
}

}  // extern "C"

namespace {
// permanova_test_mixed, with the tensor-core operands optionally prepared
int test_mixed_impl(permanova_ctx* ctx, const float* mat, uint32_t n, uint64_t ld, const void* prepared_ops,
                    const int32_t* groupings, uint32_t T, const uint32_t* Ks, const uint64_t* Ps,
                    const uint64_t* seeds, permanova_result* out_host, double* out_sW, void* stream) {
    if (!ctx) return fail(PERMANOVA_EINVAL, "ctx is NULL");
    if (!mat || !groupings || !out_host || !seeds || !Ks || !Ps)
        return fail(PERMANOVA_EINVAL, "NULL pointer argument");
    if (T == 0) return fail(PERMANOVA_EINVAL, "n_tests must be >= 1");
    if (ld < n) return fail(PERMANOVA_EINVAL, "ld < n_dims");
    uint32_t Kmax = 0;
    for (uint32_t t = 0; t < T; ++t) {
        if (Ks[t] < 2) return fail(PERMANOVA_EINVAL, "test %u: the test needs n_groups >= 2 (got %u)", t, Ks[t]);
        if (n <= Ks[t])
            return fail(PERMANOVA_EINVAL, "test %u: the test needs n_dims > n_groups (pseudo-F undefined)", t);
        if (Ps[t] == 0 || Ps[t] >= 0xFFFFFFFFull) return fail(PERMANOVA_EINVAL, "test %u: n_perms out of range", t);
        Kmax = std::max(Kmax, Ks[t]);
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // group sizes -> inv_group_sizes 1/n_g in FP64 (host), observed labels checked here
    std::vector<int32_t> hg((size_t)n * T);
    CK(cudaMemcpyAsync(hg.data(), groupings, hg.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, s),
       "copy groupings");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    std::vector<double> hw((size_t)Kmax * T, 0.0);   // test t's weights, groups >= K_t stay 0
    std::vector<uint64_t> sizes(Kmax);
    for (uint32_t t = 0; t < T; ++t) {
        std::fill(sizes.begin(), sizes.end(), 0);
        for (uint32_t i = 0; i < n; ++i) {
            const int32_t lab = hg[(size_t)t * n + i];
            if (lab < 0 || (uint32_t)lab >= Ks[t])
                return fail(PERMANOVA_EINVAL, "test %u: grouping[%u] = %d outside [0, %u)", t, i, lab, Ks[t]);
            sizes[lab] += 1;
        }
        for (uint32_t k = 0; k < Ks[t]; ++k) {
            if (sizes[k] == 0) return fail(PERMANOVA_EINVAL, "test %u: group %u is empty", t, k);
            hw[(size_t)t * Kmax + k] = 1.0 / (double)sizes[k];
        }
    }

    // Each test runs in the kernel form a lone test of its sizes gets; tests of
    // one form share one s_W pass (label rows of every such test, n_groups =
    // the largest of them, per-test weights, unused groups weighted 0), so the
    // batch is processed in form order.  Every per-row result is independent
    // of the other rows in its launch and of the padded group count, so each
    // test's s_W, F and p equal those of the same test run alone.
    // tests are grouped by their whole plan (form and knobs: every knob that
    // changes the arithmetic is the same for the tests of one launch)
    std::vector<Plan> plans;
    std::vector<uint32_t> pid(T);
    for (uint32_t t = 0; t < T; ++t) {
        const Plan pl = plan_for(ctx, n, Ks[t], Ps[t] + 1);
        uint32_t k = 0;
        while (k < plans.size() && !(plans[k] == pl)) ++k;
        if (k == plans.size()) plans.push_back(pl);
        pid[t] = k;
    }
    std::vector<uint32_t> order(T);
    for (uint32_t t = 0; t < T; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return pid[x] < pid[y]; });
    std::vector<uint64_t> rs(T + 1, 0);      // row starts in form order
    std::vector<uint32_t> ks(T);
    std::vector<uint64_t> sd(T);
    for (uint32_t k = 0; k < T; ++k) {
        rs[k + 1] = rs[k] + Ps[order[k]] + 1;
        ks[k] = Ks[order[k]];
        sd[k] = seeds[order[k]];
    }
    const uint64_t rows = rs[T];
    const int lt = Kmax <= 256 ? LABEL_U8 : Kmax <= 65536 ? LABEL_U16 : LABEL_I32;
    // form groups [gb[q], gb[q+1]) of the ordered tests, each with its own
    // weight table (stride = the group's n_groups) and row starts
    struct FormGroup { uint32_t t0, t1, K; Plan plan; size_t w_off, rs_off; };
    std::vector<FormGroup> groups;
    std::vector<double> gw;
    std::vector<uint64_t> grs;
    for (uint32_t k = 0; k < T;) {
        uint32_t e = k;
        uint32_t Kg = 0;
        while (e < T && pid[order[e]] == pid[order[k]]) Kg = std::max(Kg, ks[e++]);
        FormGroup fg{k, e, Kg, plans[pid[order[k]]], gw.size(), grs.size()};
        if (prepared_ops && fg.plan.form == PERMANOVA_FORM_GEMM) fg.plan.prepared = true;
        for (uint32_t q = k; q < e; ++q)
            for (uint32_t c = 0; c < Kg; ++c) gw.push_back(hw[(size_t)order[q] * Kmax + c]);
        for (uint32_t q = k; q <= e; ++q) grs.push_back(rs[q] - rs[k]);
        groups.push_back(fg);
        k = e;
    }
    size_t sw_scratch = 0;
    for (const FormGroup& fg : groups) {
        SWLayout L;
        int rc = layout_for(ctx, fg.plan, n, ld, nullptr, lt, fg.K, rs[fg.t1] - rs[fg.t0], &L);
        if (rc) return rc;
        sw_scratch = std::max(sw_scratch, L.total);
    }
    size_t off = align_up(sw_scratch);
    const size_t lab_off = off;
    off = align_up(off + (size_t)n * rows * label_bytes(lt));
    const size_t sw_off = off;
    off = align_up(off + (size_t)rows * sizeof(double));
    const uint32_t chunks = brute_chunks(n, ctx->sm_count, 1);
    const size_t st_off = off;
    off = align_up(off + (size_t)(chunks + 1) * sizeof(double));
    const size_t w_off = off;
    off = align_up(off + gw.size() * sizeof(double));
    const size_t grs_off = off;
    off = align_up(off + grs.size() * sizeof(uint64_t));
    const size_t rs_off = off;
    off = align_up(off + (size_t)(T + 1) * sizeof(uint64_t));
    const size_t seed_off = off;
    off = align_up(off + (size_t)T * sizeof(uint64_t));
    const size_t ks_off = off;
    off = align_up(off + (size_t)T * sizeof(uint32_t));
    const size_t src_off = off;
    off = align_up(off + (size_t)T * sizeof(uint32_t));
    const size_t res_off = off;
    off = align_up(off + (size_t)T * sizeof(TestScalars));
    int rc = ensure_arena(ctx, off);
    if (rc) return rc;
    char* base = static_cast<char*>(ctx->arena);
    void* labels = base + lab_off;
    double* sW = reinterpret_cast<double*>(base + sw_off);
    double* st_part = reinterpret_cast<double*>(base + st_off);
    double* dw = reinterpret_cast<double*>(base + w_off);
    uint64_t* dgrs = reinterpret_cast<uint64_t*>(base + grs_off);
    uint64_t* drs = reinterpret_cast<uint64_t*>(base + rs_off);
    uint64_t* dseeds = reinterpret_cast<uint64_t*>(base + seed_off);
    uint32_t* dks = reinterpret_cast<uint32_t*>(base + ks_off);
    uint32_t* dsrc = reinterpret_cast<uint32_t*>(base + src_off);
    TestScalars* dres = reinterpret_cast<TestScalars*>(base + res_off);

    CK(cudaMemcpyAsync(dw, gw.data(), gw.size() * sizeof(double), cudaMemcpyHostToDevice, s), "copy weights");
    CK(cudaMemcpyAsync(dgrs, grs.data(), grs.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s),
       "copy row starts");
    CK(cudaMemcpyAsync(drs, rs.data(), rs.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s),
       "copy row starts");
    CK(cudaMemcpyAsync(dseeds, sd.data(), sd.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s), "copy seeds");
    CK(cudaMemcpyAsync(dks, ks.data(), ks.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s),
       "copy group counts");
    CK(cudaMemcpyAsync(dsrc, order.data(), order.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s),
       "copy test order");
    CK(launch_permutations_batch(groupings, dsrc, n, T, drs, rows - T, dseeds, labels, lt, s),
       "permutation kernels");
    for (const FormGroup& fg : groups) {
        const uint64_t r0 = rs[fg.t0], nr = rs[fg.t1] - r0;
        void* glab = static_cast<char*>(labels) + (size_t)n * r0 * label_bytes(lt);
        SWLayout L;
        rc = layout_for(ctx, fg.plan, n, ld, glab, lt, fg.K, nr, &L);
        if (rc) return rc;
        SWProblem pr{mat, n, ld, glab, lt, fg.K, nr, dw + fg.w_off, sW + r0};
        pr.w_row_start = dgrs + fg.rs_off;
        pr.w_sets = fg.t1 - fg.t0;
        rc = run_sW(ctx, L, pr, nullptr, s, nullptr, fg.plan.prepared ? prepared_ops : nullptr);
        if (rc) return rc;
    }
    CK(launch_sumsq_triangle(mat, n, ld, chunks, st_part, s), "sum of squares kernel");
    CK(launch_reduce_rows(st_part, chunks, 1, st_part + chunks, s), "reduce s_T");
    CK(launch_finalize_batch(sW, T, drs, dks, st_part + chunks, n, dres, s), "finalize kernel");
    if (out_sW) {
        // caller order: test t's rows after those of tests 0 .. t-1
        std::vector<uint64_t> dst(T + 1, 0);
        for (uint32_t t = 0; t < T; ++t) dst[t + 1] = dst[t] + Ps[t] + 1;
        for (uint32_t k = 0; k < T; ++k) {
            const uint32_t t = order[k];
            CK(cudaMemcpyAsync(out_sW + dst[t], sW + rs[k], (size_t)(Ps[t] + 1) * sizeof(double),
                               cudaMemcpyDeviceToDevice, s),
               "copy s_W");
        }
    }
    std::vector<TestScalars> hres(T);
    CK(cudaMemcpyAsync(hres.data(), dres, (size_t)T * sizeof(TestScalars), cudaMemcpyDeviceToHost, s),
       "copy results");
    rc = read_status(ctx, s);
    if (rc) return rc;
    for (uint32_t k = 0; k < T; ++k) {
        const uint32_t t = order[k];
        out_host[t].s_T = hres[k].s_T;
        out_host[t].s_W_obs = hres[k].s_W_obs;
        out_host[t].F_obs = hres[k].F_obs;
        out_host[t].p_value = hres[k].p_value;
        out_host[t].n_ge = hres[k].n_ge;
        out_host[t].n_perms = hres[k].n_perms;
    }
    return PERMANOVA_OK;
}
}  // namespace

extern "C" {

int permanova_test_mixed(permanova_ctx* ctx, const float* mat, uint32_t n, uint64_t ld,
                         const int32_t* groupings, uint32_t T, const uint32_t* Ks, const uint64_t* Ps,
                         const uint64_t* seeds, permanova_result* out_host, double* out_sW,
                         void* stream) {
    return test_mixed_impl(ctx, mat, n, ld, nullptr, groupings, T, Ks, Ps, seeds, out_host, out_sW, stream);
}

int permanova_prepare(permanova_ctx* ctx, const float* mat, uint32_t n, uint64_t ld, permanova_prepared** out,
                      void* stream) {
    if (!ctx || !out) return fail(PERMANOVA_EINVAL, "NULL argument");
    *out = nullptr;
    if (!mat) return fail(PERMANOVA_EINVAL, "mat is NULL");
    if (n < 2) return fail(PERMANOVA_EINVAL, "n_dims must be >= 2 (got %u)", n);
    if (ld < n) return fail(PERMANOVA_EINVAL, "ld (%llu) < n_dims (%u)", (unsigned long long)ld, n);
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const GemmPlan gp = gemm_plan(n, 1, 1);   // the operands depend on n alone
    auto* p = new permanova_prepared();
    p->device = ctx->device;
    p->mat = mat;
    p->n = n;
    p->ld = ld;
    p->bytes = gemm_scratch_bytes(gp, 0);
    cudaError_t e = cudaMalloc(&p->ops, p->bytes);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaMalloc(prepared operands)");
    }
    SWProblem pr{mat, n, ld, nullptr, LABEL_U8, 1, 1, nullptr, nullptr};
    e = launch_gemm_prep(pr, gp, p->ops, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(p->ops);
        delete p;
        return cuda_fail(e, "operand preparation");
    }
    *out = p;
    return PERMANOVA_OK;
}

void permanova_prepared_destroy(permanova_prepared* p) {
    if (!p) return;
    {
        DeviceGuard g(p->device);
        cudaDeviceSynchronize();
        if (p->ops) cudaFree(p->ops);
    }
    delete p;
}

int permanova_sW_prepared(permanova_ctx* ctx, const permanova_prepared* prep, const void* groupings,
                          int label_type, uint32_t K, uint64_t P, const float* w, double* out, void* stream) {
    if (!ctx || !prep) return fail(PERMANOVA_EINVAL, "NULL argument");
    if (prep->device != ctx->device) return fail(PERMANOVA_EINVAL, "prepared on another device");
    int rc = check_sW_args(prep->mat, prep->n, prep->ld, groupings, label_type, K, P, w, out);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Plan pl = plan_for(ctx, prep->n, K, P);
    if (pl.form == PERMANOVA_FORM_GEMM) pl.prepared = true;
    SWLayout L;
    rc = layout_for(ctx, pl, prep->n, prep->ld, groupings, label_type, K, P, &L);
    if (rc) return rc;
    rc = ensure_arena(ctx, L.total);
    if (rc) return rc;
    SWProblem pr{prep->mat, prep->n, prep->ld, groupings, label_type, K, P, nullptr, out};
    return run_sW(ctx, L, pr, w, s, nullptr, pl.prepared ? prep->ops : nullptr);
}

int permanova_test_mixed_prepared(permanova_ctx* ctx, const permanova_prepared* prep, const int32_t* groupings,
                                  uint32_t T, const uint32_t* Ks, const uint64_t* Ps, const uint64_t* seeds,
                                  permanova_result* out_host, double* out_sW, void* stream) {
    if (!ctx || !prep) return fail(PERMANOVA_EINVAL, "NULL argument");
    if (prep->device != ctx->device) return fail(PERMANOVA_EINVAL, "prepared on another device");
    return test_mixed_impl(ctx, prep->mat, prep->n, prep->ld, prep->ops, groupings, T, Ks, Ps, seeds, out_host,
                           out_sW, stream);
}

}  // extern "C"
