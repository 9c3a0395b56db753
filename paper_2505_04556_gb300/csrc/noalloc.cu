// s_W without any device allocation.
//
// Some callers cannot call cudaMalloc: plugins of host frameworks that own
// every device allocation themselves (and forbid others), and processes that
// run inside a fixed device-memory pool with no headroom, where a fresh
// allocation would fail or evict the framework's own buffers.  For them,
// permanova_sW_noalloc runs an s_W kernel with its scratch (FP64 partial sums,
// FP64 weights, the device error word) in one fixed file-scope device array
// instead of context memory: the perm-block kernel (D tiles in shared memory
// shared by 256 label rows, about ten times the brute force's rate) when the
// labels are uint8 or uint16 codes whose rows start on 16-byte boundaries and
// its partials (one row per 64-row band) fit the array, else the brute-force
// kernel, whose partials shrink to fit.  It needs no context.
//
// The array is NOALLOC_BYTES (8 MiB) and stays resident on every GPU that
// loads this library until the process exits.  All calls on a device share
// it, so calls whose work overlaps on that GPU (different streams or host
// threads) race; callers must serialise them.  Each call clears the error
// word before use and overwrites the partials and weights it reads.
//
// Host code cannot use the array's name as an address (in host code it names
// a host-side stand-in), so the device address is looked up with
// cudaGetSymbolAddress at set-up: on the first call on a device, with that
// device current, and again whenever the device's context has been replaced
// (after a cudaDeviceReset, say), which the cache detects through the
// context's process-unique ID.
#include "../../include/permanova.h"
#include "common.cuh"

#include <cuda.h>

#include <cstdio>
#include <mutex>

namespace pmn {

constexpr size_t NOALLOC_BYTES = 8u << 20;
constexpr size_t NOALLOC_STATUS = 0;       // DevStatus
constexpr size_t NOALLOC_W = 256;          // K doubles
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

namespace {
std::mutex g_noalloc_mu;
struct NoallocSlot {
    unsigned long long ctx_id = 0;   // process-unique ID of the context the address belongs to
    void* ptr = nullptr;
};
NoallocSlot g_noalloc_slot[NOALLOC_MAX_DEVICES];
// driver entry points (signatures of cuCtxGetCurrent and cuCtxGetId), found
// through the runtime so the library needs no link against the driver
using CtxCurrentFn = CUresult (*)(CUcontext*);
using CtxIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxCurrentFn g_ctx_current = nullptr;
CtxIdFn g_ctx_id = nullptr;

// Process-unique ID of the calling thread's current context (0 if none).
cudaError_t current_context_id(unsigned long long* id) {
    *id = 0;
    if (!g_ctx_current || !g_ctx_id) {
        cudaDriverEntryPointQueryResult q1, q2;
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorSymbolNotFound;
        g_ctx_current = reinterpret_cast<CtxCurrentFn>(f1);
        g_ctx_id = reinterpret_cast<CtxIdFn>(f2);
    }
    CUcontext c = nullptr;
    if (g_ctx_current(&c) != CUDA_SUCCESS || c == nullptr) return cudaErrorDeviceUninitialized;
    if (g_ctx_id(c, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}
}  // namespace

// Device address of the scratch array on the current device.  Set-up runs on
// the first call on a device (and after the device's context was replaced):
// it makes sure the device's primary context exists, then looks the address
// up; that call must therefore come before any stream capture on the device.
static cudaError_t noalloc_base(int dev, void** out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    // selecting the (already current) device initialises its primary context
    // if that has not happened yet, so the context below exists
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) return e;
    unsigned long long id = 0;
    e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    NoallocSlot& slot = g_noalloc_slot[dev];
    if (slot.ptr == nullptr || slot.ctx_id != id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        slot.ptr = p;
        slot.ctx_id = id;
    }
    *out = slot.ptr;
    return cudaSuccess;
}

}  // namespace pmn

using namespace pmn;

extern "C" int permanova_sW_noalloc(const float* mat, uint32_t n, uint64_t ld, const void* groupings,
                                    int label_type, uint32_t K, uint64_t P,
                                    const float* inv_group_sizes, double* out_sW, void* stream) {
    char msg[256];
    auto err = [&](int code, const char* text) {
        set_last_error(text);   // readable through permanova_last_error(NULL)
        return code;
    };
    if (!mat || !groupings || !inv_group_sizes || !out_sW) return err(PERMANOVA_EINVAL, "NULL pointer argument");
    if (n < 2) return err(PERMANOVA_EINVAL, "n_dims must be >= 2");
    if (ld < n) return err(PERMANOVA_EINVAL, "ld < n_dims");
    if (K == 0 || P == 0) return err(PERMANOVA_EINVAL, "n_groups and n_perms must be >= 1");
    if (label_type != LABEL_I32 && label_type != LABEL_U16 && label_type != LABEL_U8)
        return err(PERMANOVA_EINVAL, "unknown label type");
    if ((label_type == LABEL_U8 && K > 256) || (label_type == LABEL_U16 && K > 65536))
        return err(PERMANOVA_EINVAL, "label type too narrow for n_groups");
    // capacity: K weights after the status word, then chunks x P partials
    const size_t part_off = (NOALLOC_W + (size_t)K * sizeof(double) + 255) / 256 * 256;
    if (part_off >= NOALLOC_BYTES) {
        snprintf(msg, sizeof msg, "n_groups = %u exceeds the no-allocation scratch (%zu bytes)", K,
                 NOALLOC_BYTES);
        return err(PERMANOVA_EINVAL, msg);
    }
    const uint64_t max_rows = (NOALLOC_BYTES - part_off) / ((uint64_t)P * sizeof(double));
    if (max_rows < 1) {
        snprintf(msg, sizeof msg,
                 "n_perms = %llu exceeds the no-allocation scratch (at most %zu label rows per call)",
                 (unsigned long long)P, (NOALLOC_BYTES - part_off) / sizeof(double));
        return err(PERMANOVA_EINVAL, msg);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return err(PERMANOVA_ECUDA, "no current CUDA device");
    void* base = nullptr;
    cudaError_t e = noalloc_base(dev, &base);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "no-allocation scratch set-up: %s", cudaGetErrorString(e));
        return err(PERMANOVA_ECUDA, msg);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* b = static_cast<unsigned char*>(base);
    DevStatus* st = reinterpret_cast<DevStatus*>(b + NOALLOC_STATUS);
    double* wd = reinterpret_cast<double*>(b + NOALLOC_W);
    double* partials = reinterpret_cast<double*>(b + part_off);
    // the perm-block kernel reads the caller's codes in place (16-byte rows)
    const uint64_t elem = label_type == LABEL_U8 ? 1 : label_type == LABEL_U16 ? 2 : 4;
    const bool rows16 = elem <= 2 && ((uint64_t)n * elem) % 16 == 0 &&
                        reinterpret_cast<uintptr_t>(groupings) % 16 == 0;
    const uint32_t pb_bands = permblock_bands(n);
    const bool permblock = rows16 && (uint64_t)pb_bands <= max_rows;
    uint32_t chunks = permblock ? pb_bands : brute_chunks(n, 0);
    if ((uint64_t)chunks > max_rows) chunks = (uint32_t)max_rows;

    SWProblem pr{mat, n, ld, groupings, label_type, K, P, wd, out_sW};
    if ((e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s)) == cudaSuccess &&
        (e = launch_widen(inv_group_sizes, K, wd, s)) == cudaSuccess &&
        (e = launch_validate_labels(groupings, label_type, (uint64_t)n * P, K, st, s)) == cudaSuccess &&
        (e = permblock ? launch_permblock_internal(pr, n, partials, st, s, 0)
                       : launch_brute(pr, chunks, partials, st, s)) == cudaSuccess &&
        (e = launch_reduce_rows(partials, chunks, P, out_sW, s)) == cudaSuccess) {
        DevStatus h{};
        e = cudaMemcpyAsync(&h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) {
            if (h.code == DEV_BAD_LABEL) {
                snprintf(msg, sizeof msg, "label >= n_groups at flat index %llu", h.info);
                return err(PERMANOVA_EINVAL, msg);
            }
            if (h.code != DEV_OK) return err(PERMANOVA_ECUDA, "device error");
            return PERMANOVA_OK;
        }
    }
    cudaGetLastError();
    snprintf(msg, sizeof msg, "CUDA error: %s", cudaGetErrorString(e));
    return err(PERMANOVA_ECUDA, msg);
}
