// Device-side helpers shared by the s_W kernels of libpermanova.
//
// Label element types (int32 / uint16 / uint8, perm-major rows as in the
// paper's Algorithm 1 driver: labels of row p at groupings + p*n), the
// device error word, and the launch prototypes the host runtime calls.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pmn {

// Device error word.  Kernels never trap: they record the first problem here
// and the host reports it at the next synchronising call.
struct DevStatus {
    unsigned int code;       // 0 = ok, see DEV_* below
    unsigned int where;      // kernel-specific detail (row, stage, ...)
    unsigned long long info; // e.g. flat index of a bad label
};
enum : unsigned int { DEV_OK = 0, DEV_BAD_LABEL = 1, DEV_TIMEOUT = 2 };

enum LabelType : int { LABEL_I32 = 0, LABEL_U16 = 1, LABEL_U8 = 2 };

template <typename L>
__device__ __forceinline__ uint32_t label_at(const L* __restrict__ p, uint64_t idx) {
    return (uint32_t)__ldg(p + idx);
}

__device__ __forceinline__ void raise_status(DevStatus* st, unsigned int code, unsigned int where,
                                             unsigned long long info) {
    if (atomicCAS(&st->code, 0u, code) == 0u) {
        st->where = where;
        st->info = info;
    }
}

// Number of strict-upper-triangle pairs in rows [0, r) of an n x n matrix.
__host__ __device__ __forceinline__ uint64_t pairs_before_row(uint64_t r, uint64_t n) {
    return r * n - r * (r + 1) / 2;
}

// First row r with pairs_before_row(r) >= target (0 <= target <= total).
__host__ __device__ __forceinline__ uint32_t row_for_pair(uint64_t target, uint32_t n) {
    uint32_t lo = 0, hi = n;  // answer in [lo, hi]
    while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (pairs_before_row(mid, n) >= target) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Weights of the label rows of one s_W launch: one set of K FP64 weights for
// every row, or one set per test when several tests share the launch (set t
// covers rows [row_start[t], row_start[t+1]), or rows [t*set_rows,
// (t+1)*set_rows) when row_start is NULL and set_rows > 0).
struct WeightMap {
    const double* w;
    uint64_t set_rows;          // equal-sized sets (0: see row_start / one set)
    const uint64_t* row_start;  // DEVICE, n_sets + 1 ascending row offsets, or NULL
    uint32_t n_sets;
    uint32_t K;                 // weights per set
    // Index of the weight set label row p uses.
    __device__ __forceinline__ uint64_t set_of(uint64_t p) const {
        if (row_start) {
            uint32_t lo = 0, hi = n_sets - 1;   // last set whose first row is <= p
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) / 2;
                if (__ldg(row_start + mid) <= p) lo = mid; else hi = mid - 1;
            }
            return lo;
        }
        return set_rows ? p / set_rows : 0;
    }
    // The K weights label row p uses.
    __device__ __forceinline__ const double* row(uint64_t p) const { return w + set_of(p) * K; }
};

struct SWProblem {
    const float* mat;
    uint32_t n;
    uint64_t ld;
    const void* labels;
    int label_type;
    uint32_t K;
    uint64_t P;
    const double* w;       // inv_group_sizes widened to FP64 (device)
    double* out;
    // Weight sets: 0 = one set of K weights for every label row; otherwise
    // label row p uses w[(p / w_set_rows) * K + g] (several tests in one pass).
    uint64_t w_set_rows;
    // Layout of mat: 0 = row-major with row stride ld; 1 = band-flat (see
    // band_flat_offset; tensor-core form only), holding bands [band0, ...).
    uint32_t banded;
    uint32_t band0;
    // Ragged weight sets (override w_set_rows): set t covers label rows
    // [w_row_start[t], w_row_start[t+1]) (DEVICE, w_sets + 1 entries).
    const uint64_t* w_row_start;
    uint32_t w_sets;
    WeightMap weights() const {
        return WeightMap{w, w_row_start ? 0ull : w_set_rows, w_row_start, w_sets, K};
    }
};

// Band-flat layout (the host entry point's staging of D for the tensor-core
// form): band I (rows [128 I, 128 I + 128)) is the contiguous range of the
// row-major n x ld matrix from element (128 I, 128 I) to the end of the band's
// last row, ((rows - 1) ld + n - 128 I) floats, which one flat copy moves;
// the bands of a staging slot are stored back to back.  Offset (in floats) of
// band I's first element from band 0's: sum_{I' < I} (127 ld + n - 128 I').
__host__ __device__ __forceinline__ uint64_t band_flat_offset(uint64_t I, uint64_t ld, uint64_t n) {
    return I * (127ull * ld + n) - (I ? 64ull * I * (I - 1) : 0ull);
}
// Floats of band I in that layout (the last band may have fewer rows).
__host__ __device__ __forceinline__ uint64_t band_flat_floats(uint64_t I, uint64_t ld, uint64_t n) {
    const uint64_t r0 = 128ull * I, rows = n - r0 < 128ull ? n - r0 : 128ull;
    return (rows - 1) * ld + (n - r0);
}
// Address of element (i, 0) of row i in either layout (in the band-flat one
// only elements j >= 128 * (i / 128) exist, and the address itself may lie
// before the row's first stored element).
__host__ __device__ __forceinline__ const float* d_row(const float* mat, uint64_t ld, uint32_t banded,
                                                       uint32_t n, uint32_t i, uint32_t band0 = 0) {
    if (!banded) return mat + (uint64_t)i * ld;
    const uint64_t I = i >> 7;
    return mat + (band_flat_offset(I, ld, n) - band_flat_offset(band0, ld, n)) + (uint64_t)(i - 128 * I) * ld -
           128 * I;
}

// inv_group_sizes (fp32, the paper's input) -> FP64 copy used by the kernels
cudaError_t launch_widen(const float* in, uint32_t K, double* out, cudaStream_t s);

// Sets the calling thread's error text (returned by permanova_last_error).
void set_last_error(const char* msg);

// Count of kernels the library has launched (all contexts); launchers return
// launched(k) after issuing k kernels.
void note_launches(unsigned k);
uint64_t kernel_launch_count();
inline cudaError_t launched(unsigned k) {
    note_launches(k);
    return cudaGetLastError();
}

// ---- launchers (defined in the .cu files) --------------------------------
cudaError_t launch_validate_labels(const void* labels, int type, uint64_t count, uint32_t K,
                                   DevStatus* st, cudaStream_t s);
cudaError_t launch_reduce_rows(const double* partials, uint32_t rows, uint64_t P, double* out,
                               cudaStream_t s);

// brute force (Algorithm 3 semantics): partials is n_chunks x P
// mult > 1 splits each label row's triangle into that many times more chunks
uint32_t brute_chunks(uint32_t n, int sm_count, uint32_t mult = 1);
cudaError_t launch_brute(const SWProblem& pr, uint32_t n_chunks, double* partials,
                         const DevStatus* st, cudaStream_t s);
// sum of squares of the strict upper triangle: partials is n_chunks x 1
cudaError_t launch_sumsq_triangle(const float* mat, uint32_t n, uint64_t ld, uint32_t n_chunks,
                                  double* partials, cudaStream_t s);

// perm-block CUDA-core form: partials is permblock_bands(n) x P; labels are
// uint8/uint16 codes with a 16-byte-multiple row stride of lstride elements
uint32_t permblock_bands(uint32_t n);
// variant 0: the paired FP16-compare kernel for uint8 and uint16 codes (default);
// variant 2: the same sized for 4 CTAs per SM; variant 1: the FP32
// compare-and-set kernel
cudaError_t launch_permblock_internal(const SWProblem& pr, uint64_t lstride, double* partials,
                                      const DevStatus* st, cudaStream_t s, int variant = 0);

// labels -> uint8/uint16 codes with row stride lstride (padding = 0); labels
// >= K raise DEV_BAD_LABEL and are clamped to K-1
cudaError_t launch_repack_labels(const void* in, int in_type, uint32_t n, uint64_t P, uint32_t K,
                                 void* out, int out_type, uint64_t lstride, DevStatus* st,
                                 cudaStream_t s);

// tcgen05 GEMM form
struct GemmPlan {
    uint32_t n_pad;        // n rounded up to 128
    uint32_t n_bands;      // n_pad / 128
    uint32_t perms_per_tile;
    uint64_t n_ptiles;
    uint64_t plane_elems;  // bf16 elements per plane (hi or lo) of the banded upper triangle
};
bool gemm_available();
// work counters of one call's GEMM launches (one per launch, at most this many)
constexpr uint32_t kGemmWorkCounters = 32;
// ppt_div > 1 divides the label rows per tile (narrower MMA tiles, more work
// units per band)
GemmPlan gemm_plan(uint32_t n, uint32_t K, uint64_t P, uint32_t ppt_div = 1);
size_t gemm_scratch_bytes(const GemmPlan& gp, uint64_t P);
// label rows -> (tile, k-block) blocks of uint8 codes read by the GEMM kernel
size_t gemm_label_bytes(const GemmPlan& gp);
cudaError_t launch_repack_gemm(const void* in, int in_type, uint32_t n, uint64_t P, uint32_t K,
                               const GemmPlan& gp, void* out, DevStatus* st, cudaStream_t s);
// D^2 -> per-band scale, then BF16 hi / FP16 (or BF16) lo operand tiles in the
// scratch, for the 128-row bands [I0, I1) (a band's tiles and scale are made from
// the band's rows of D only)
cudaError_t launch_gemm_prep(const SWProblem& pr, const GemmPlan& gp, void* scratch, cudaStream_t s,
                             uint32_t I0 = 0, uint32_t I1 = 0xFFFFFFFFu);
// the tensor-core kernel over bands [I0, I1): partials is gp.n_bands x P, this
// launch writes the rows of its bands
// drain_kb: k-blocks accumulated in tensor memory between FP64 drains (0 =
// default); work: the launch's work counter (DEVICE, zeroed by the caller on
// the launch's stream before it runs), from which the kernel takes its units
cudaError_t launch_gemm_main(const SWProblem& pr, const GemmPlan& gp, const void* scratch,
                             double* partials, DevStatus* st, int sm_count, cudaStream_t s,
                             uint32_t I0, uint32_t I1, uint32_t drain_kb, unsigned long long* work);

// a bounded wait on an mbarrier that never completes (failure-detection self-test)
cudaError_t launch_wait_selftest(DevStatus* st, long long limit_cycles, cudaStream_t s);

// permutation test helpers
cudaError_t launch_permutations(const int32_t* grouping, uint32_t n, uint64_t n_perms,
                                uint64_t seed, void* out, int label_type, cudaStream_t s);
struct TestScalars {
    double s_T;
    double s_W_obs;
    double F_obs;
    double p_value;
    unsigned long long n_ge;
    unsigned long long n_perms;
};
// n_tests tests in one pass: test t owns label rows [rs[t], rs[t+1]) (DEVICE
// offsets), its observed grouping is row src[t] of `groupings`, its seed
// seeds[t] and its group count Ks[t]; results go to out[t]
cudaError_t launch_finalize_batch(const double* sW, uint32_t n_tests, const uint64_t* rs,
                                  const uint32_t* Ks, const double* sT_sum, uint32_t n,
                                  TestScalars* out, cudaStream_t s);
cudaError_t launch_permutations_batch(const int32_t* groupings, const uint32_t* src, uint32_t n,
                                      uint32_t n_tests, const uint64_t* rs, uint64_t total_perms,
                                      const uint64_t* seeds, void* out, int label_type, cudaStream_t s);

}  // namespace pmn
