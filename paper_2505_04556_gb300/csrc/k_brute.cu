// Brute-force s_W (the semantics of the paper's GPU listing, Algorithm 3):
// every label row streams the strict upper triangle of D from HBM once.
//
// Work split: one CTA = (label row p, chunk c of the triangle).  Chunks hold
// equal numbers of pairs (rows are found by binary search on the pair prefix
// count), so the CTAs that run together are the chunks of one or two label
// rows and D is re-read from HBM for every row, as in Algorithm 3.  Loads are
// 128-bit and coalesced along the row; the row's weight is applied once per
// row segment (the reuse Algorithm 2 introduces); per-thread FP32 row
// segments are added in FP64 and the CTA writes one FP64 partial per
// (chunk, p), summed later in fixed order.
#include "common.cuh"

namespace pmn {

constexpr int BR_THREADS = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    return s;
}

template <typename L, bool VEC>
__global__ void __launch_bounds__(BR_THREADS)
k_sw_brute(const float* __restrict__ mat, uint32_t n, uint64_t ld, const L* __restrict__ labels,
           uint64_t P, const WeightMap wm, uint32_t K, uint32_t n_chunks,
           double* __restrict__ partials, const DevStatus* __restrict__ st) {
    __shared__ double red[BR_THREADS / 32];
    const uint64_t unit = blockIdx.x;
    const uint64_t p = unit / n_chunks;
    const uint32_t c = (uint32_t)(unit % n_chunks);
    if (p >= P) return;
    // labels failed validation: skip the work (a block-uniform vote, so the
    // barrier in the block sum is never left by only some threads)
    if (__syncthreads_or(st->code != DEV_OK)) {
        if (threadIdx.x == 0) partials[(uint64_t)c * P + p] = 0.0;
        return;
    }
    const uint64_t total = pairs_before_row(n, n);
    const uint32_t r0 = row_for_pair(total * c / n_chunks, n);
    const uint32_t r1 = row_for_pair(total * (c + 1) / n_chunks, n);
    const L* g = labels + p * n;
    const double* wrow = wm.row(p);
    double acc = 0.0;
    for (uint32_t i = r0; i < r1 && i + 1 < n; ++i) {
        const uint32_t gi = min(label_at(g, i), K - 1);
        const double wi = __ldg(wrow + gi);
        const float* row = mat + (uint64_t)i * ld;
        float s = 0.f;
        uint32_t j = i + 1;
        if (VEC) {
            // scalar head up to a multiple of 4, then float4 body
            const uint32_t jv = min((j + 3u) & ~3u, n);
            if (j + threadIdx.x < jv) {
                const uint32_t jj = j + threadIdx.x;
                const float v = __ldg(row + jj);
                s += (label_at(g, jj) == gi) ? v * v : 0.f;
            }
            const uint32_t nv = (n - jv) / 4;  // full float4 groups
            const float4* row4 = reinterpret_cast<const float4*>(row + jv);
            uint32_t k = threadIdx.x;
#pragma unroll 4
            for (; k < nv; k += BR_THREADS) {
                const float4 v = __ldg(row4 + k);
                const uint32_t jj = jv + 4 * k;
                const uint32_t g0 = label_at(g, jj), g1 = label_at(g, jj + 1);
                const uint32_t g2 = label_at(g, jj + 2), g3 = label_at(g, jj + 3);
                s += (g0 == gi) ? v.x * v.x : 0.f;
                s += (g1 == gi) ? v.y * v.y : 0.f;
                s += (g2 == gi) ? v.z * v.z : 0.f;
                s += (g3 == gi) ? v.w * v.w : 0.f;
            }
            const uint32_t jt = jv + 4 * nv;
            if (jt + threadIdx.x < n) {
                const uint32_t jj = jt + threadIdx.x;
                const float v = __ldg(row + jj);
                s += (label_at(g, jj) == gi) ? v * v : 0.f;
            }
        } else {
            for (uint32_t jj = j + threadIdx.x; jj < n; jj += BR_THREADS) {
                const float v = __ldg(row + jj);
                s += (label_at(g, jj) == gi) ? v * v : 0.f;
            }
        }
        acc += (double)s * wi;
    }
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) partials[(uint64_t)c * P + p] = tot;
}

uint32_t brute_chunks(uint32_t n, int sm_count, uint32_t mult) {
    // about 32K pairs per CTA at least, at most 4 CTAs per SM per label row
    // (times mult)
    if (mult < 1) mult = 1;
    const uint64_t pairs = pairs_before_row(n, n);
    uint64_t c = pairs * mult / 32768;
    const uint64_t cap = (uint64_t)(sm_count > 0 ? sm_count : 152) * 4 * mult;
    if (c > cap) c = cap;
    if (c > n - 1) c = n - 1;
    return c < 1 ? 1u : (uint32_t)c;
}

template <typename L>
static cudaError_t launch_brute_t(const SWProblem& pr, uint32_t n_chunks, double* partials,
                                  const DevStatus* st, cudaStream_t s) {
    const bool vec = (pr.ld % 4 == 0) && ((uintptr_t)pr.mat % 16 == 0);
    const uint64_t blocks = pr.P * n_chunks;
    if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    if (vec)
        k_sw_brute<L, true><<<(unsigned)blocks, BR_THREADS, 0, s>>>(
            pr.mat, pr.n, pr.ld, (const L*)pr.labels, pr.P, pr.weights(), pr.K, n_chunks,
            partials, st);
    else
        k_sw_brute<L, false><<<(unsigned)blocks, BR_THREADS, 0, s>>>(
            pr.mat, pr.n, pr.ld, (const L*)pr.labels, pr.P, pr.weights(), pr.K, n_chunks,
            partials, st);
    return launched(1);
}

cudaError_t launch_brute(const SWProblem& pr, uint32_t n_chunks, double* partials,
                         const DevStatus* st, cudaStream_t s) {
    if (pr.label_type == LABEL_U8) return launch_brute_t<uint8_t>(pr, n_chunks, partials, st, s);
    if (pr.label_type == LABEL_U16) return launch_brute_t<uint16_t>(pr, n_chunks, partials, st, s);
    return launch_brute_t<int32_t>(pr, n_chunks, partials, st, s);
}

// ---------------------------------------------------------------------------
// sum_{i<j} d_ij^2 (numerator of s_T), same chunking, no labels.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BR_THREADS)
k_sumsq_triangle(const float* __restrict__ mat, uint32_t n, uint64_t ld, uint32_t n_chunks,
                 double* __restrict__ partials) {
    __shared__ double red[BR_THREADS / 32];
    const uint32_t c = blockIdx.x;
    const uint64_t total = pairs_before_row(n, n);
    const uint32_t r0 = row_for_pair(total * c / n_chunks, n);
    const uint32_t r1 = row_for_pair(total * (c + 1) / n_chunks, n);
    double acc = 0.0;
    for (uint32_t i = r0; i < r1 && i + 1 < n; ++i) {
        const float* row = mat + (uint64_t)i * ld;
        float s = 0.f;
        for (uint32_t j = i + 1 + threadIdx.x; j < n; j += BR_THREADS) {
            const float v = __ldg(row + j);
            s += v * v;
        }
        acc += (double)s;
    }
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) partials[c] = tot;
}

cudaError_t launch_sumsq_triangle(const float* mat, uint32_t n, uint64_t ld, uint32_t n_chunks,
                                  double* partials, cudaStream_t s) {
    k_sumsq_triangle<<<n_chunks, BR_THREADS, 0, s>>>(mat, n, ld, n_chunks, partials);
    return launched(1);
}

}  // namespace pmn
