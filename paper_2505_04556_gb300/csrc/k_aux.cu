// Auxiliary kernels of the s_W path: label validation, the fixed-order
// cross-tile reduction, device permutation generation for the permutation
// test (Sec. 1) and the test's final statistics.
#include "common.cuh"

#include <atomic>

namespace pmn {

// ---------------------------------------------------------------------------
// Label validation: every label must index inv_group_sizes (0 <= g < K).
// ---------------------------------------------------------------------------
template <typename L>
__global__ void k_validate(const L* __restrict__ lab, uint64_t count, uint32_t K, DevStatus* st) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        uint32_t g = (uint32_t)lab[i];
        if (g >= K) {
            raise_status(st, DEV_BAD_LABEL, 0u, (unsigned long long)i);
            return;
        }
    }
}

// uint8 labels, 16 at a time when the buffer allows it.
__global__ void k_validate_u8x16(const uint4* __restrict__ lab, uint64_t count16, uint32_t K,
                                 DevStatus* st) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count16; i += stride) {
        uint4 v = __ldg(lab + i);
        uint32_t w[4] = {v.x, v.y, v.z, v.w};
        uint32_t bad = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int b = 0; b < 4; ++b) bad |= (((w[k] >> (8 * b)) & 0xFFu) >= K);
        if (bad) {
            raise_status(st, DEV_BAD_LABEL, 0u, (unsigned long long)(i * 16));
            return;
        }
    }
}

cudaError_t launch_validate_labels(const void* labels, int type, uint64_t count, uint32_t K,
                                   DevStatus* st, cudaStream_t s) {
    const int threads = 256;
    const int blocks = 152 * 8;
    if (type == LABEL_U8) {
        if (K >= 256) return cudaSuccess;  // every byte is a valid label
        uint64_t c16 = ((uintptr_t)labels % 16 == 0) ? count / 16 : 0;
        unsigned k = 0;
        if (c16) {
            k_validate_u8x16<<<blocks, threads, 0, s>>>((const uint4*)labels, c16, K, st);
            ++k;
        }
        uint64_t done = c16 * 16;
        if (done < count) {
            k_validate<uint8_t><<<blocks, threads, 0, s>>>((const uint8_t*)labels + done,
                                                           count - done, K, st);
            ++k;
        }
        return launched(k);
    }
    if (type == LABEL_U16) {
        if (K >= 65536) return cudaSuccess;
        k_validate<uint16_t><<<blocks, threads, 0, s>>>((const uint16_t*)labels, count, K, st);
    } else {
        k_validate<int32_t><<<blocks, threads, 0, s>>>((const int32_t*)labels, count, K, st);
    }
    return launched(1);
}

static std::atomic<uint64_t> g_launches{0};
void note_launches(unsigned k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
uint64_t kernel_launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Repack label rows into uint8/uint16 codes with a padded row stride.
// ---------------------------------------------------------------------------
template <typename Lin, typename Lout>
__global__ void k_repack(const Lin* __restrict__ in, uint32_t n, uint64_t P, uint64_t lstride,
                         uint32_t K, Lout* __restrict__ out, DevStatus* st) {
    for (uint64_t p = blockIdx.x; p < P; p += gridDim.x) {
        const Lin* src = in + p * n;
        Lout* dst = out + p * lstride;
        for (uint64_t i = threadIdx.x; i < lstride; i += blockDim.x) {
            uint32_t g = 0;
            if (i < n) {
                g = (uint32_t)src[i];
                if (g >= K) {
                    raise_status(st, DEV_BAD_LABEL, 1u, (unsigned long long)(p * n + i));
                    g = K - 1;
                }
            }
            dst[i] = (Lout)g;
        }
    }
}

template <typename Lout>
static cudaError_t repack_from(const void* in, int in_type, uint32_t n, uint64_t P, uint32_t K,
                               Lout* out, uint64_t lstride, DevStatus* st, cudaStream_t s) {
    const unsigned blocks = (unsigned)(P < 152 * 16 ? P : 152 * 16);
    if (in_type == LABEL_U8)
        k_repack<uint8_t, Lout><<<blocks, 256, 0, s>>>((const uint8_t*)in, n, P, lstride, K, out, st);
    else if (in_type == LABEL_U16)
        k_repack<uint16_t, Lout><<<blocks, 256, 0, s>>>((const uint16_t*)in, n, P, lstride, K, out, st);
    else
        k_repack<int32_t, Lout><<<blocks, 256, 0, s>>>((const int32_t*)in, n, P, lstride, K, out, st);
    return launched(1);
}

cudaError_t launch_repack_labels(const void* in, int in_type, uint32_t n, uint64_t P, uint32_t K,
                                 void* out, int out_type, uint64_t lstride, DevStatus* st,
                                 cudaStream_t s) {
    if (out_type == LABEL_U8)
        return repack_from<uint8_t>(in, in_type, n, P, K, (uint8_t*)out, lstride, st, s);
    return repack_from<uint16_t>(in, in_type, n, P, K, (uint16_t*)out, lstride, st, s);
}

// ---------------------------------------------------------------------------
// Deterministic reduction: out[p] = sum_{r=0}^{rows-1} partials[r*P + p],
// always in ascending r, in FP64.  Replaces the order-dependent float
// reduction(+) of the GPU listing (Algorithm 3).
// ---------------------------------------------------------------------------
__global__ void k_reduce_rows(const double* __restrict__ partials, uint32_t rows, uint64_t P,
                              double* __restrict__ out) {
    uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double s = 0.0;
    for (uint32_t r = 0; r < rows; ++r) s += partials[(uint64_t)r * P + p];
    out[p] = s;
}

cudaError_t launch_reduce_rows(const double* partials, uint32_t rows, uint64_t P, double* out,
                               cudaStream_t s) {
    const int threads = 256;
    uint64_t blocks = (P + threads - 1) / threads;
    k_reduce_rows<<<(unsigned)blocks, threads, 0, s>>>(partials, rows, P, out);
    return launched(1);
}

__global__ void k_widen(const float* __restrict__ in, uint32_t K, double* __restrict__ out) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x)
        out[k] = (double)in[k];
}

cudaError_t launch_widen(const float* in, uint32_t K, double* out, cudaStream_t s) {
    const unsigned blocks = (K + 255) / 256 < 64 ? (K + 255) / 256 : 64;
    k_widen<<<blocks, 256, 0, s>>>(in, K, out);
    return launched(1);
}

// ---------------------------------------------------------------------------
// Permutations for the test (Sec. 1).  Counter-based Philox4x32-10 (Salmon,
// Moraes, Dror & Shaw, SC'11): 10 rounds of the 4x32 Philox S-box (two
// 32x32->64 multiplies by the round multipliers, high halves crossed and XORed
// with the other lanes and the round key), Weyl key schedule.  Each
// permutation p owns the stream of counters (block, 0, p, 0).
// ---------------------------------------------------------------------------
struct Philox4x32 {
    uint32_t k0, k1;
    uint32_t c0, c2;
    uint32_t buf[4];
    int used;

    __device__ __forceinline__ void block(uint32_t x[4]) const {
        uint32_t a0 = c0, a1 = 0u, a2 = c2, a3 = 0u;
        uint32_t key0 = k0, key1 = k1;
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            uint32_t hi0 = __umulhi(0xD2511F53u, a0), lo0 = 0xD2511F53u * a0;
            uint32_t hi1 = __umulhi(0xCD9E8D57u, a2), lo1 = 0xCD9E8D57u * a2;
            uint32_t b0 = hi1 ^ a1 ^ key0;
            uint32_t b2 = hi0 ^ a3 ^ key1;
            a0 = b0; a1 = lo1; a2 = b2; a3 = lo0;
            key0 += 0x9E3779B9u;
            key1 += 0xBB67AE85u;
        }
        x[0] = a0; x[1] = a1; x[2] = a2; x[3] = a3;
    }
    __device__ __forceinline__ uint32_t next() {
        if (used == 4) {
            block(buf);
            c0 += 1u;
            used = 0;
        }
        return buf[used++];
    }
    // Lemire (2019): high word of x*range, rejecting low words below 2^32 mod range.
    __device__ __forceinline__ uint32_t bounded(uint32_t range) {
        uint64_t m = (uint64_t)next() * range;
        uint32_t low = (uint32_t)m;
        if (low < range) {
            uint32_t thresh = (0u - range) % range;
            while (low < thresh) {
                m = (uint64_t)next() * range;
                low = (uint32_t)m;
            }
        }
        return (uint32_t)(m >> 32);
    }
};

template <typename L>
__global__ void k_copy_grouping(const int32_t* __restrict__ g, uint32_t n, uint64_t rows,
                                L* __restrict__ out) {
    uint64_t total = (uint64_t)n * rows;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += stride)
        out[k] = (L)g[k % n];
}

// One thread shuffles one row in place (row p = 1 + thread index).
template <typename L>
__global__ void k_fisher_yates(uint32_t n, uint64_t n_perms, uint64_t seed, L* __restrict__ out) {
    uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_perms) return;
    uint32_t p = (uint32_t)(t + 1);
    L* a = out + (uint64_t)p * n;
    Philox4x32 rng;
    rng.k0 = (uint32_t)seed;
    rng.k1 = (uint32_t)(seed >> 32);
    rng.c0 = 0u;
    rng.c2 = p;
    rng.used = 4;
    for (uint32_t i = n - 1; i >= 1; --i) {
        uint32_t j = rng.bounded(i + 1);
        L ai = a[i];
        a[i] = a[j];
        a[j] = ai;
    }
}

cudaError_t launch_permutations(const int32_t* grouping, uint32_t n, uint64_t n_perms,
                                uint64_t seed, void* out, int label_type, cudaStream_t s) {
    uint64_t rows = n_perms + 1;
    const int threads = 128;
    unsigned blocks = (unsigned)((n_perms + threads - 1) / threads);
    if (label_type == LABEL_U8) {
        k_copy_grouping<uint8_t><<<152 * 8, 256, 0, s>>>(grouping, n, rows, (uint8_t*)out);
        k_fisher_yates<uint8_t><<<blocks, threads, 0, s>>>(n, n_perms, seed, (uint8_t*)out);
    } else if (label_type == LABEL_U16) {
        k_copy_grouping<uint16_t><<<152 * 8, 256, 0, s>>>(grouping, n, rows, (uint16_t*)out);
        k_fisher_yates<uint16_t><<<blocks, threads, 0, s>>>(n, n_perms, seed, (uint16_t*)out);
    } else {
        k_copy_grouping<int32_t><<<152 * 8, 256, 0, s>>>(grouping, n, rows, (int32_t*)out);
        k_fisher_yates<int32_t><<<blocks, threads, 0, s>>>(n, n_perms, seed, (int32_t*)out);
    }
    return launched(2);
}

// ---------------------------------------------------------------------------
// Several tests in one pass.  Test t owns the label rows [rs[t], rs[t+1]) of
// the batch (rs: n_tests + 1 ascending offsets in device memory): the first
// is its observed grouping (row src[t] of `groupings`), the others its
// n_perms_t = rs[t+1] - rs[t] - 1 permutations, each the same shuffle a
// single test with that seed draws.
// ---------------------------------------------------------------------------
// Last test whose first row is <= row.
__device__ __forceinline__ uint32_t test_of_row(const uint64_t* __restrict__ rs, uint32_t n_tests,
                                                uint64_t row) {
    uint32_t lo = 0, hi = n_tests - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) / 2;
        if (rs[mid] <= row) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename L>
__global__ void k_copy_groupings(const int32_t* __restrict__ g, const uint32_t* __restrict__ src,
                                 uint32_t n, uint32_t n_tests, const uint64_t* __restrict__ rs,
                                 L* __restrict__ out) {
    const uint64_t total = (uint64_t)n * rs[n_tests];
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += stride) {
        const uint64_t row = k / n;
        const uint32_t t = test_of_row(rs, n_tests, row);
        out[k] = (L)g[(uint64_t)src[t] * n + (k - row * n)];
    }
}

// One thread per permutation: permutation index idx runs over all tests'
// permutations; test t's come after those of tests 0 .. t-1 (rs[t] - t of them).
template <typename L>
__global__ void k_fisher_yates_batch(uint32_t n, uint32_t n_tests, const uint64_t* __restrict__ rs,
                                     const uint64_t* __restrict__ seeds, uint64_t total_perms,
                                     L* __restrict__ out) {
    const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total_perms) return;
    uint32_t lo = 0, hi = n_tests - 1;   // last test with rs[t] - t <= idx
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) / 2;
        if (rs[mid] - mid <= idx) lo = mid; else hi = mid - 1;
    }
    const uint32_t t = lo;
    const uint32_t p = (uint32_t)(idx - (rs[t] - t) + 1);
    L* a = out + (rs[t] + p) * n;
    Philox4x32 rng;
    const uint64_t seed = seeds[t];
    rng.k0 = (uint32_t)seed;
    rng.k1 = (uint32_t)(seed >> 32);
    rng.c0 = 0u;
    rng.c2 = p;
    rng.used = 4;
    for (uint32_t i = n - 1; i >= 1; --i) {
        const uint32_t j = rng.bounded(i + 1);
        const L ai = a[i];
        a[i] = a[j];
        a[j] = ai;
    }
}

template <typename L>
static void perms_batch_t(const int32_t* g, const uint32_t* src, uint32_t n, uint32_t n_tests,
                          const uint64_t* rs, uint64_t total_perms, const uint64_t* seeds, L* out,
                          cudaStream_t s) {
    k_copy_groupings<L><<<152 * 8, 256, 0, s>>>(g, src, n, n_tests, rs, out);
    if (total_perms) {
        const unsigned blocks = (unsigned)((total_perms + 127) / 128);
        k_fisher_yates_batch<L><<<blocks, 128, 0, s>>>(n, n_tests, rs, seeds, total_perms, out);
    }
}

cudaError_t launch_permutations_batch(const int32_t* groupings, const uint32_t* src, uint32_t n,
                                      uint32_t n_tests, const uint64_t* rs, uint64_t total_perms,
                                      const uint64_t* seeds, void* out, int label_type, cudaStream_t s) {
    if (label_type == LABEL_U8)
        perms_batch_t<uint8_t>(groupings, src, n, n_tests, rs, total_perms, seeds, (uint8_t*)out, s);
    else if (label_type == LABEL_U16)
        perms_batch_t<uint16_t>(groupings, src, n, n_tests, rs, total_perms, seeds, (uint16_t*)out, s);
    else
        perms_batch_t<int32_t>(groupings, src, n, n_tests, rs, total_perms, seeds, (int32_t*)out, s);
    return launched(total_perms ? 2 : 1);
}

// ---------------------------------------------------------------------------
// Test statistics: s_T = (sum_{i<j} d^2)/n, F_obs, and the exceedance count
// #{p >= 1 : s_W[p] <= s_W[0]}.  For fixed s_T, n and K, pseudo-F decreases
// strictly in s_W, so F_p >= F_obs is the same event as s_W[p] <= s_W_obs.
// One block per test; test t's label rows are sW[rs[t] .. rs[t+1]), K = Ks[t].
// ---------------------------------------------------------------------------
__global__ void k_finalize(const double* __restrict__ sW_all, const uint64_t* __restrict__ rs,
                           const uint32_t* __restrict__ Ks, const double* __restrict__ sT_sum,
                           uint32_t n, TestScalars* out_all) {
    __shared__ unsigned long long cnt[32];
    const uint32_t t = blockIdx.x;
    const double* sW = sW_all + rs[t];
    const uint64_t n_perms = rs[t + 1] - rs[t] - 1;
    const uint32_t K = Ks[t];
    TestScalars* out = out_all + t;
    const double obs = sW[0];
    unsigned long long c = 0;
    for (uint64_t p = 1 + threadIdx.x; p <= n_perms; p += blockDim.x) c += (sW[p] <= obs) ? 1ull : 0ull;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) cnt[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tot = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += cnt[k];
        double s_T = sT_sum[0] / (double)n;
        double F = ((s_T - obs) / (double)(K - 1)) / (obs / (double)(n - K));
        out->s_T = s_T;
        out->s_W_obs = obs;
        out->F_obs = F;
        out->n_ge = tot;
        out->n_perms = n_perms;
        out->p_value = (double)(1 + tot) / (double)(1 + n_perms);
    }
}

cudaError_t launch_finalize_batch(const double* sW, uint32_t n_tests, const uint64_t* rs,
                                  const uint32_t* Ks, const double* sT_sum, uint32_t n,
                                  TestScalars* out, cudaStream_t s) {
    k_finalize<<<n_tests, 1024, 0, s>>>(sW, rs, Ks, sT_sum, n, out);
    return launched(1);
}

}  // namespace pmn
