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

// ---------------------------------------------------------------------------
// Shuffles.  Every permutation row is a Fisher-Yates shuffle of its test's
// observed labels: for i = n-1 down to 1, swap a[i] with a[j], j drawn
// uniformly from [0, i] by the row's Philox stream (seed of the test, counter
// (block, 0, p, 0) for row p).  One thread per row: a step depends on the
// previous one, so a row takes n steps of memory latency, and where the row
// lives decides that latency.
//
// Staged path (rows that fit, 4 or more to a block): a block copies the
// observed labels of up to 128 rows into shared memory, each thread shuffles
// its row there (a step is a few shared-memory accesses), and the block
// writes the rows back coalesced.  Global path (longer rows): each thread
// shuffles its row in place in HBM (the rows copied there first); every step
// then waits on an L2 or DRAM round trip.
//
// Rows of a batch map to (test, p) by the tests' row starts: test t owns rows
// [rs[t], rs[t+1]) of the output, the first its observed grouping (row src[t]
// of the groupings), then its permutations p = 1 .. n_perms_t; the
// permutation index idx runs over all tests' permutations in test order.
// ---------------------------------------------------------------------------
struct SingleRows {            // one test: rows 1 .. n_perms after the observed row 0
    uint64_t seed;
    __device__ __forceinline__ void get(uint64_t idx, uint32_t& p, uint64_t& sd, uint64_t& src,
                                        uint64_t& dst) const {
        p = (uint32_t)(idx + 1);
        sd = seed;
        src = 0;
        dst = idx + 1;
    }
};
struct BatchRows {             // several tests, rows by the row starts rs
    const uint64_t* rs;
    const uint64_t* seeds;
    const uint32_t* src_rows;
    uint32_t n_tests;
    __device__ __forceinline__ void get(uint64_t idx, uint32_t& p, uint64_t& sd, uint64_t& src,
                                        uint64_t& dst) const {
        uint32_t lo = 0, hi = n_tests - 1;   // last test with rs[t] - t <= idx
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) / 2;
            if (rs[mid] - mid <= idx) lo = mid; else hi = mid - 1;
        }
        p = (uint32_t)(idx - (rs[lo] - lo) + 1);
        sd = seeds[lo];
        src = src_rows[lo];
        dst = rs[lo] + p;
    }
};

// Philox4x32-10 block `blk` of row p's stream: counter (blk, 0, p, 0).
__device__ __forceinline__ void philox_block(uint32_t k0, uint32_t k1, uint32_t blk, uint32_t p,
                                             uint32_t x[4]) {
    Philox4x32 r;
    r.k0 = k0;
    r.k1 = k1;
    r.c0 = blk;
    r.c2 = p;
    r.block(x);
}

// The row's shuffle.  Draw w of the stream is word w % 4 of block w / 4, and
// step j's range is i + 1.  Steps go in groups of four while the stream is at
// a block boundary: one block gives the group's four draws, and when none of
// them needs Lemire's rejection check (low word >= range, the common case) the
// group's four swaps run on them.  The next group's block is computed before
// this group's swaps (it does not depend on them), so its arithmetic overlaps
// their memory accesses.  Any other step (a draw that needs the check, the
// stream off a block boundary after a rejection, the last steps) takes the
// draws one at a time exactly as the plain loop does, so every step uses the
// same draws in the same order.
template <typename L>
__device__ __forceinline__ void shuffle_row(L* a, uint32_t n, uint64_t seed, uint32_t p) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    uint32_t w = 0;                       // draws consumed (n - 1 steps need fewer than 2^32)
    uint32_t i = n - 1;
    uint32_t x[4];
    bool have = false;                    // x holds block w / 4
    while (i >= 1) {
        if ((w & 3u) == 0 && i >= 4) {
            if (!have) philox_block(k0, k1, w >> 2, p, x);
            uint32_t J[4];
            bool ok = true;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint64_t m = (uint64_t)x[q] * (uint64_t)(i + 1 - q);
                J[q] = (uint32_t)(m >> 32);
                ok = ok && (uint32_t)m >= i + 1 - q;
            }
            if (ok) {
                uint32_t y[4];
                const bool next = i >= 8;
                if (next) philox_block(k0, k1, (w >> 2) + 1, p, y);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t ii = i - q;
                    const L ai = a[ii];
                    a[ii] = a[J[q]];
                    a[J[q]] = ai;
                }
                i -= 4;
                w += 4;
                if (next) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) x[q] = y[q];
                }
                have = next;
                continue;
            }
        }
        // one step, draws one at a time (Lemire: reject low words below 2^32 mod range)
        have = false;
        const uint32_t range = i + 1;
        uint32_t z[4];
        philox_block(k0, k1, w >> 2, p, z);
        uint64_t m = (uint64_t)z[w & 3u] * range;
        ++w;
        if ((uint32_t)m < range) {
            const uint32_t thresh = (0u - range) % range;
            while ((uint32_t)m < thresh) {
                philox_block(k0, k1, w >> 2, p, z);
                m = (uint64_t)z[w & 3u] * range;
                ++w;
            }
        }
        const uint32_t j = (uint32_t)(m >> 32);
        const L ai = a[i];
        a[i] = a[j];
        a[j] = ai;
        --i;
    }
}

constexpr uint32_t FY_THREADS = 128;                 // threads of a staged block (rows <= this)
constexpr uint32_t FY_SMEM_MAX = 220u * 1024u;       // shared memory for a staged block's rows

// Staged path: block b shuffles permutation indices [b rows, (b+1) rows).
template <typename L, typename Rows>
__global__ void __launch_bounds__(FY_THREADS)
k_shuffle_staged(uint32_t n, uint64_t total, uint32_t rows, const int32_t* __restrict__ g,
                 L* __restrict__ out, Rows map) {
    extern __shared__ __align__(16) uint8_t fy_smem[];
    L* buf = reinterpret_cast<L*>(fy_smem);          // [rows][n]
    __shared__ uint64_t s_src[FY_THREADS], s_dst[FY_THREADS];
    const uint64_t idx0 = (uint64_t)blockIdx.x * rows;
    const uint32_t nr = (uint32_t)min((uint64_t)rows, total - idx0);
    uint32_t p = 0;
    uint64_t seed = 0;
    if (threadIdx.x < nr) {
        uint64_t src, dst;
        map.get(idx0 + threadIdx.x, p, seed, src, dst);
        s_src[threadIdx.x] = src * n;
        s_dst[threadIdx.x] = dst * n;
    }
    __syncthreads();
    for (uint32_t r = 0; r < nr; ++r)
        for (uint32_t c = threadIdx.x; c < n; c += FY_THREADS)
            buf[(uint64_t)r * n + c] = (L)g[s_src[r] + c];
    __syncthreads();
    if (threadIdx.x < nr) shuffle_row(buf + (uint64_t)threadIdx.x * n, n, seed, p);
    __syncthreads();
    for (uint32_t r = 0; r < nr; ++r)
        for (uint32_t c = threadIdx.x; c < n; c += FY_THREADS)
            out[s_dst[r] + c] = buf[(uint64_t)r * n + c];
}

// Global path: one thread per permutation index, its row already holding the
// observed labels.
template <typename L, typename Rows>
__global__ void k_shuffle_global(uint32_t n, uint64_t total, L* __restrict__ out, Rows map) {
    const uint64_t idx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    uint32_t p;
    uint64_t seed, src, dst;
    map.get(idx, p, seed, src, dst);
    shuffle_row(out + dst * n, n, seed, p);
}

// Observed rows: test t's grouping (row src[t] of g) into output row rs[t]; with
// `all`, into every row of the test (the global path shuffles them in place).
template <typename L>
__global__ void k_copy_groupings(const int32_t* __restrict__ g, const uint32_t* __restrict__ src,
                                 uint32_t n, uint32_t n_tests, const uint64_t* __restrict__ rs,
                                 bool all, L* __restrict__ out) {
    for (uint32_t t = blockIdx.y; t < n_tests; t += gridDim.y) {
        const uint64_t r0 = rs[t], r1 = all ? rs[t + 1] : r0 + 1;
        const int32_t* gs = g + (uint64_t)src[t] * n;
        const uint64_t total = (r1 - r0) * n;
        for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
             k += (uint64_t)gridDim.x * blockDim.x)
            out[r0 * n + k] = (L)gs[k % n];
    }
}
template <typename L>
__global__ void k_copy_grouping(const int32_t* __restrict__ g, uint32_t n, uint64_t rows,
                                L* __restrict__ out) {
    const uint64_t total = (uint64_t)n * rows;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (uint64_t)gridDim.x * blockDim.x)
        out[k] = (L)g[k % n];
}

static int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        sms = 152;
    return sms;
}
// Rows per staged block: as many as fit (at most 128) and no more than an even
// spread over the SMs needs; 0 selects the global path (fewer than 4 fit).
static uint32_t staged_rows(uint32_t n, size_t elem, uint64_t total) {
    const uint64_t fit = FY_SMEM_MAX / ((uint64_t)n * elem);
    if (fit < 4) return 0;
    const int sms = device_sms();
    const uint64_t spread = (total + (uint64_t)sms - 1) / (uint64_t)sms;
    uint64_t r = fit < FY_THREADS ? fit : FY_THREADS;
    if (spread < r) r = spread ? spread : 1;
    return (uint32_t)r;
}

// The shuffles of `total` permutation rows; `rows` from staged_rows (the global
// path's rows must already hold the observed labels).
template <typename L, typename Rows>
static cudaError_t launch_shuffles(uint32_t n, uint64_t total, const int32_t* g, L* out, Rows map,
                                   uint32_t rows, cudaStream_t s) {
    if (total == 0) return cudaSuccess;
    if (rows) {
        const size_t smem = (size_t)rows * n * sizeof(L);
        cudaError_t e = cudaFuncSetAttribute(k_shuffle_staged<L, Rows>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        const uint64_t blocks = (total + rows - 1) / rows;
        if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
        k_shuffle_staged<L, Rows><<<(unsigned)blocks, FY_THREADS, smem, s>>>(n, total, rows, g, out, map);
    } else {
        // one thread per row, the rows spread over every SM (a step's accesses
        // touch a different cache line in every lane): blocks of
        // ceil(rows / SMs) threads, at most a warp
        const int sms = device_sms();
        const uint64_t per_sm = (total + (uint64_t)sms - 1) / (uint64_t)sms;
        const unsigned threads = (unsigned)(per_sm < 32 ? per_sm : 32);
        if ((total + threads - 1) / threads > 0x7FFFFFFFull) return cudaErrorInvalidValue;
        k_shuffle_global<L, Rows><<<(unsigned)((total + threads - 1) / threads), threads, 0, s>>>(
            n, total, out, map);
    }
    return cudaGetLastError();
}

template <typename L>
static cudaError_t permutations_t(const int32_t* grouping, uint32_t n, uint64_t n_perms, uint64_t seed,
                                  L* out, cudaStream_t s) {
    const uint32_t rows = staged_rows(n, sizeof(L), n_perms);
    // staged: only the observed row is copied; global: every row, then shuffled in place
    k_copy_grouping<L><<<152 * 8, 256, 0, s>>>(grouping, n, rows ? 1 : n_perms + 1, out);
    return launch_shuffles<L>(n, n_perms, grouping, out, SingleRows{seed}, rows, s);
}

cudaError_t launch_permutations(const int32_t* grouping, uint32_t n, uint64_t n_perms,
                                uint64_t seed, void* out, int label_type, cudaStream_t s) {
    cudaError_t e;
    if (label_type == LABEL_U8)
        e = permutations_t<uint8_t>(grouping, n, n_perms, seed, (uint8_t*)out, s);
    else if (label_type == LABEL_U16)
        e = permutations_t<uint16_t>(grouping, n, n_perms, seed, (uint16_t*)out, s);
    else
        e = permutations_t<int32_t>(grouping, n, n_perms, seed, (int32_t*)out, s);
    return e != cudaSuccess ? e : launched(2);
}

template <typename L>
static cudaError_t perms_batch_t(const int32_t* g, const uint32_t* src, uint32_t n, uint32_t n_tests,
                                 const uint64_t* rs, uint64_t total_perms, const uint64_t* seeds, L* out,
                                 cudaStream_t s) {
    const uint32_t rows = staged_rows(n, sizeof(L), total_perms);
    const dim3 cgrid(152 * 2, n_tests < 65535u ? n_tests : 65535u);
    k_copy_groupings<L><<<cgrid, 256, 0, s>>>(g, src, n, n_tests, rs, rows == 0, out);
    return launch_shuffles<L>(n, total_perms, g, out, BatchRows{rs, seeds, src, n_tests}, rows, s);
}

cudaError_t launch_permutations_batch(const int32_t* groupings, const uint32_t* src, uint32_t n,
                                      uint32_t n_tests, const uint64_t* rs, uint64_t total_perms,
                                      const uint64_t* seeds, void* out, int label_type, cudaStream_t s) {
    cudaError_t e;
    if (label_type == LABEL_U8)
        e = perms_batch_t<uint8_t>(groupings, src, n, n_tests, rs, total_perms, seeds, (uint8_t*)out, s);
    else if (label_type == LABEL_U16)
        e = perms_batch_t<uint16_t>(groupings, src, n, n_tests, rs, total_perms, seeds, (uint16_t*)out, s);
    else
        e = perms_batch_t<int32_t>(groupings, src, n, n_tests, rs, total_perms, seeds, (int32_t*)out, s);
    return e != cudaSuccess ? e : launched(total_perms ? 2 : 1);
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
