// Auxiliary kernels of the s_W path: label validation, the fixed-order
// cross-tile reduction, device permutation generation for the permutation
// test (Sec. 1) and the test's final statistics.
#include "common.cuh"

#include <algorithm>
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
// (block, 0, p, 0) for row p).  A step depends on the previous one, so a row
// takes n dependent steps; where the row lives and what sits on a step's
// chain decide their latency (fy_plan picks the path).
//
// Shared-memory path (k_shuffle_warp): a block copies the observed labels of
// up to 128 rows into shared memory, one to four rows to a warp; one lane per
// row walks its steps there (a step is a few shared-memory accesses) while
// the row's other lanes prepare the draws and swap targets, and the block
// writes the rows back coalesced.  Global path (rows too long for shared
// memory): each thread shuffles its row in place in HBM (the rows copied
// there first); every step then waits on an L2 or DRAM round trip.
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

// Four Fisher-Yates steps i, i-1, i-2, i-3 with targets J[0..3] (J[t] <= i-t).
// When no target falls among the four positions and the targets differ, the
// four swaps touch disjoint positions, so all eight loads go out before the
// eight stores (one memory round trip instead of four); otherwise the swaps
// run one after the other.  Either way the result is that of the sequence.
template <typename L>
__device__ __forceinline__ void swap4(L* a, uint32_t i, const uint32_t (&J)[4]) {
    const uint32_t lo = i - 3;
    const bool disjoint = J[0] < lo && J[1] < lo && J[2] < lo && J[3] < lo && J[0] != J[1] &&
                          J[0] != J[2] && J[0] != J[3] && J[1] != J[2] && J[1] != J[3] && J[2] != J[3];
    if (disjoint) {
        const L v0 = a[i], v1 = a[i - 1], v2 = a[i - 2], v3 = a[i - 3];
        const L u0 = a[J[0]], u1 = a[J[1]], u2 = a[J[2]], u3 = a[J[3]];
        a[i] = u0;
        a[i - 1] = u1;
        a[i - 2] = u2;
        a[i - 3] = u3;
        a[J[0]] = v0;
        a[J[1]] = v1;
        a[J[2]] = v2;
        a[J[3]] = v3;
    } else {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint32_t ii = i - t;
            const L ai = a[ii];
            a[ii] = a[J[t]];
            a[J[t]] = ai;
        }
    }
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
                swap4(a, i, J);
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

constexpr uint32_t FY_SMEM_MAX = 220u * 1024u;       // shared memory for a block's rows

// Shared-memory path: one to four rows per warp, each with 32 / RPW lanes,
// the rows in shared memory.  With a thread per row, a block's rows would sit
// on the lanes of a few warps, every step a chain of dependent instructions
// (Philox rounds, multiplies, checks, swaps) with few other warps to hide it,
// and the lanes' rows would share banks.  Here the first lane of each
// row's group walks the row's steps and the group prepares them: at each
// refill the row's next Philox blocks (32 blocks, 128 draws, for a row alone in
// its warp, else 16 blocks, 64 draws) are computed and, assuming
// no rejection since the refill, for each block the swap targets of the four
// steps its draws serve, whether any of the draws needs Lemire's rejection
// check (FY_OK clear) and whether the four swaps touch disjoint positions
// (FY_DISJOINT); both flags ride in the top bits of the first target (n <
// 2^30 here).  Without a rejection, i + w (step index plus draws consumed)
// stays constant, so the walker uses a prepared group exactly while i + w
// equals its value at the refill.  Off that path (a step whose draw needs the
// check, the steps after a rejection up to the next refill, the last three
// steps) the walker computes its draws from the Philox blocks itself, one at
// a time exactly as the plain loop.  The rows are bit-identical to the other
// paths.
// draws prepared per refill (a row's targets and flags take 4 bytes a draw)
__host__ __device__ constexpr uint32_t fy_words(int rpw) { return rpw == 1 ? 128u : 64u; }
constexpr uint32_t FY_ROWS_MAX = 128;          // rows of a warp-path block (4 to a warp)
constexpr uint32_t FY_OK = 1u << 31, FY_DISJOINT = 1u << 30, FY_J = FY_DISJOINT - 1u;
constexpr uint64_t FY_GLOBAL_RATIO = 8;       // rows / warp-path residency from which HBM wins
constexpr uint64_t FY_GLOBAL_MAX_FIT = 3;     // ... for rows that fit at most this many to a block

// The walker's steps while its draws lie in [wbase, wbase + WORDS): from
// step i (range i + 1) and draw w until the row is done or the next step's
// first draw lies beyond.  wj: the prepared groups, valid while i + w == inv.
template <typename L, uint32_t WORDS>
__device__ __forceinline__ void fy_steps(L* a, const uint32_t* wj, uint32_t wbase, uint32_t inv,
                                         uint32_t& i_, uint32_t& w_, uint32_t k0, uint32_t k1,
                                         uint32_t p) {
    uint32_t i = i_, w = w_;
    const uint32_t wend = wbase + WORDS;
    uint32_t zb = 0xFFFFFFFFu, z[4];             // Philox block zb, computed on demand
    while (i >= 1 && w < wend) {
        if ((w & 3u) == 0 && i >= 4 && w + 4 <= wend) {
            if (i + w == inv) {
                // prepared groups; the next group is read before this group's swaps
                uint32_t gq = (w - wbase) >> 2;
                uint4 jq = *reinterpret_cast<const uint4*>(wj + 4 * gq);
                while ((jq.x & FY_OK) && i >= 4) {
                    const uint32_t J[4] = {jq.x & FY_J, jq.y, jq.z, jq.w};
                    const bool dis = (jq.x & FY_DISJOINT) != 0;
                    const bool more = gq + 1 < WORDS / 4;
                    if (more) jq = *reinterpret_cast<const uint4*>(wj + 4 * (gq + 1));
                    if (dis) {
                        const L v0 = a[i], v1 = a[i - 1], v2 = a[i - 2], v3 = a[i - 3];
                        const L u0 = a[J[0]], u1 = a[J[1]], u2 = a[J[2]], u3 = a[J[3]];
                        a[i] = u0;
                        a[i - 1] = u1;
                        a[i - 2] = u2;
                        a[i - 3] = u3;
                        a[J[0]] = v0;
                        a[J[1]] = v1;
                        a[J[2]] = v2;
                        a[J[3]] = v3;
                    } else {
                        swap4(a, i, J);
                    }
                    i -= 4;
                    w += 4;
                    ++gq;
                    if (!more) break;
                }
                if (w >= wend || i < 1) break;
                if (!((w & 3u) == 0 && i >= 4 && i + w == inv && !(wj[w - wbase] & FY_OK))) continue;
                // else: this group's draws need the check; one plain step below
            } else {
                // after a rejection: the group from its Philox block
                uint32_t x[4];
                philox_block(k0, k1, w >> 2, p, x);
                uint32_t J[4];
                bool ok = true;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint64_t m = (uint64_t)x[t] * (uint64_t)(i + 1 - t);
                    J[t] = (uint32_t)(m >> 32);
                    ok = ok && (uint32_t)m >= i + 1 - t;
                }
                if (ok) {
                    swap4(a, i, J);
                    i -= 4;
                    w += 4;
                    continue;
                }
            }
        }
        const uint32_t range = i + 1;
        if (zb != (w >> 2)) {
            zb = w >> 2;
            philox_block(k0, k1, zb, p, z);
        }
        uint64_t m = (uint64_t)z[w & 3u] * range;
        ++w;
        if ((uint32_t)m < range) {
            const uint32_t thresh = (0u - range) % range;
            while ((uint32_t)m < thresh) {
                if (zb != (w >> 2)) {
                    zb = w >> 2;
                    philox_block(k0, k1, zb, p, z);
                }
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
    i_ = i;
    w_ = w;
}

// Block b shuffles permutation indices [b rows, (b+1) rows), RPW rows to a
// warp (rows <= 32 RPW), row r of the block at r * ns in shared memory after
// the rows' prepared groups.  The walkers of one warp advance together (their
// rows have the same length).
template <typename L, typename Rows, int RPW>
__global__ void __launch_bounds__(1024)
k_shuffle_warp(uint32_t n, uint32_t ns, uint64_t total, uint32_t rows, const int32_t* __restrict__ g,
               L* __restrict__ out, Rows map) {
    constexpr uint32_t HL = 32 / RPW;            // lanes per row
    constexpr uint32_t WORDS = fy_words(RPW);
    extern __shared__ __align__(16) uint8_t fy_smem[];
    L* buf = reinterpret_cast<L*>(fy_smem + (size_t)rows * WORDS * 4);   // [rows][ns]
    __shared__ uint64_t s_src[FY_ROWS_MAX], s_dst[FY_ROWS_MAX], s_seed[FY_ROWS_MAX];
    __shared__ uint32_t s_p[FY_ROWS_MAX];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t h = lane % HL, walker = lane - h;   // helper index, the group's first lane
    const uint32_t row = warp * RPW + lane / HL;
    const uint64_t idx0 = (uint64_t)blockIdx.x * rows;
    const uint32_t nr = (uint32_t)min((uint64_t)rows, total - idx0);
    if (threadIdx.x < nr) {
        uint32_t p;
        uint64_t seed, src, dst;
        map.get(idx0 + threadIdx.x, p, seed, src, dst);
        s_src[threadIdx.x] = src * n;
        s_dst[threadIdx.x] = dst * n;
        s_seed[threadIdx.x] = seed;
        s_p[threadIdx.x] = p;
    }
    __syncthreads();
    for (uint32_t r = 0; r < nr; ++r)
        for (uint32_t c = threadIdx.x; c < n; c += blockDim.x)
            buf[(uint64_t)r * ns + c] = (L)g[s_src[r] + c];
    __syncthreads();
    if (warp * RPW < nr) {
        const bool active = row < nr;
        const uint32_t rr = active ? row : 0;
        L* a = buf + (uint64_t)rr * ns;
        uint32_t* wj = reinterpret_cast<uint32_t*>(fy_smem + (size_t)rr * WORDS * 4);
        const uint64_t seed = s_seed[rr];
        const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32), p = s_p[rr];
        uint32_t i = active ? n - 1 : 0, w = 0;   // the row's step and draw (its walker's)
        while (__any_sync(0xffffffffu, i >= 1)) {
            const uint32_t blk0 = w >> 2;
            const uint32_t inv = i + w;
            if (i >= 1) {
                for (uint32_t b = h; b < WORDS / 4; b += HL) {   // this lane's blocks
                    uint32_t x[4];
                    philox_block(k0, k1, blk0 + b, p, x);
                    // block b's group: steps il .. il - 3 on draws 4 (blk0 + b) .. +3
                    const uint32_t w4 = 4 * (blk0 + b);
                    uint32_t flags = 0, J[4] = {0u, 0u, 0u, 0u};
                    if (w4 >= w && w4 + 4 <= inv) {
                        const uint32_t il = inv - w4;
                        bool ok = true;
#pragma unroll
                        for (int t = 0; t < 4; ++t) {
                            const uint64_t m = (uint64_t)x[t] * (uint64_t)(il + 1 - t);
                            J[t] = (uint32_t)(m >> 32);
                            ok = ok && (uint32_t)m >= il + 1 - t;
                        }
                        const uint32_t lo = il - 3;
                        const bool dis = J[0] < lo && J[1] < lo && J[2] < lo && J[3] < lo && J[0] != J[1] &&
                                         J[0] != J[2] && J[0] != J[3] && J[1] != J[2] && J[1] != J[3] &&
                                         J[2] != J[3];
                        flags = (ok ? FY_OK : 0u) | (dis ? FY_DISJOINT : 0u);
                    }
                    *reinterpret_cast<uint4*>(wj + 4 * b) = make_uint4(J[0] | flags, J[1], J[2], J[3]);
                }
            }
            __syncwarp();
            if (h == 0 && i >= 1) fy_steps<L, WORDS>(a, wj, 4 * blk0, inv, i, w, k0, k1, p);
            __syncwarp();
            i = __shfl_sync(0xffffffffu, i, walker);
            w = __shfl_sync(0xffffffffu, w, walker);
        }
    }
    __syncthreads();
    for (uint32_t r = 0; r < nr; ++r)
        for (uint32_t c = threadIdx.x; c < n; c += blockDim.x)
            out[s_dst[r] + c] = buf[(uint64_t)r * ns + c];
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
// Where the rows are shuffled.  In shared memory (k_shuffle_warp), a block
// taking as many rows as fit (at most FY_ROWS_MAX), then as few as keep the
// same number of waves over the SMs.  When not one row fits, and for very
// long rows (at most FY_GLOBAL_MAX_FIT to a block) when the rows to shuffle
// number FY_GLOBAL_RATIO times what shared memory holds on the GPU at once,
// in place in HBM (global path, rows == 0): every row runs at once, a step's
// latency an HBM round trip per four steps.  Measured alone (uint8 rows,
// ms): n = 15,000 / 9,999 rows: shared memory 3.1, global 4.7; 30,000 /
// 9,999: 9.5, 10.5; 60,000 / 9,999: 41.6 (earlier shared-memory kernel),
// 23.2; 100,000 / 8,191: 84.9 (earlier), 35.4; 100,000 / 999: 11.9, 16.7.
// Beside other kernels (a server's fused batches) the global path fares
// worse: taken for every row count above 10x the shared-memory residency, it
// cut a served mix's capacity by 14 %.  A thread per row in shared memory
// (the previous kernel) was slower at every size measured, up to 2.5x.
struct FyPlan {
    uint32_t rows;  // rows to a block (0: the global path)
    uint32_t rpw;   // rows to a warp (1, 2 or 4)
    uint32_t ns;    // shared-memory row stride (elements)
};
static FyPlan fy_plan(uint32_t n, size_t elem, uint64_t total) {
    const int sms = device_sms();
    uint64_t spread = (total + (uint64_t)sms - 1) / (uint64_t)sms;
    if (spread < 1) spread = 1;
    // rows in shared memory start an odd number of 4-byte words apart, so the
    // same position of up to 32 rows falls in 32 distinct banks
    uint64_t words = ((uint64_t)n * elem + 3) / 4;
    if ((words & 1u) == 0) ++words;
    const uint64_t row_bytes = words * 4;
    const uint32_t ns = (uint32_t)(row_bytes / elem);
    // as many rows as fit (at most FY_ROWS_MAX), then as few as keep the same
    // number of waves over the SMs, so the last wave is not a sliver
    uint64_t fit_w = FY_SMEM_MAX / (row_bytes + 4 * fy_words(2));
    if (fit_w <= 32) fit_w = FY_SMEM_MAX / (row_bytes + 4 * fy_words(1));   // a row alone in its warp
    if (fit_w == 0) return FyPlan{0u, 0u, ns};
    if (fit_w <= FY_GLOBAL_MAX_FIT && total >= FY_GLOBAL_RATIO * fit_w * (uint64_t)sms)
        return FyPlan{0u, 0u, ns};
    const uint64_t cap = std::min<uint64_t>(fit_w, FY_ROWS_MAX);
    const uint64_t waves = (total + cap * sms - 1) / (cap * sms);
    const uint64_t r64 = std::min<uint64_t>(cap, (total + waves * sms - 1) / (waves * sms));
    uint32_t r = (uint32_t)std::max<uint64_t>(r64, 1);
    auto rpw_of = [](uint32_t rows) { return rows <= 32 ? 1u : rows <= 64 ? 2u : 4u; };
    while (r > 1 && (uint64_t)r * (row_bytes + 4 * fy_words((int)rpw_of(r))) > FY_SMEM_MAX) --r;
    return FyPlan{r, rpw_of(r), ns};
}

template <typename L, typename Rows, int RPW>
static cudaError_t launch_warp_path(uint32_t n, uint32_t ns, uint64_t total, const int32_t* g, L* out,
                                    Rows map, uint32_t rows, cudaStream_t s) {
    const size_t smem = (size_t)rows * (4 * fy_words(RPW) + (size_t)ns * sizeof(L));
    // the kernel's shared-memory limit is one value for every launch (a call
    // that set its own size could race with another thread's launch of a
    // larger block and make that launch fail); smem <= FY_SMEM_MAX by plan
    cudaError_t e = cudaFuncSetAttribute(k_shuffle_warp<L, Rows, RPW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FY_SMEM_MAX);
    if (e != cudaSuccess) return e;
    const uint64_t blocks = (total + rows - 1) / rows;
    if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    const unsigned threads = 32u * ((rows + RPW - 1) / RPW);
    k_shuffle_warp<L, Rows, RPW><<<(unsigned)blocks, threads, smem, s>>>(n, ns, total, rows, g, out, map);
    return cudaSuccess;
}

// The shuffles of `total` permutation rows by the plan from fy_plan (the global
// path's rows must already hold the observed labels).
template <typename L, typename Rows>
static cudaError_t launch_shuffles(uint32_t n, uint64_t total, const int32_t* g, L* out, Rows map,
                                   FyPlan pl, cudaStream_t s) {
    if (total == 0) return cudaSuccess;
    const uint32_t rows = pl.rows;
    if (rows) {
        cudaError_t e = pl.rpw == 4   ? launch_warp_path<L, Rows, 4>(n, pl.ns, total, g, out, map, rows, s)
                        : pl.rpw == 2 ? launch_warp_path<L, Rows, 2>(n, pl.ns, total, g, out, map, rows, s)
                                      : launch_warp_path<L, Rows, 1>(n, pl.ns, total, g, out, map, rows, s);
        if (e != cudaSuccess) return e;
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
    const FyPlan pl = fy_plan(n, sizeof(L), n_perms);
    // shared-memory path: only the observed row is copied; global: every
    // row, then shuffled in place
    k_copy_grouping<L><<<152 * 8, 256, 0, s>>>(grouping, n, pl.rows ? 1 : n_perms + 1, out);
    return launch_shuffles<L>(n, n_perms, grouping, out, SingleRows{seed}, pl, s);
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
    const FyPlan pl = fy_plan(n, sizeof(L), total_perms);
    const dim3 cgrid(152 * 2, n_tests < 65535u ? n_tests : 65535u);
    k_copy_groupings<L><<<cgrid, 256, 0, s>>>(g, src, n, n_tests, rs, pl.rows == 0, out);
    return launch_shuffles<L>(n, total_perms, g, out, BatchRows{rs, seeds, src, n_tests}, pl, s);
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
