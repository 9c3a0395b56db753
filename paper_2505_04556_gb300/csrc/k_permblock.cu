// Perm-blocked CUDA-core s_W: one 64 x 64 tile of D^2 in shared memory is
// reused by a block of label rows.  Two kernels: the paired kernel below the
// first (uint8 codes, the default: 256 label rows per block, two per thread,
// one packed FP16 compare per two evaluations) and this one (128 label rows
// per block, one per thread, FP32 compare-and-set; uint16 codes and plan
// variant 1).
//
// Algorithm 1 evaluates, per label row p and pair i < j, the test
// g_p(i) == g_p(j) and adds d_ij^2 * w_{g_p(i)} (Sec. 2).  Here a CTA owns a
// band of 64 rows and 128 label rows and walks the band's column tiles from
// the diagonal to the end:
//   * the tile is loaded once (128-bit, coalesced), squared, and masked to the
//     strict upper triangle (j > i, j < n) before it is stored, so the hot
//     loop needs no bounds or triangle tests;
//   * every thread keeps its row's 64 column labels in registers as floats
//     2^23 + g, so one float compare yields the 0/1 selector, and two
//     selectors feed one packed FP32x2 FMA (2 evaluations per FFMA2);
//   * D^2 is read from shared memory with 128-bit broadcast loads;
//   * as in Algorithm 2, the row segment is summed unweighted and multiplied
//     by w_{g_p(i)} once.  Each thread converts its 64 row weights to FP32
//     once per CTA (shared memory); a row segment (64 terms, four FP32
//     partial sums) is weighted with one FP32 FMA into a group sum of 8
//     rows, and each group sum is added to an FP64 total, so the slow FP64
//     pipe sees two operations per 512 evaluations.  Worst-case relative
//     error of a group: about 28 unit roundoffs (16-term chains, the partial
//     reduction, the weight's rounding and product, the 8-row chain), 1.7e-6;
//     each thread's 64 row labels are staged in shared memory once per CTA
//     (not re-read from global memory for every column tile); the CTA writes
//     one FP64 partial per (band, label row).
// Labels arrive as uint8 (K <= 256) or uint16 codes whose row stride is a
// multiple of 16 bytes, so each thread loads its 64 column labels of a full
// tile with 16-byte loads (the ragged last tile uses guarded scalar loads).
#include "common.cuh"

namespace pmn {

constexpr int PB_P = 128;  // label rows per CTA (one per thread)
constexpr int PB_T = 64;   // band height and column-tile width
constexpr int PB_G = 8;    // rows per FP32 group sum
constexpr uint32_t PB_D2_BYTES = PB_T * PB_T * 4;   // 16 KB
constexpr uint32_t PB_W_BYTES = PB_T * PB_P * 4;    // 32 KB
template <typename L>
constexpr uint32_t pb_smem_bytes() { return PB_D2_BYTES + PB_W_BYTES + PB_T * PB_P * sizeof(L); }

__device__ __forceinline__ float code_u8(uint32_t word, int k) {
    // bytes: [label byte k, 0, 0, 0x4B] -> float 2^23 + label
    return __uint_as_float(__byte_perm(word, 0x4B000000u, 0x7440u | (uint32_t)k));
}
__device__ __forceinline__ float code_u16(uint32_t word, int k) {
    return __uint_as_float(__byte_perm(word, 0x4B000000u, k ? 0x7432u : 0x7410u));
}
__device__ __forceinline__ float code_of(uint32_t g) { return __uint_as_float(0x4B000000u | g); }

// 1.0f if a == b else 0.0f, in one compare-and-set
__device__ __forceinline__ float select_eq(float a, float b) {
    float d;
    asm("set.eq.f32.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

template <typename L>
__device__ __forceinline__ void load_col_codes(const L* __restrict__ g, uint32_t j0, float* cl);

template <>
__device__ __forceinline__ void load_col_codes<uint8_t>(const uint8_t* __restrict__ g, uint32_t j0,
                                                        float* cl) {
    const uint4* src = reinterpret_cast<const uint4*>(g + j0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 v = __ldg(src + q);
        const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int k = 0; k < 4; ++k) cl[16 * q + 4 * t + k] = code_u8(w4[t], k);
    }
}

template <>
__device__ __forceinline__ void load_col_codes<uint16_t>(const uint16_t* __restrict__ g,
                                                         uint32_t j0, float* cl) {
    const uint4* src = reinterpret_cast<const uint4*>(g + j0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint4 v = __ldg(src + q);
        const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int k = 0; k < 2; ++k) cl[8 * q + 2 * t + k] = code_u16(w4[t], k);
    }
}

template <typename L, bool VEC>
__global__ void __launch_bounds__(PB_P, 4)
k_sw_permblock(const float* __restrict__ mat, uint32_t n, uint64_t ld, const L* __restrict__ labels,
               uint64_t lstride, uint64_t P, const WeightMap wm, uint32_t K,
               uint32_t n_pblocks, double* __restrict__ partials, const DevStatus* __restrict__ st) {
    // dynamic shared memory: the D^2 tile, then per (row, thread) the row's
    // FP32 weight and its label (clamped to K - 1)
    extern __shared__ __align__(16) uint8_t pb_smem[];
    float (*d2)[PB_T] = reinterpret_cast<float (*)[PB_T]>(pb_smem);
    float (*wrow)[PB_P] = reinterpret_cast<float (*)[PB_P]>(pb_smem + PB_D2_BYTES);
    L (*lrow)[PB_P] = reinterpret_cast<L (*)[PB_P]>(pb_smem + PB_D2_BYTES + PB_W_BYTES);
    const uint32_t band = blockIdx.x / n_pblocks;
    const uint32_t q = blockIdx.x % n_pblocks;
    const uint64_t p = (uint64_t)q * PB_P + threadIdx.x;
    const bool active = p < P;
    // a recorded device error skips the work; the vote keeps the exit uniform
    // across the block even if the status word changes while threads read it
    if (__syncthreads_or(st->code != DEV_OK)) {
        if (active) partials[(uint64_t)band * P + p] = 0.0;
        return;
    }
    // inactive threads of the last block mirror the last row so loads stay in bounds
    const L* g = labels + (active ? p : P - 1) * lstride;
    const double* w = wm.row(active ? p : P - 1);
    const uint32_t r0 = band * PB_T;
    const uint32_t rows = min((uint32_t)PB_T, n - 1 - r0);  // row n-1 has no pairs
    double total = 0.0;
    for (uint32_t r = 0; r < rows; ++r) {
        const uint32_t gr = min((uint32_t)g[r0 + r], K - 1);
        lrow[r][threadIdx.x] = (L)gr;
        wrow[r][threadIdx.x] = (float)__ldg(w + gr);
    }

    for (uint32_t j0 = r0; j0 < n; j0 += PB_T) {
        __syncthreads();  // the previous tile has been consumed
        // ---- stage the D^2 tile, masked to j > i and j < n ----
#pragma unroll
        for (int e = threadIdx.x; e < PB_T * PB_T / 4; e += PB_P) {
            const int rr = e >> 4, cc = (e & 15) * 4;
            const uint32_t i = r0 + rr, j = j0 + cc;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < n) {
                const float* src = mat + (uint64_t)i * ld + j;
                if (VEC && j + 3 < n) {
                    v = __ldg(reinterpret_cast<const float4*>(src));
                } else {
                    if (j < n) v.x = __ldg(src);
                    if (j + 1 < n) v.y = __ldg(src + 1);
                    if (j + 2 < n) v.z = __ldg(src + 2);
                    if (j + 3 < n) v.w = __ldg(src + 3);
                }
            }
            v.x = (j > i && j < n) ? v.x * v.x : 0.f;
            v.y = (j + 1 > i && j + 1 < n) ? v.y * v.y : 0.f;
            v.z = (j + 2 > i && j + 2 < n) ? v.z * v.z : 0.f;
            v.w = (j + 3 > i && j + 3 < n) ? v.w * v.w : 0.f;
            *reinterpret_cast<float4*>(&d2[rr][cc]) = v;
        }
        // ---- this thread's 64 column labels (padding beyond n is 0; its D^2 is 0) ----
        float cl[PB_T];
        if (j0 + PB_T <= n) {
            load_col_codes<L>(g, j0, cl);
        } else {
#pragma unroll
            for (int c = 0; c < PB_T; ++c) cl[c] = code_of(j0 + c < n ? (uint32_t)g[j0 + c] : 0u);
        }
        __syncthreads();

        for (uint32_t rg = 0; rg < rows; rg += PB_G) {
            const uint32_t rend = min(rg + PB_G, rows);
            float group = 0.f;
            // two rows per iteration: their compare/FMA streams interleave
#pragma unroll 2
            for (uint32_t r = rg; r < rend; ++r) {
                const float fgi = code_of(lrow[r][threadIdx.x]);
                const float4* drow = reinterpret_cast<const float4*>(&d2[r][0]);
                float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
                for (int c4 = 0; c4 < PB_T / 4; ++c4) {
                    const float4 dv = drow[c4];
                    const float e0 = select_eq(cl[4 * c4 + 0], fgi);
                    const float e1 = select_eq(cl[4 * c4 + 1], fgi);
                    const float e2 = select_eq(cl[4 * c4 + 2], fgi);
                    const float e3 = select_eq(cl[4 * c4 + 3], fgi);
                    a0 = __ffma2_rn(make_float2(e0, e1), make_float2(dv.x, dv.y), a0);
                    a1 = __ffma2_rn(make_float2(e2, e3), make_float2(dv.z, dv.w), a1);
                }
                // weight applied once per row segment (Algorithm 2)
                group = fmaf((a0.x + a0.y) + (a1.x + a1.y), wrow[r][threadIdx.x], group);
            }
            total += (double)group;
        }
    }
    if (active) partials[(uint64_t)band * P + p] = total;
}

// ---------------------------------------------------------------------------
// Paired variant (uint8 or uint16 codes): each thread evaluates TWO label rows
// p and p' (p' = p + 128) at once.  Its 64 column labels of both rows are held
// as FP16 pairs (uint8 code L as the pattern 0x43LL, uint16 code L < 2048 as
// 0x4000 + L: distinct finite normal values either way), and one packed FP16
// equality test against the row key (the pattern pair of g_p(i), g_p'(i)) sets
// two predicates, which gate two FP32 adds of the same d^2:
//   setp.eq.f16x2  P|Q, cl[j], key     (one compare for two evaluations)
//   @P add.f32     acc_p,  acc_p,  d2
//   @Q add.f32     acc_p', acc_p', d2
// so a pair-evaluation costs one compare and two adds, none of them a
// compare-and-set.  Row segments are summed in FP32 (two chains per label
// row), weighted once per row segment (Algorithm 2) in FP32 into an 8-row
// group sum, and group sums are added in FP64, as in the kernel above.  The
// weight sets of the CTA's label rows are staged once as an FP32 table in
// shared memory (the launcher uses this kernel only when they fit), so the
// FP64 pipe sees no per-row work.
// ---------------------------------------------------------------------------
constexpr int PB2_THREADS = 128;              // threads per CTA
constexpr int PB2_ROWS = 2 * PB2_THREADS;     // label rows per CTA
constexpr uint32_t PB2_WTAB = 2048;                          // FP32 weights staged per CTA (8 KB)

// The codes of the paired kernel: a row entry holds a row's codes for p and
// p' (uint8: 8 bits each, uint16: 16 bits each), key() makes their FP16
// pattern pair, cols() the pattern pairs of 64 columns from 16-byte loads.
template <typename L> struct PairCodes;
template <> struct PairCodes<uint8_t> {
    using Row = uint16_t;
    static __device__ __forceinline__ Row pack(uint32_t la, uint32_t lb) { return (Row)(la | (lb << 8)); }
    static __device__ __forceinline__ uint32_t key(uint32_t row) { return __byte_perm(row, 0x43u, 0x4140); }
    static __device__ __forceinline__ uint32_t la(uint32_t row) { return row & 0xFFu; }
    static __device__ __forceinline__ uint32_t lb(uint32_t row) { return row >> 8; }
    static __device__ __forceinline__ uint32_t col(uint32_t a, uint32_t b) { return 0x43004300u | a | (b << 16); }
    static __device__ __forceinline__ void cols(const uint8_t* ga, const uint8_t* gb, uint32_t (&cl)[PB_T]) {
        const uint4* sa = reinterpret_cast<const uint4*>(ga);
        const uint4* sb = reinterpret_cast<const uint4*>(gb);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const uint4 va = __ldg(sa + h), vb = __ldg(sb + h);
            const uint32_t xa[4] = {va.x, va.y, va.z, va.w}, xb[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint32_t lo = __byte_perm(xa[t], xb[t], 0x5140);   // a0 b0 a1 b1
                const uint32_t hi = __byte_perm(xa[t], xb[t], 0x7362);   // a2 b2 a3 b3
                cl[16 * h + 4 * t + 0] = __byte_perm(lo, 0x43u, 0x4140);
                cl[16 * h + 4 * t + 1] = __byte_perm(lo, 0x43u, 0x4342);
                cl[16 * h + 4 * t + 2] = __byte_perm(hi, 0x43u, 0x4140);
                cl[16 * h + 4 * t + 3] = __byte_perm(hi, 0x43u, 0x4342);
            }
        }
    }
};
template <> struct PairCodes<uint16_t> {
    using Row = uint32_t;
    static __device__ __forceinline__ Row pack(uint32_t la, uint32_t lb) { return la | (lb << 16); }
    static __device__ __forceinline__ uint32_t key(uint32_t row) { return row + 0x40004000u; }
    static __device__ __forceinline__ uint32_t la(uint32_t row) { return row & 0xFFFFu; }
    static __device__ __forceinline__ uint32_t lb(uint32_t row) { return row >> 16; }
    static __device__ __forceinline__ uint32_t col(uint32_t a, uint32_t b) { return 0x40004000u + (a | (b << 16)); }
    static __device__ __forceinline__ void cols(const uint16_t* ga, const uint16_t* gb, uint32_t (&cl)[PB_T]) {
        const uint4* sa = reinterpret_cast<const uint4*>(ga);
        const uint4* sb = reinterpret_cast<const uint4*>(gb);
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const uint4 va = __ldg(sa + h), vb = __ldg(sb + h);
            const uint32_t xa[4] = {va.x, va.y, va.z, va.w}, xb[4] = {vb.x, vb.y, vb.z, vb.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                cl[8 * h + 2 * t + 0] = __byte_perm(xa[t], xb[t], 0x5410) + 0x40004000u;   // a0 b0
                cl[8 * h + 2 * t + 1] = __byte_perm(xa[t], xb[t], 0x7632) + 0x40004000u;   // a1 b1
            }
        }
    }
};
template <typename L>
constexpr uint32_t pb2_smem_bytes() {
    return PB_D2_BYTES + PB_T * PB2_THREADS * (uint32_t)sizeof(typename PairCodes<L>::Row) + PB2_WTAB * 4;
}

// acc0 += d where the low FP16 halves of a and b are equal, acc1 += d where
// the high halves are.
__device__ __forceinline__ void pair_add(float& acc0, float& acc1, uint32_t a, uint32_t b, float d) {
    asm("{\n\t.reg .pred p, q;\n\tsetp.eq.f16x2 p|q, %2, %3;\n\t"
        "@p add.f32 %0, %0, %4;\n\t@q add.f32 %1, %1, %4;\n\t}"
        : "+f"(acc0), "+f"(acc1)
        : "r"(a), "r"(b), "f"(d));
}

template <typename L, bool VEC, int MINB>
__global__ void __launch_bounds__(PB2_THREADS, MINB)
k_sw_permblock_pair(const float* __restrict__ mat, uint32_t n, uint64_t ld,
                    const L* __restrict__ labels, uint64_t lstride, uint64_t P, const WeightMap wm,
                    uint32_t K, uint32_t n_pblocks, double* __restrict__ partials,
                    const DevStatus* __restrict__ st) {
    using C = PairCodes<L>;
    using Row = typename C::Row;
    constexpr uint32_t LAB_BYTES = PB_T * PB2_THREADS * (uint32_t)sizeof(Row);   // row codes of p and p'
    extern __shared__ __align__(16) uint8_t pb_smem[];
    float (*d2)[PB_T] = reinterpret_cast<float (*)[PB_T]>(pb_smem);
    Row (*lrow)[PB2_THREADS] = reinterpret_cast<Row (*)[PB2_THREADS]>(pb_smem + PB_D2_BYTES);
    const uint32_t band = blockIdx.x / n_pblocks;
    const uint32_t q = blockIdx.x % n_pblocks;
    const uint64_t pa = (uint64_t)q * PB2_ROWS + threadIdx.x, pb = pa + PB2_THREADS;
    const bool act_a = pa < P, act_b = pb < P;
    if (__syncthreads_or(st->code != DEV_OK)) {
        if (act_a) partials[(uint64_t)band * P + pa] = 0.0;
        if (act_b) partials[(uint64_t)band * P + pb] = 0.0;
        return;
    }
    // inactive label rows mirror the last row so every load stays in bounds
    const uint64_t ra = act_a ? pa : P - 1, rb = act_b ? pb : P - 1;
    const L* ga = labels + ra * lstride;
    const L* gb = labels + rb * lstride;
    // the weight sets of the CTA's label rows as an FP32 table in shared memory
    float* wtab = reinterpret_cast<float*>(pb_smem + PB_D2_BYTES + LAB_BYTES);
    const uint64_t p_first = (uint64_t)q * PB2_ROWS, p_last = min(P, p_first + PB2_ROWS) - 1;
    const uint64_t set_lo = wm.set_of(p_first);
    const uint64_t n_sets_cta = wm.set_of(p_last) - set_lo + 1;
    // (the launcher takes this kernel only when every CTA's sets fit the table)
    for (uint32_t e = threadIdx.x; e < n_sets_cta * K; e += PB2_THREADS)
        wtab[e] = (float)__ldg(wm.w + set_lo * K + e);
    // the two rows' weight sets as shared-memory addresses (one register each)
    const uint32_t wsa = (uint32_t)__cvta_generic_to_shared(wtab + (wm.set_of(ra) - set_lo) * K);
    const uint32_t wsb = (uint32_t)__cvta_generic_to_shared(wtab + (wm.set_of(rb) - set_lo) * K);
    const uint32_t r0 = band * PB_T;
    const uint32_t rows = min((uint32_t)PB_T, n - 1 - r0);  // row n-1 has no pairs
    for (uint32_t r = 0; r < rows; ++r) {
        const uint32_t la = min((uint32_t)ga[r0 + r], K - 1), lb = min((uint32_t)gb[r0 + r], K - 1);
        lrow[r][threadIdx.x] = C::pack(la, lb);
    }
    double tot_a = 0.0, tot_b = 0.0;

    for (uint32_t j0 = r0; j0 < n; j0 += PB_T) {
        __syncthreads();  // the previous tile has been consumed
#pragma unroll
        for (int e = threadIdx.x; e < PB_T * PB_T / 4; e += PB2_THREADS) {
            const int rr = e >> 4, cc = (e & 15) * 4;
            const uint32_t i = r0 + rr, j = j0 + cc;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (i < n) {
                const float* src = mat + (uint64_t)i * ld + j;
                if (VEC && j + 3 < n) {
                    v = __ldg(reinterpret_cast<const float4*>(src));
                } else {
                    if (j < n) v.x = __ldg(src);
                    if (j + 1 < n) v.y = __ldg(src + 1);
                    if (j + 2 < n) v.z = __ldg(src + 2);
                    if (j + 3 < n) v.w = __ldg(src + 3);
                }
            }
            v.x = (j > i && j < n) ? v.x * v.x : 0.f;
            v.y = (j + 1 > i && j + 1 < n) ? v.y * v.y : 0.f;
            v.z = (j + 2 > i && j + 2 < n) ? v.z * v.z : 0.f;
            v.w = (j + 3 > i && j + 3 < n) ? v.w * v.w : 0.f;
            *reinterpret_cast<float4*>(&d2[rr][cc]) = v;
        }
        // column labels of both rows as FP16 pairs (padding beyond n is label 0;
        // its d^2 is 0)
        uint32_t cl[PB_T];
        if (j0 + PB_T <= n) {
            C::cols(ga + j0, gb + j0, cl);
        } else {
#pragma unroll
            for (int c = 0; c < PB_T; ++c) {
                const uint32_t j = j0 + c;
                const uint32_t a = j < n ? ga[j] : 0u, b = j < n ? gb[j] : 0u;
                cl[c] = C::col(a, b);
            }
        }
        __syncthreads();

        for (uint32_t rg = 0; rg < rows; rg += PB_G) {
            const uint32_t rend = min(rg + PB_G, rows);
            float grp_a = 0.f, grp_b = 0.f;
#pragma unroll 2
            for (uint32_t r = rg; r < rend; ++r) {
                const uint32_t lab = lrow[r][threadIdx.x];
                const uint32_t key = C::key(lab);     // the FP16 patterns of la and lb
                const float4* drow = reinterpret_cast<const float4*>(&d2[r][0]);
                float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll
                for (int c4 = 0; c4 < PB_T / 4; ++c4) {
                    const float4 dv = drow[c4];
                    pair_add(a0, b0, cl[4 * c4 + 0], key, dv.x);
                    pair_add(a1, b1, cl[4 * c4 + 1], key, dv.y);
                    pair_add(a0, b0, cl[4 * c4 + 2], key, dv.z);
                    pair_add(a1, b1, cl[4 * c4 + 3], key, dv.w);
                }
                // each row segment weighted once (Algorithm 2)
                float w_a, w_b;
                asm("ld.shared.f32 %0, [%1];" : "=f"(w_a) : "r"(wsa + (C::la(lab) << 2)));
                asm("ld.shared.f32 %0, [%1];" : "=f"(w_b) : "r"(wsb + (C::lb(lab) << 2)));
                grp_a = fmaf(a0 + a1, w_a, grp_a);
                grp_b = fmaf(b0 + b1, w_b, grp_b);
            }
            tot_a += (double)grp_a;
            tot_b += (double)grp_b;
        }
    }
    if (act_a) partials[(uint64_t)band * P + pa] = tot_a;
    if (act_b) partials[(uint64_t)band * P + pb] = tot_b;
}

uint32_t permblock_bands(uint32_t n) { return (n - 1 + PB_T - 1) / PB_T; }

template <typename L>
static cudaError_t launch_pb_t(const SWProblem& pr, uint64_t lstride, double* partials,
                               const DevStatus* st, cudaStream_t s) {
    const bool vec = (pr.ld % 4 == 0) && ((uintptr_t)pr.mat % 16 == 0);
    const uint32_t n_bands = permblock_bands(pr.n);
    const uint64_t n_pblocks = (pr.P + PB_P - 1) / PB_P;
    const uint64_t blocks = (uint64_t)n_bands * n_pblocks;
    if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    const uint32_t smem = pb_smem_bytes<L>();
    cudaError_t e = cudaFuncSetAttribute(k_sw_permblock<L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sw_permblock<L, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (vec)
        k_sw_permblock<L, true><<<(unsigned)blocks, PB_P, smem, s>>>(
            pr.mat, pr.n, pr.ld, (const L*)pr.labels, lstride, pr.P, pr.weights(), pr.K,
            (uint32_t)n_pblocks, partials, st);
    else
        k_sw_permblock<L, false><<<(unsigned)blocks, PB_P, smem, s>>>(
            pr.mat, pr.n, pr.ld, (const L*)pr.labels, lstride, pr.P, pr.weights(), pr.K,
            (uint32_t)n_pblocks, partials, st);
    return launched(1);
}

// minb: CTAs per SM the register budget is sized for (3: 168 registers a
// thread, the default, measured 0.87-0.91 of the issue roofline at n = 20k;
// 4: 128 registers, more warps but spills, 0.81-0.86)
template <typename L, int MINB>
static cudaError_t launch_pb_pair(const SWProblem& pr, uint64_t lstride, double* partials,
                                  const DevStatus* st, cudaStream_t s) {
    const bool vec = (pr.ld % 4 == 0) && ((uintptr_t)pr.mat % 16 == 0);
    const uint32_t n_bands = permblock_bands(pr.n);
    const uint64_t n_pblocks = (pr.P + PB2_ROWS - 1) / PB2_ROWS;
    const uint64_t blocks = (uint64_t)n_bands * n_pblocks;
    if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    const uint32_t smem = pb2_smem_bytes<L>();
    cudaError_t e = cudaFuncSetAttribute(k_sw_permblock_pair<L, true, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sw_permblock_pair<L, false, MINB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (vec)
        k_sw_permblock_pair<L, true, MINB><<<(unsigned)blocks, PB2_THREADS, smem, s>>>(
            pr.mat, pr.n, pr.ld, (const L*)pr.labels, lstride, pr.P, pr.weights(), pr.K,
            (uint32_t)n_pblocks, partials, st);
    else
        k_sw_permblock_pair<L, false, MINB><<<(unsigned)blocks, PB2_THREADS, smem, s>>>(
            pr.mat, pr.n, pr.ld, (const L*)pr.labels, lstride, pr.P, pr.weights(), pr.K,
            (uint32_t)n_pblocks, partials, st);
    return launched(1);
}

// pr.labels must be uint8 (pr.label_type == LABEL_U8) or uint16 codes with a
// row stride of lstride elements, lstride * sizeof(code) a multiple of 16 and
// the base address 16-byte aligned.  variant 0: the paired FP16-compare
// kernel for codes whose weight sets fit its FP32 table (at most 2,048
// weights, so K <= 2,048 and the uint16 patterns 0x4000 + L stay normal FP16
// values), sized for 3 CTAs per SM, else the FP32 compare-and-set kernel;
// variant 2: the same paired kernel sized for 4 CTAs per SM; variant 1: the
// FP32 compare-and-set kernel.
cudaError_t launch_permblock_internal(const SWProblem& pr, uint64_t lstride, double* partials,
                                      const DevStatus* st, cudaStream_t s, int variant) {
    // weight sets a CTA of the paired kernel can meet: one, a run of equal
    // sets, or (ragged sets) at most all of them
    const WeightMap wm = pr.weights();
    const uint64_t sets = wm.row_start ? wm.n_sets
                          : wm.set_rows ? (PB2_ROWS + wm.set_rows - 1) / wm.set_rows + 1 : 1;
    const bool fits = sets * pr.K <= PB2_WTAB;
    if (pr.label_type == LABEL_U8) {
        if (fits && variant == 0) return launch_pb_pair<uint8_t, 3>(pr, lstride, partials, st, s);
        if (fits && variant == 2) return launch_pb_pair<uint8_t, 4>(pr, lstride, partials, st, s);
        return launch_pb_t<uint8_t>(pr, lstride, partials, st, s);
    }
    if (fits && variant == 0) return launch_pb_pair<uint16_t, 3>(pr, lstride, partials, st, s);
    if (fits && variant == 2) return launch_pb_pair<uint16_t, 4>(pr, lstride, partials, st, s);
    return launch_pb_t<uint16_t>(pr, lstride, partials, st, s);
}

}  // namespace pmn
