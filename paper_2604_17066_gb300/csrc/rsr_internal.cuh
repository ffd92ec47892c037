// rsr_internal.cuh -- device helpers and workspace layout shared by the
// kernels of librsr (RSR hot path, arXiv 2604.17066, on sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rsr.h"

namespace rsr {

// ---------------------------------------------------------------------------
// Limits (documented in rsr.h).
// ---------------------------------------------------------------------------
constexpr int kMaxK = 16;
constexpr int kMaxKenc = 1024;                 // n*(K-1) thermometer bits
constexpr int kClassifyDefaultK0 = 2;          // first-pass chunk steps of the two-pass bit-packed path
constexpr int64_t kTwoPassMinN = int64_t(1) << 19;   // calls with fewer samples run one pass
constexpr int64_t kClassifyDeepCap = int64_t(1) << 22;   // deep-queue entries at most (32 MB)
constexpr int kMaxWords = kMaxKenc / 32;       // 32-bit words per encoded state
constexpr int kTcKPad = 32;                    // FP8 MMA K step (bytes)

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products
// on counter words 0 and 2, xor of the high halves into words 1 / 3 and the
// round key, word permutation, and a Weyl bump of the key between rounds.
// ---------------------------------------------------------------------------
struct U32x4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U32x4{c0, c1, c2, c3};
}

// Component state from one uniform word: x = #{k in 1..K-1 : u >= T_{i,k}}.
// Thresholds are 33-bit values (T <= 2^32) held in uint64.
__device__ __forceinline__ uint32_t state_from_uniform(uint32_t u, const unsigned long long *thr_row,
                                                       int km1) {
    uint32_t x = 0;
    for (int k = 0; k < km1; ++k) x += ((unsigned long long)u >= thr_row[k]) ? 1u : 0u;
    return x;
}

// Binary components (K = 2): x = [u >= T] with T <= 2^32.  The bit-packed
// classifiers keep T as 32 bits, T32 = min(T, 2^32 - 1), plus a "never" bit
// for T = 2^32 (the state 1 has probability 0): x = [u >= T32] AND NOT never,
// which equals [u >= T] for every u < 2^32.  Entries i >= n are "never", so
// padding bits stay 0.  Tables hold roundup(n, 8) thresholds and
// ceil(roundup(n, 8) / 32) never-words.
__device__ __forceinline__ void binary_tables_to_smem(const unsigned long long *__restrict__ thr, int n,
                                                      uint32_t *s_t32, uint32_t *s_never, int tid, int nthreads) {
    const int npad = (n + 7) & ~7;
    for (int i = tid; i < npad; i += nthreads) {
        const unsigned long long T = i < n ? thr[i] : (1ull << 32);
        s_t32[i] = T >= (1ull << 32) ? 0xffffffffu : (uint32_t)T;
    }
    for (int w = tid; 32 * w < npad; w += nthreads) {
        uint32_t m = 0u;
        for (int b = 0; b < 32; ++b) {
            const int i = 32 * w + b;
            if (i >= n || thr[i] >= (1ull << 32)) m |= 1u << b;
        }
        s_never[w] = m;
    }
}

// Philox-sample a binary state straight into its thermometer words (bit i =
// x_i), eight components per step, and write the words to col[w * stride];
// words up to WB - 1 beyond the state are zeroed.  Same draws as
// state_from_uniform(): u_i = word (i mod 4) of Philox(h, i / 4).
template <int WB, int stride>
__device__ __forceinline__ void sample_binary_words(uint64_t h, uint32_t key0, uint32_t key1, int n,
                                                    const uint32_t *s_t32, const uint32_t *s_never,
                                                    uint32_t *col) {
    const uint32_t h0 = (uint32_t)h, h1 = (uint32_t)(h >> 32);
    const uint4 *t4 = reinterpret_cast<const uint4 *>(s_t32);
    uint32_t word = 0u;
    int w = 0;
    for (int q = 0; 4 * q < n; q += 2) {
        const U32x4 ra = philox4x32_10(h0, h1, (uint32_t)q, 0u, key0, key1);
        const U32x4 rb = philox4x32_10(h0, h1, (uint32_t)(q + 1), 0u, key0, key1);
        const uint4 ta = t4[q], tb = t4[q + 1];
        const uint32_t byte = (ra.x >= ta.x ? 1u : 0u) | (ra.y >= ta.y ? 2u : 0u) | (ra.z >= ta.z ? 4u : 0u) |
                              (ra.w >= ta.w ? 8u : 0u) | (rb.x >= tb.x ? 16u : 0u) | (rb.y >= tb.y ? 32u : 0u) |
                              (rb.z >= tb.z ? 64u : 0u) | (rb.w >= tb.w ? 128u : 0u);
        const int i0 = 4 * q;  // a multiple of 8: the byte never straddles two words
        word |= byte << (i0 & 31);
        if (((i0 + 8) & 31) == 0 || i0 + 8 >= n) {
            w = i0 >> 5;
            col[w * stride] = word & ~s_never[w];
            ++w;
            word = 0u;
        }
    }
    for (; w < WB; ++w) col[w * stride] = 0u;
}

// Multi-state components (K > 2): thermometer bit j = i(K-1) + k-1 is
// [u_i >= T_{i,k}], T <= 2^32.  As for binary states, each threshold is kept
// as 32 bits, T32 = min(T, 2^32 - 1), with a never bit for T = 2^32 (the bit
// is then 0 for every u < 2^32).  Thresholds do not decrease in k, so a
// component's never bits are its top bits and its bits stay a thermometer.
// Layout: s_t32k[k * npad + i] with npad = roundup(n, 8), so that one level's
// thresholds of four consecutive components load as one 16-byte word; the
// never-words (one bit per thermometer bit, ceil(n(K-1)/32) words) follow at
// s_t32k + (K-1) * npad.  Needs (K-1) * npad + ceil(n(K-1)/32) words.
__device__ __forceinline__ void multi_tables_to_smem(const unsigned long long *__restrict__ thr, int n, int km1,
                                                     uint32_t *s_t32k, int tid, int nthreads) {
    const int npad = (n + 7) & ~7, kenc = n * km1;
    for (int e = tid; e < km1 * npad; e += nthreads) {
        const int k = e / npad, i = e - k * npad;
        const unsigned long long T = i < n ? thr[(size_t)i * km1 + k] : (1ull << 32);
        s_t32k[e] = T >= (1ull << 32) ? 0xffffffffu : (uint32_t)T;
    }
    uint32_t *s_never = s_t32k + km1 * npad;
    for (int w = tid; 32 * w < kenc; w += nthreads) {
        uint32_t m = 0u;
        for (int b = 0; b < 32 && 32 * w + b < kenc; ++b)
            if (thr[32 * w + b] >= (1ull << 32)) m |= 1u << b;
        s_never[w] = m;
    }
}

// Philox-sample a multi-state state straight into its thermometer words, four
// components (one Philox block) per step (x_i = #{k : u_i >= T32_{i,k}}, then
// x_i ones at bits i(K-1) ..), never bits cleared as each word is written to
// col[w * stride]; words up to WB - 1 beyond the state are zeroed.  Same draws
// and words as state_from_uniform() with thresholds held in 64 bits.  (One
// block per step, not two as for binary states: the level compares give the
// step its parallelism, and the kernels that inline this stay within their
// register budget.)
// KM1 > 0: the level count K-1 is a compile-time constant (level loop
// unrolled); KM1 = 0: it is km1_rt.
template <int WB, int stride, int KM1>
__device__ __forceinline__ void sample_multi_words_k(uint64_t h, uint32_t key0, uint32_t key1, int n, int km1_rt,
                                                     const uint32_t *s_t32k, uint32_t *col) {
    const int km1 = KM1 > 0 ? KM1 : km1_rt;
    const int npad = (n + 7) & ~7;
    const uint32_t *s_never = s_t32k + km1 * npad;
    const uint32_t h0 = (uint32_t)h, h1 = (uint32_t)(h >> 32);
    uint32_t cur = 0u;
    int pos = 0, w = 0;
    for (int q = 0; 4 * q < n; ++q) {
        const U32x4 r = philox4x32_10(h0, h1, (uint32_t)q, 0u, key0, key1);
        uint32_t x0 = 0u, x1 = 0u, x2 = 0u, x3 = 0u;
#pragma unroll
        for (int k = 0; k < km1; ++k) {
            const uint4 t = *reinterpret_cast<const uint4 *>(s_t32k + k * npad + 4 * q);
            x0 += r.x >= t.x ? 1u : 0u;
            x1 += r.y >= t.y ? 1u : 0u;
            x2 += r.z >= t.z ? 1u : 0u;
            x3 += r.w >= t.w ? 1u : 0u;
        }
        const uint32_t xs[4] = {x0, x1, x2, x3};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (4 * q + c >= n) break;
            const uint32_t bits = (1u << xs[c]) - 1u;   // x <= K-1 <= 15
            cur |= bits << pos;
            const int np = pos + km1;
            if (np >= 32) {
                col[w * stride] = cur & ~s_never[w];
                ++w;
                cur = (np > 32) ? (bits >> (32 - pos)) : 0u;
                pos = np - 32;
            } else {
                pos = np;
            }
        }
    }
    if (pos > 0) {
        col[w * stride] = cur & ~s_never[w];
        ++w;
    }
    for (; w < WB; ++w) col[w * stride] = 0u;
}

// K = 3 and K = 4 (two or three levels per component) with the level loop
// unrolled; other K with it at run time.
template <int WB, int stride>
__device__ __forceinline__ void sample_multi_words(uint64_t h, uint32_t key0, uint32_t key1, int n, int km1,
                                                   const uint32_t *s_t32k, uint32_t *col) {
    if (km1 == 3) sample_multi_words_k<WB, stride, 3>(h, key0, key1, n, km1, s_t32k, col);
    else if (km1 == 2) sample_multi_words_k<WB, stride, 2>(h, key0, key1, n, km1, s_t32k, col);
    else sample_multi_words_k<WB, stride, 0>(h, key0, key1, n, km1, s_t32k, col);
}

// ---------------------------------------------------------------------------
// Visiting order of the two reference sets, in chunks (tiles) of references.
// Without an overlapping pair (no upper reference below a lower one) a sample
// matches at most one set and any match is final, so the sets alternate chunk
// by chunk, upper first, until one runs out: a sample that belongs to either
// set meets its set within the first chunks.  With an overlapping pair every
// lower chunk comes first (Algorithm 1: lower takes precedence).
// step in [0, nU + nL) -> (*upper, *idx = chunk index within that set).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ void chunk_at(int64_t step, int64_t nU, int64_t nL, bool overlap, bool *upper,
                                                  int64_t *idx) {
    if (overlap) {
        *upper = step >= nL;
        *idx = *upper ? step - nL : step;
        return;
    }
    const int64_t m = nU < nL ? nU : nL;
    if (step < 2 * m) {
        *upper = (step & 1) == 0;
        *idx = step >> 1;
        return;
    }
    *upper = nU > nL;
    *idx = m + (step - 2 * m);
}

// The bit-packed classifiers' order, visited step by step (the same on every
// thread of a block).  Without an overlapping pair: upper chunk 0, lower chunk
// 0, then bursts of upper chunks that double in length between lower chunks
// (U0 L0 U1 L1 U2 U3 L2 U4..U7 L3 U8..U15 L4 ...), each set continuing alone
// once the other runs out.  With the upper index an upper chunk costs a small
// fraction of a lower chunk scanned reference by reference, and lower matches
// sit in the first chunks (the references are ordered by probability), so a
// sample whose first upper match lies k chunks deep meets about log2(k) lower
// chunks instead of k.  Without the index (grow = false) the bursts stay at one
// chunk: strict alternation, as chunk_at().  With an overlapping pair: every
// lower chunk first.
struct ChunkWalk {
    int64_t nU, nL;
    int32_t u = 0, l = 0, burst = 1;   // chunk counts stay far below 2^31
    bool overlap, grow;
    __host__ __device__ ChunkWalk(int64_t nU_, int64_t nL_, bool ov, bool grow_)
        : nU(nU_), nL(nL_), overlap(ov), grow(grow_) {}
    // next chunk: *upper and *idx; call at most nU + nL times
    __host__ __device__ __forceinline__ void next(bool *upper, int64_t *idx) {
        bool up;
        if (overlap) up = l >= nL;
        else if (u >= nU) up = false;
        else if (l >= nL) up = true;
        else up = burst > 0;
        if (up) {
            *upper = true;
            *idx = u++;
            --burst;
        } else {
            *upper = false;
            *idx = l++;
            burst = !grow ? 1 : (l >= 31 ? 0x7fffffff : (1 << (l - 1)));
        }
    }
};

// ---------------------------------------------------------------------------
// Workspace layout.  The caller passes one 256-byte aligned buffer; offsets
// below are derived from the problem sizes only (rsr_workspace_size()).
// ---------------------------------------------------------------------------
struct WsHeader {
    int32_t overlap;   // 1 if some upper reference lies below some lower reference
    int32_t error;     // device error code (0 = none); kept until rsr_prepare / rsr_update_pmf
    int32_t grad_bad;  // rsr_grad: a listed index lies outside [0, N) (cleared by each call)
    int32_t pad;
    unsigned long long tune_counts[3];  // rsr_autotune: counts of its timing runs
    uint32_t reserved[54];
};
static_assert(sizeof(WsHeader) == 256, "header is one 256-byte line");

struct WsLayout {
    int32_t n = 0, K = 0, kenc = 0, words = 0;
    int64_t R_L = 0, R_U = 0;
    int32_t tc_kpad = 0;        // FP8 row length in bytes (multiple of 32, with slack for the bias)
    int64_t tc_rows_L = 0;      // references padded to the tensor-core tile
    int64_t tc_rows_U = 0;
    size_t off_thr = 0;         // uint64 [n*(K-1)]
    size_t off_popc_L = 0;      // uint32 [R_L][words]  (complement of the reference thermometer)
    size_t off_popc_U = 0;      // uint32 [R_U][words]  (reference thermometer)
    size_t off_tc_L = 0;        // FP8 tiles of the lower references
    size_t off_tc_U = 0;        // FP8 tiles of the upper references
    size_t off_table = 0;       // float [2][n*K]: per-state log-probability tables (reference ordering)
    size_t off_score = 0;       // float [max(R_L, R_U)]: reference scores (ordering)
    size_t off_perm = 0;        // int32 [max(R_L, R_U)]: reference order (ordering)
    size_t off_popc_UT = 0;     // uint32 [ceil(R_U/256)][32*words][8]: component-major index of the upper set
    size_t off_popc_UA = 0;     // uint32 [ceil(R_U/256)][words]: per index chunk, the AND of its references
    size_t off_popc_LG = 0;     // uint32 [ceil(R_L/256)][2][words]: per lower chunk, AND row and guard row
    size_t total = 0;
};

constexpr int kTcRefTile = 128;  // rows per encoded reference tile (the MMA's B is 128 or 256 rows)
constexpr int kTcRowPad = 256;   // encoded reference rows are padded to this multiple

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline WsLayout make_layout(int32_t n, int32_t K, int64_t R_L, int64_t R_U, int32_t words_b) {
    WsLayout L;
    L.n = n;
    L.K = K;
    L.kenc = n * (K - 1);
    L.words = words_b;  // 32-bit words per encoded state, rounded up to a kernel bucket
    L.R_L = R_L;
    L.R_U = R_U;
    // FP8 row: kenc 0/1 bytes, then a constant-one column block that carries the
    // survival bias (see classify_tc.cu); rounded up to the 32-byte MMA K step.
    const int bias_cols = (L.kenc + 15) / 16;
    L.tc_kpad = ((L.kenc + bias_cols + kTcKPad - 1) / kTcKPad) * kTcKPad;
    L.tc_rows_L = ((R_L + kTcRowPad - 1) / kTcRowPad) * kTcRowPad;
    L.tc_rows_U = ((R_U + kTcRowPad - 1) / kTcRowPad) * kTcRowPad;
    size_t off = align256(sizeof(WsHeader));
    L.off_thr = off;
    off = align256(off + sizeof(unsigned long long) * (size_t)n * (K - 1));
    L.off_popc_L = off;
    off = align256(off + sizeof(uint32_t) * (size_t)R_L * L.words);
    L.off_popc_U = off;
    off = align256(off + sizeof(uint32_t) * (size_t)R_U * L.words);
    L.off_tc_L = off;
    off = align256(off + (size_t)L.tc_rows_L * L.tc_kpad);
    L.off_tc_U = off;
    off = align256(off + (size_t)L.tc_rows_U * L.tc_kpad);
    const size_t rmax = (size_t)(R_L > R_U ? R_L : R_U) + 1;
    L.off_table = off;
    off = align256(off + sizeof(float) * 2 * (size_t)n * K);
    L.off_score = off;
    off = align256(off + sizeof(float) * rmax);
    L.off_perm = off;
    off = align256(off + sizeof(int32_t) * rmax);
    // placed last so that the offsets of the regions above do not depend on it
    L.off_popc_UT = off;
    off = align256(off + sizeof(uint32_t) * (size_t)((R_U + 255) / 256) * 256 * L.words);
    L.off_popc_UA = off;
    off = align256(off + sizeof(uint32_t) * (size_t)((R_U + 255) / 256) * L.words);
    L.off_popc_LG = off;
    off = align256(off + sizeof(uint32_t) * (size_t)((R_L + 255) / 256) * 2 * L.words);
    L.total = off;
    return L;
}

// Parameters of one classification launch (both paths).
struct ClassifyParams {
    int32_t n, K, km1, kenc, words;
    int64_t N;
    uint64_t seed, offset;
    const uint8_t *samples;            // NULL = Philox
    const unsigned long long *thr;     // [n*(K-1)]
    const uint32_t *popc_L, *popc_U;   // bit-packed references
    const uint32_t *popc_UT;           // component-major index of the upper set, or NULL (no index)
    const uint32_t *popc_UA;           // per index chunk: AND of its references (with popc_UT)
    const uint32_t *popc_LG;           // per lower chunk: AND row and guard row ([2][words]), or NULL
    const uint8_t *tc_L, *tc_U;        // FP8 reference tiles
    int64_t R_L, R_U;
    int32_t tc_kpad;
    uint8_t *labels;
    unsigned long long *counts3;
    unsigned long long *grad_counts;   // [n*K] or NULL
    unsigned long long *exec_tests;    // [1] or NULL
    WsHeader *hdr;
    int32_t dense;
    int32_t test_stall;                // RSR_FLAG_TEST_STALL: the producer never starts
    // bit-packed early-exit mode, staged passes (NULL / 0: one pass)
    int64_t *deep;                     // [2][deep_cap]: two queues of the indices of deferred samples
    unsigned long long *deep_count;    // [2]: entries appended to each queue (may exceed deep_cap)
    int64_t deep_cap;                  // entries per queue
    int32_t k0;                        // chunk steps of the first pass (0: one pass)
    int64_t two_pass_min_n;            // fewer samples: one pass (kTwoPassMinN; 1 under RSR_FLAG_TEST_TWO_PASS)
    // set by the launcher for each pass
    int32_t q_in, q_out;               // queue read (-1: the call's tiles) and written (-1: none)
    int64_t step_lo, step_hi;          // the chunk steps this pass walks: [step_lo, step_hi)
};

// Stages of the staged bit-packed path: the first walks chunk steps [0, k0), each
// later one kDeferGrowth times as far as the step it starts at, the last to the
// end; a stage that would end past half of the steps walks to the end instead
// (no short last stage).
constexpr int kDeferGrowth = 4;
__host__ __device__ inline int64_t next_stage_end(int64_t hi, int64_t nsteps) {
    const int64_t next = hi * kDeferGrowth;
    return 2 * next > nsteps ? nsteps : next;
}
__host__ __device__ inline int staged_passes(int64_t nsteps, int64_t k0) {
    if (k0 <= 0 || k0 >= nsteps) return 1;
    int passes = 1;
    for (int64_t hi = k0; hi < nsteps; hi = next_stage_end(hi, nsteps)) ++passes;
    return passes;
}

}  // namespace rsr
