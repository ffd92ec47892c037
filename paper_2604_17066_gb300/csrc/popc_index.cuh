// popc_index.cuh -- component-major index of the upper reference set, used by
// the bit-packed classifiers (classify_popc.cu, batch.cu) in early-exit mode.
//
// The upper test of Algorithm 1 asks whether some upper reference r satisfies
// x >= r.  In thermometer bits (t_j = [x_i >= k], j = i(K-1) + k-1) a reference
// is ruled out by a sample exactly when the reference has a bit j set that the
// sample lacks.  Scanning reference by reference costs one word test per
// reference; when the first match lies thousands of references deep (samples
// whose likely paths are all cut near a hazard) that is the whole cost.  The
// index turns the scan around: for each chunk of 256 references and each
// thermometer bit j it stores the 256-bit set
//     B_j = { references r of the chunk with t_j(r) = 1 },
// so the references of the chunk that the sample rules out are the union of
// B_j over the sample's zero bits, and the sample matches some reference of
// the chunk iff that union is not the whole chunk.  The cost per chunk is one
// 256-bit OR per zero bit of the sample instead of 256 reference tests.
//
// Only one zero bit per component is needed: for a component with x_i = v <
// K-1 the zero bits are k = v+1..K-1, and B_{(i,k)} is contained in
// B_{(i,v+1)} (r_i >= k implies r_i >= v+1).  The lowest zero bit of each
// component is a zero bit that is a component's first bit or follows a one.
//
// Layout (uint32): [chunk c][row j < 32*WB][word q < 8]; bit b of word q is
// [reference 256c + 32q + b exists and has t_j = 1].  Rows j >= n(K-1) are 0.
// A chunk therefore holds 256*WB words, the size of 256 bit-packed references.
//
// Both tests below return exactly what the reference-by-reference scan returns
// for the same chunk (a match exists or not); which reference matches is not
// needed by the classification.
#pragma once

#include <stdint.h>

#include "rsr_internal.cuh"

namespace rsr {

constexpr int kIdxChunk = 256;               // references per index chunk
constexpr int kIdxWords = kIdxChunk / 32;    // 32-bit words of reference bits per row

// Bits of encoding word w that are thermometer bits (j < kenc).
__device__ __forceinline__ uint32_t enc_valid_bits(int kenc, int w) {
    const int lo = kenc - 32 * w;
    return lo >= 32 ? 0xffffffffu : (lo <= 0 ? 0u : ((1u << lo) - 1u));
}

// Reference bits of word q of a chunk holding cnt references that exist (1 = ruled out from the start).
__device__ __forceinline__ uint32_t idx_missing_refs(int cnt, int q) {
    const int v = cnt - 32 * q;
    return v >= 32 ? 0u : (v <= 0 ? 0xffffffffu : (0xffffffffu << v));
}

// The decisive zero bits of encoding word w: the lowest zero bit of every
// component below its top state.  first_w marks the bits of word w that start
// a component (all bits when K = 2); prev_w is word w-1 of t (ignored for w = 0,
// whose bit 0 starts a component).
__device__ __forceinline__ uint32_t decisive_zeros(uint32_t t_w, uint32_t prev_w, uint32_t first_w, int kenc,
                                                   int w) {
    const uint32_t z = ~t_w & enc_valid_bits(kenc, w);
    return z & (first_w | (t_w << 1) | (prev_w >> 31));
}

// One sample per lane: does some reference of the staged index chunk (cnt
// references, rows in s_idx) lie below the sample?  s_first[w] = component
// start bits of word w; s_zero = 8 zero words (16-byte aligned), read in place
// of a second row when a word has an odd number of decisive zeros.  Two rows
// per iteration, combined with three-input ORs.  *ops += the 32-bit logic
// operations on index data: 4 per row (8 words, two rows per three-input OR)
// and 8 per encoding word visited (the all-ruled-out test).
template <int WB>
__device__ __forceinline__ bool idx_match_lane(const uint32_t (&t)[WB], const uint32_t *__restrict__ s_idx,
                                               const uint32_t *__restrict__ s_first,
                                               const uint32_t *__restrict__ s_zero, int kenc, int cnt,
                                               unsigned long long *ops) {
    uint32_t bl[kIdxWords];
#pragma unroll
    for (int q = 0; q < kIdxWords; ++q) bl[q] = idx_missing_refs(cnt, q);
    uint32_t prev = 0u;
#pragma unroll
    for (int w = 0; w < WB; ++w) {
        if (32 * w >= kenc) break;
        uint32_t z = decisive_zeros(t[w], prev, s_first[w], kenc, w);
        prev = t[w];
        *ops += 8u + 4u * (unsigned)__popc(z);
        while (z) {
            const int b0 = __ffs(z) - 1;
            z &= z - 1u;
            const uint4 *r0 = reinterpret_cast<const uint4 *>(s_idx + (size_t)(w * 32 + b0) * kIdxWords);
            const uint4 *r1 = z ? reinterpret_cast<const uint4 *>(s_idx + (size_t)(w * 32 + __ffs(z) - 1) * kIdxWords)
                                : reinterpret_cast<const uint4 *>(s_zero);
            z &= z - 1u;
            const uint4 a0 = r0[0], c0 = r0[1], a1 = r1[0], c1 = r1[1];
            bl[0] |= a0.x | a1.x;
            bl[1] |= a0.y | a1.y;
            bl[2] |= a0.z | a1.z;
            bl[3] |= a0.w | a1.w;
            bl[4] |= c0.x | c1.x;
            bl[5] |= c0.y | c1.y;
            bl[6] |= c0.z | c1.z;
            bl[7] |= c0.w | c1.w;
        }
        // every reference of the chunk ruled out: no need to look further
        if ((bl[0] & bl[1] & bl[2] & bl[3] & bl[4] & bl[5] & bl[6] & bl[7]) == 0xffffffffu) return false;
    }
    return (bl[0] & bl[1] & bl[2] & bl[3] & bl[4] & bl[5] & bl[6] & bl[7]) != 0xffffffffu;
}

// One sample per warp, its encoding words read from shared memory (word w at
// col[w * stride], the same for every lane): lane = 8g + q takes the zero bits
// in byte g of every word and reference word q of the chunk; the four byte
// groups are OR-combined with two shuffles.  All lanes return the same answer.
// *ops += this lane's ORs of index words.
template <int WB, int stride>
__device__ __forceinline__ bool idx_match_warp(const uint32_t *col, const uint32_t *__restrict__ s_idx,
                                               const uint32_t *__restrict__ s_first, int kenc, int cnt,
                                               int lane, unsigned long long *ops) {
    const int q = lane & (kIdxWords - 1);
    const uint32_t gmask = 0xffu << (8 * (lane >> 3));
    uint32_t bl = idx_missing_refs(cnt, q);
    uint32_t prev = 0u;
#pragma unroll 1
    for (int w = 0; w < WB; ++w) {
        if (32 * w >= kenc) break;
        const uint32_t tw = col[w * stride];
        uint32_t z = decisive_zeros(tw, prev, s_first[w], kenc, w) & gmask;
        prev = tw;
        *ops += (unsigned)__popc(z);
        while (z) {
            const int b = __ffs(z) - 1;
            z &= z - 1u;
            bl |= s_idx[(size_t)(w * 32 + b) * kIdxWords + q];
        }
    }
    bl |= __shfl_xor_sync(0xffffffffu, bl, 8);
    bl |= __shfl_xor_sync(0xffffffffu, bl, 16);
    return __any_sync(0xffffffffu, bl != 0xffffffffu);
}

// ---- asynchronous chunk copies (cp.async, global -> shared) ------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stage one chunk into shared memory, without waiting: an index chunk (kenc
// rows of 8 words, from idx_src) or cnt bit-packed references of WB words
// (from rows_src), and the chunk's and_words words of skip rows (from and_src
// when not NULL: an index chunk's AND row, or a lower chunk's AND and guard
// rows; and_words <= nthreads).  Every address is 16-byte aligned: chunks start
// at multiples of 256 references in 256-byte aligned regions.  The caller
// waits with cp_async_wait_all() and a block barrier before reading.
template <int WB, int nthreads>
__device__ __forceinline__ void load_chunk_async(uint32_t *dst, bool idx_chunk, const uint32_t *idx_src, int kenc,
                                                 const uint32_t *and_src, int and_words, uint32_t *and_dst,
                                                 const uint32_t *rows_src, int cnt, int tid) {
    if (and_src && tid < and_words) cp_async4(and_dst + tid, and_src + tid);
    if (idx_chunk) {
        for (int i = tid; i < kenc * 2; i += nthreads) cp_async16(dst + 4 * i, idx_src + 4 * i);
    } else {
        const int nw = cnt * WB, n16 = nw >> 2;
        for (int i = tid; i < n16; i += nthreads) cp_async16(dst + 4 * i, rows_src + 4 * i);
        for (int i = 4 * n16 + tid; i < nw; i += nthreads) cp_async4(dst + i, rows_src + i);
    }
    cp_async_commit();
}

// Lower chunk skip (rows ag: the AND of the chunk's forbidden-bit rows, then
// the OR of their guard bits, all zero for no guard test): does the sample
// have a 1 at a bit every reference of the chunk forbids, or a 1 at every
// guard of the chunk?  Then it lies below none of them.
template <int WB>
__device__ __forceinline__ bool lower_chunk_ruled_out(const uint32_t (&t)[WB], const uint32_t *ag) {
    uint32_t hit = 0u, miss = 0u, any = 0u;
#pragma unroll
    for (int w = 0; w < WB; ++w) {
        hit |= t[w] & ag[w];
        miss |= ag[WB + w] & ~t[w];
        any |= ag[WB + w];
    }
    return hit != 0u || (any != 0u && miss == 0u);
}

// Does the sample (words t) lack a bit that every reference of the chunk has
// (chunk AND row a)?  Then it dominates none of them.
template <int WB>
__device__ __forceinline__ bool chunk_ruled_out(const uint32_t (&t)[WB], const uint32_t *a) {
    uint32_t acc = 0u;
#pragma unroll
    for (int w = 0; w < WB; ++w) acc |= a[w] & ~t[w];
    return acc != 0u;
}

// Component start bits of encoding word w for K-1 bits per component.
__device__ __forceinline__ uint32_t component_first_bits(int km1, int kenc, int w) {
    uint32_t m = 0u;
    if (km1 == 1) return 0xffffffffu;
    int j0 = 32 * w;
    int b = (j0 % km1 == 0) ? 0 : km1 - j0 % km1;
    for (; b < 32 && j0 + b < kenc; b += km1) m |= 1u << b;
    return m;
}

}  // namespace rsr
