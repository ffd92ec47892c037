// maintain.cu -- reference-set maintenance and order-preserving selection.
//
// * Non-dominance (Sec. 2.2, Eqs. (2)-(3)): a reference set keeps only states
//   that no other state of the set dominates.  On thermometer words t(r)
//   (bit (i,k) = [r_i >= k]) the tests are word-wise: r_j <= r_i iff
//   t(r_j) AND NOT t(r_i) = 0, and r_j = r_i iff the words are equal.  One
//   reference per thread against the set streamed through shared memory (the
//   same shape as the bit-packed classifier), a block leaving as soon as all
//   of its references are known to be dominated; a (bit count, hash) key per
//   row skips the pairs that cannot dominate.
// * Selection: the first `limit` indices i (ascending) with flags[i] == value,
//   in three launches (per-tile counts, one-block exclusive scan of the
//   counts, ballot-ranked scatter).  Stage 1 uses it to pick unclassified
//   samples as search starts and to compact reference rows in order.
#include <algorithm>

#include <cuda_runtime.h>

#include "rsr_internal.cuh"
#include "rsr_launch.h"

namespace rsr {

namespace {

constexpr int kNdThreads = 256;
constexpr int kSelTile = 4096;
constexpr int kSelThreads = 256;
constexpr int kScanThreads = 1024;

// Row key for the pair filter: the number of thermometer bits (the sum of the
// states) and a 32-bit hash of the words.
template <int WB>
__device__ __forceinline__ void row_key(const uint32_t *row, uint32_t *pop, uint32_t *hash) {
    uint32_t c = 0u, h = 0x811C9DC5u;
#pragma unroll
    for (int w = 0; w < WB; ++w) {
        c += __popc(row[w]);
        h = (h ^ row[w]) * 0x01000193u;
        h ^= h >> 15;
    }
    *pop = c;
    *hash = h;
}

// Clears keep[j] for the candidates j in [c0, c1) that a row i in this block's
// slice of [d0, d1) dominates, or equals with i < j (indices are global rows of
// enc; keep[] is set to 1 before the launch).  Blocks along y take consecutive
// slices of `slice` rows, so a few candidates against many rows still fill the
// machine; a candidate that another slice has already cleared is skipped.
// Pair filter, exact: a row that makes row j redundant has fewer thermometer
// bits (upper set: r_i <= r_j; lower set: r_i >= r_j, so more bits), or as many
// and then equals row j.  So rows with more (upper) or fewer (lower) bits are
// skipped, and rows with as many bits are tested only when their hashes agree.
// The keys of each staged chunk are computed once in shared memory.  (Upper
// references that are spanning trees of one graph all have the same number of
// bits: then only equal hashes reach the word test.)
template <int WB>
__global__ void __launch_bounds__(kNdThreads) nondominated_kernel(const uint32_t *__restrict__ enc, int64_t c0,
                                                                  int64_t c1, int64_t d0, int64_t d1, int64_t slice,
                                                                  int upper, uint8_t *keep) {
    __shared__ __align__(16) uint32_t s_ref[kNdThreads * WB];
    __shared__ uint32_t s_pop[kNdThreads], s_hash[kNdThreads];
    const int64_t j = c0 + (int64_t)blockIdx.x * kNdThreads + threadIdx.x;
    const int64_t e0 = d0 + (int64_t)blockIdx.y * slice;
    const int64_t e1 = (d1 - e0) < slice ? d1 : e0 + slice;
    uint32_t a[WB];
#pragma unroll
    for (int w = 0; w < WB; ++w) a[w] = (j < c1) ? enc[j * WB + w] : 0u;
    uint32_t pop_j, hash_j;
    row_key<WB>(a, &pop_j, &hash_j);
    // no reference in this slot, or already dominated (by another slice)
    bool done = !(j < c1) || *((volatile const uint8_t *)&keep[j]) == 0;
    bool dominated = false;     // found here
    for (int64_t base = e0; base < e1; base += kNdThreads) {
        if (__syncthreads_and(done)) break;
        const int cnt = (int)((e1 - base) < kNdThreads ? (e1 - base) : kNdThreads);
        for (int idx = threadIdx.x; idx < cnt * WB; idx += kNdThreads) s_ref[idx] = enc[base * WB + idx];
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            uint32_t row[WB];
#pragma unroll
            for (int w = 0; w < WB; ++w) row[w] = s_ref[threadIdx.x * WB + w];
            row_key<WB>(row, &s_pop[threadIdx.x], &s_hash[threadIdx.x]);
        }
        __syncthreads();
        if (!done) {
            for (int r = 0; r < cnt; ++r) {
                const int64_t i = base + r;
                if (i == j) continue;
                const uint32_t pi = s_pop[r];
                if (upper ? (pi > pop_j) : (pi < pop_j)) continue;
                if (pi == pop_j && s_hash[r] != hash_j) continue;
                uint32_t viol = 0u, diff = 0u;
#pragma unroll
                for (int w = 0; w < WB; ++w) {
                    const uint32_t b = s_ref[r * WB + w];
                    viol |= upper ? (b & ~a[w]) : (a[w] & ~b);
                    diff |= a[w] ^ b;
                }
                if (viol == 0u && (diff != 0u || i < j)) {
                    done = true;
                    dominated = true;
                    break;
                }
            }
        }
    }
    if (dominated) keep[j] = 0;
}

// *n_keep += the number of ones in keep[c0, c1).
__global__ void __launch_bounds__(kNdThreads) count_keep_kernel(const uint8_t *__restrict__ keep, int64_t c0,
                                                                int64_t c1, unsigned long long *n_keep) {
    unsigned c = 0u;
    for (int64_t i = c0 + (int64_t)blockIdx.x * kNdThreads + threadIdx.x; i < c1;
         i += (int64_t)gridDim.x * kNdThreads)
        c += keep[i];
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(n_keep, (unsigned long long)c);
}

// Candidates [c0, c1) against rows [d0, d1): keep[c0, c1) set to 1, then cleared
// for the dominated ones.  The rows are split into slices (multiples of the
// block's 256) so that the grid holds about kNdTargetBlocks blocks.
constexpr int64_t kNdTargetBlocks = 2048;

template <int WB>
cudaError_t launch_nd_wb(const uint32_t *enc, int64_t c0, int64_t c1, int64_t d0, int64_t d1, bool upper,
                         uint8_t *keep, cudaStream_t s) {
    const int64_t blocks = (c1 - c0 + kNdThreads - 1) / kNdThreads;
    if (blocks <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(keep + c0, 1, (size_t)(c1 - c0), s);
    if (e != cudaSuccess || d1 <= d0) return e;
    const int64_t chunks = (d1 - d0 + kNdThreads - 1) / kNdThreads;
    int64_t slices = std::max<int64_t>(1, std::min<int64_t>(chunks, kNdTargetBlocks / blocks));
    slices = std::min<int64_t>(slices, 65535);
    const int64_t slice = ((chunks + slices - 1) / slices) * kNdThreads;
    slices = (d1 - d0 + slice - 1) / slice;
    nondominated_kernel<WB><<<dim3((unsigned)blocks, (unsigned)slices), kNdThreads, 0, s>>>(
        enc, c0, c1, d0, d1, slice, upper ? 1 : 0, keep);
    return cudaGetLastError();
}

cudaError_t launch_count_keep(const uint8_t *keep, int64_t c0, int64_t c1, unsigned long long *n_keep,
                              cudaStream_t s) {
    if (c1 <= c0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((c1 - c0 + kNdThreads - 1) / kNdThreads, 1024);
    count_keep_kernel<<<(unsigned)blocks, kNdThreads, 0, s>>>(keep, c0, c1, n_keep);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kSelThreads) select_count_kernel(const uint8_t *__restrict__ flags, uint8_t value,
                                                                   int64_t N, int64_t *__restrict__ tile_cnt) {
    __shared__ int s_warp[kSelThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kSelTile;
    int c = 0;
    for (int i = threadIdx.x; i < kSelTile; i += kSelThreads) {
        const int64_t g = base + i;
        if (g < N && flags[g] == value) ++c;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kSelThreads / 32; ++w) t += s_warp[w];
        tile_cnt[blockIdx.x] = t;
    }
}

// One block: tile counts -> exclusive offsets, in place; *n_out = min(total, limit).
__global__ void __launch_bounds__(kScanThreads) select_scan_kernel(int64_t *tile_cnt, int64_t n_tiles, int64_t limit,
                                                                   int64_t *n_out) {
    __shared__ int64_t s[kScanThreads];
    int64_t carry = 0;
    for (int64_t base = 0; base < n_tiles; base += kScanThreads) {
        const int64_t g = base + threadIdx.x;
        const int64_t v = g < n_tiles ? tile_cnt[g] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int d = 1; d < kScanThreads; d <<= 1) {
            const int64_t add = threadIdx.x >= (unsigned)d ? s[threadIdx.x - d] : 0;
            __syncthreads();
            s[threadIdx.x] += add;
            __syncthreads();
        }
        if (g < n_tiles) tile_cnt[g] = carry + s[threadIdx.x] - v;
        carry += s[kScanThreads - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_out = carry < limit ? carry : limit;
}

__global__ void __launch_bounds__(kSelThreads) select_scatter_kernel(const uint8_t *__restrict__ flags, uint8_t value,
                                                                     int64_t N, const int64_t *__restrict__ tile_off,
                                                                     int64_t limit, int64_t *__restrict__ out_idx) {
    __shared__ int s_warp[kSelThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * kSelTile;
    int64_t off = tile_off[blockIdx.x];
    if (off >= limit) return;   // block-uniform
    for (int chunk = 0; chunk < kSelTile; chunk += kSelThreads) {
        const int64_t g = base + chunk + threadIdx.x;
        const bool f = g < N && flags[g] == value;
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (lane == 0) s_warp[warp] = __popc(m);
        __syncthreads();
        int before = 0, total = 0;
        for (int w = 0; w < kSelThreads / 32; ++w) {
            before += w < warp ? s_warp[w] : 0;
            total += s_warp[w];
        }
        if (f) {
            const int64_t pos = off + before + __popc(m & ((1u << lane) - 1u));
            if (pos < limit) out_idx[pos] = g;
        }
        off += total;
        __syncthreads();
    }
}

__global__ void gather_rows_kernel(const uint8_t *__restrict__ src, const int64_t *__restrict__ idx, int64_t count,
                                   int n, uint8_t *__restrict__ dst) {
    const int64_t total = count * n;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = g / n;
        const int i = (int)(g - k * n);
        dst[g] = src[idx[k] * n + i];
    }
}

}  // namespace

namespace {
cudaError_t launch_nd_range(const uint32_t *enc, int64_t c0, int64_t c1, int64_t d0, int64_t d1, int words_b,
                            bool upper, uint8_t *keep, cudaStream_t s) {
    switch (words_b) {
        case 1: return launch_nd_wb<1>(enc, c0, c1, d0, d1, upper, keep, s);
        case 2: return launch_nd_wb<2>(enc, c0, c1, d0, d1, upper, keep, s);
        case 4: return launch_nd_wb<4>(enc, c0, c1, d0, d1, upper, keep, s);
        case 6: return launch_nd_wb<6>(enc, c0, c1, d0, d1, upper, keep, s);
        case 8: return launch_nd_wb<8>(enc, c0, c1, d0, d1, upper, keep, s);
        case 10: return launch_nd_wb<10>(enc, c0, c1, d0, d1, upper, keep, s);
        case 12: return launch_nd_wb<12>(enc, c0, c1, d0, d1, upper, keep, s);
        case 16: return launch_nd_wb<16>(enc, c0, c1, d0, d1, upper, keep, s);
        case 24: return launch_nd_wb<24>(enc, c0, c1, d0, d1, upper, keep, s);
        case 32: return launch_nd_wb<32>(enc, c0, c1, d0, d1, upper, keep, s);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

cudaError_t launch_nondominated(const uint32_t *enc, int64_t R, int words_b, bool upper, uint8_t *keep,
                                unsigned long long *n_keep, cudaStream_t s) {
    if (R <= 0) return cudaSuccess;
    cudaError_t e = launch_nd_range(enc, 0, R, 0, R, words_b, upper, keep, s);
    if (e != cudaSuccess) return e;
    return launch_count_keep(keep, 0, R, n_keep, s);
}

// Rows [0, R_old) are already non-dominated among themselves (no row dominates
// another and none repeats), rows [R_old, R) are new.  An old row can then only
// be dominated by a new one (an equal new row comes later and does not count),
// and a new row by any row: the same keep mask as the full test, with
// 2 R_old (R - R_old) + (R - R_old)^2 row tests instead of R^2.
cudaError_t launch_nondominated_appended(const uint32_t *enc, int64_t R_old, int64_t R, int words_b, bool upper,
                                         uint8_t *keep, unsigned long long *n_keep, cudaStream_t s) {
    if (R <= 0) return cudaSuccess;
    cudaError_t e = launch_nd_range(enc, 0, R_old, R_old, R, words_b, upper, keep, s);
    if (e != cudaSuccess) return e;
    if ((e = launch_nd_range(enc, R_old, R, 0, R, words_b, upper, keep, s)) != cudaSuccess) return e;
    return launch_count_keep(keep, 0, R, n_keep, s);
}

size_t select_scratch_bytes(int64_t N) {
    const int64_t tiles = (N + kSelTile - 1) / kSelTile;
    return (size_t)(tiles + 1) * sizeof(int64_t);
}

cudaError_t launch_select(const uint8_t *flags, uint8_t value, int64_t N, int64_t limit, int64_t *out_idx,
                          int64_t *n_out, int64_t *scratch, cudaStream_t s) {
    if (N <= 0 || limit <= 0) return cudaMemsetAsync(n_out, 0, sizeof(int64_t), s);
    const int64_t tiles = (N + kSelTile - 1) / kSelTile;
    select_count_kernel<<<(unsigned)tiles, kSelThreads, 0, s>>>(flags, value, N, scratch);
    select_scan_kernel<<<1, kScanThreads, 0, s>>>(scratch, tiles, limit, n_out);
    select_scatter_kernel<<<(unsigned)tiles, kSelThreads, 0, s>>>(flags, value, N, scratch, limit, out_idx);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const uint8_t *src, const int64_t *idx, int64_t count, int n, uint8_t *dst,
                               cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int64_t total = count * n;
    int64_t blocks = (total + 255) / 256;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (blocks > cap) blocks = cap;
    gather_rows_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, idx, count, n, dst);
    return cudaGetLastError();
}

}  // namespace rsr
