// prep_kernels.cu -- reference encoding, the precedence pre-check, sample
// materialisation and the gradient correction pass.
#include <algorithm>

#include <cuda_runtime.h>

#include "rsr_internal.cuh"
#include "rsr_launch.h"

namespace rsr {

namespace {

constexpr int kMaxCorrHist = 2048;  // n*K <= n + n(K-1) <= 2 * 1024 (K >= 2)

// Thermometer word w of reference r: bit j = i*(K-1) + (k-1) is [r_i >= k];
// lower references are stored complemented (within the n*(K-1) valid bits) so
// that the classifier's failure test is t(x) AND stored == 0 (Sec. 3.3: the
// subset test H . Rbar = 0).
__global__ void encode_popc_kernel(const uint8_t *__restrict__ refs, const int32_t *__restrict__ perm, int64_t R,
                                   int n, int km1, int words_b, int complement, uint32_t *__restrict__ out) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= R * words_b) return;
    const int64_t slot = gid / words_b;
    const int64_t r = perm ? (int64_t)perm[slot] : slot;  // reference stored in this slot
    const int w = (int)(gid % words_b);
    const int kenc = n * km1;
    uint32_t word = 0;
    for (int b = 0; b < 32; ++b) {
        const int j = w * 32 + b;
        if (j >= kenc) break;
        const int i = j / km1;
        const int k = j % km1 + 1;
        const uint32_t a = refs[r * n + i] >= k ? 1u : 0u;
        word |= (complement ? (a ^ 1u) : a) << b;
    }
    out[gid] = word;
}

// Component-major index of the upper set (layout in popc_index.cuh): word q of
// row j of chunk c has bit b = t_j of the reference in slot 256c + 32q + b, 0
// past R_U and for rows j >= kenc.  Slot r holds bit-packed row perm[r] (the
// clustered order; identity without perm).  One warp per (chunk, word q,
// encoding word jw): lane b loads word jw of slot 256c + 32q + b, and 32
// ballots transpose the 32 x 32 bit block into rows 32jw .. 32jw + 31.
__global__ void encode_index_kernel(const uint32_t *__restrict__ popc_U, const int32_t *__restrict__ perm,
                                    int64_t R_U, int words_b, int kenc, int64_t nwarps, uint32_t *__restrict__ out) {
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= nwarps) return;   // whole warps: nwarps * 32 threads, blocks of 256
    const int jw = (int)(wid % words_b);
    const int q = (int)((wid / words_b) % 8);
    const int64_t c = wid / ((int64_t)words_b * 8);
    const int64_t slot = c * 256 + 32 * q + lane;
    uint32_t v = 0u;
    if (slot < R_U) v = popc_U[(perm ? (int64_t)perm[slot] : slot) * words_b + jw];
    for (int jb = 0; jb < 32; ++jb) {
        const uint32_t m = __ballot_sync(0xffffffffu, (v >> jb) & 1u);
        if (lane == jb) {
            const int j = 32 * jw + jb;
            out[((size_t)c * 32 * words_b + j) * 8 + q] = j < kenc ? m : 0u;
        }
    }
}

// Per index chunk, the AND of its references' bit-packed rows: the bits every
// reference of the chunk has.  A sample lacking one of them dominates no
// reference of the chunk.  One warp per (chunk, word), eight slots per lane.
__global__ void chunk_and_kernel(const uint32_t *__restrict__ popc_U, const int32_t *__restrict__ perm, int64_t R_U,
                                 int words_b, int64_t nwarps, uint32_t *__restrict__ out) {
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= nwarps) return;
    const int w = (int)(wid % words_b);
    const int64_t c = wid / words_b;
    uint32_t a = 0xffffffffu;
    for (int k = 0; k < 8; ++k) {
        const int64_t slot = c * 256 + 32 * k + lane;
        if (slot < R_U) a &= popc_U[(perm ? (int64_t)perm[slot] : slot) * words_b + w];
    }
    a = __reduce_and_sync(0xffffffffu, a);
    if (lane == 0) out[wid] = a;
}

// Clustering key of each upper reference: its bits at up to 32 chosen
// thermometer positions (most significant first).
__global__ void cluster_keys_kernel(const uint32_t *__restrict__ popc_U, int64_t R_U, int words_b, KeyBits kb,
                                    uint32_t *__restrict__ keys) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R_U) return;
    uint32_t k = 0;
    for (int b = 0; b < kb.nbits; ++b) {
        const int j = kb.pos[b];
        k |= ((popc_U[r * words_b + (j >> 5)] >> (j & 31)) & 1u) << (31 - b);
    }
    keys[r] = k;
}

// Overlap pre-check: some upper reference r^U <= some lower reference r^L iff
// OR_w (t_w(r^U) AND NOT t_w(r^L)) == 0 for that pair.  One upper reference
// per thread against lower references streamed through shared memory.
template <int WB>
__global__ void __launch_bounds__(256) overlap_kernel(const uint32_t *__restrict__ popc_L, int64_t R_L,
                                                      const uint32_t *__restrict__ popc_U, int64_t R_U,
                                                      WsHeader *hdr) {
    __shared__ __align__(16) uint32_t s_ref[256 * WB];
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t a[WB];
#pragma unroll
    for (int w = 0; w < WB; ++w) a[w] = (u < R_U) ? popc_U[u * WB + w] : 0xffffffffu;
    bool found = false;
    for (int64_t base = 0; base < R_L; base += 256) {
        const int cnt = (int)((R_L - base) < 256 ? (R_L - base) : 256);
        __syncthreads();
        for (int idx = threadIdx.x; idx < cnt * WB; idx += blockDim.x) s_ref[idx] = popc_L[base * WB + idx];
        __syncthreads();
        if (u < R_U && !found) {
            for (int r = 0; r < cnt; ++r) {
                uint32_t acc = 0;
#pragma unroll
                for (int w = 0; w < WB; ++w) acc |= a[w] & s_ref[r * WB + w];
                if (acc == 0u) {
                    found = true;
                    break;
                }
            }
        }
        if (__syncthreads_or(found)) break;
    }
    if (found && u < R_U) atomicOr(&hdr->overlap, 1);
}

template <int WB>
cudaError_t launch_overlap_wb(const uint32_t *popc_L, int64_t R_L, const uint32_t *popc_U, int64_t R_U,
                              WsHeader *hdr, cudaStream_t s) {
    const int64_t grid = (R_U + 255) / 256;
    overlap_kernel<WB><<<(unsigned)grid, 256, 0, s>>>(popc_L, R_L, popc_U, R_U, hdr);
    return cudaGetLastError();
}

// Reference score for ordering: sum over components of a per-(component,
// state) table (log P(X_i <= v) for lower references, log P(X_i >= v) for
// upper ones), i.e. the log-probability of the reference's dominated region.
__global__ void score_refs_kernel(const uint8_t *__restrict__ refs, int64_t R, int n, int K,
                                  const float *__restrict__ table, float *__restrict__ score) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    float acc = 0.0f;
    for (int i = 0; i < n; ++i) acc += table[i * K + refs[r * n + i]];
    score[r] = acc;
}

// Materialised samples: thread per sample, same Philox layout and thresholds
// as the classifiers.
__global__ void sample_kernel(const ClassifyParams p, uint8_t *__restrict__ states) {
    const int64_t hl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (hl >= p.N) return;
    const uint64_t h = p.offset + (uint64_t)hl;
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    uint8_t *row = states + hl * (int64_t)p.n;
    for (int q = 0; 4 * q < p.n; ++q) {
        const U32x4 r = philox4x32_10((uint32_t)h, (uint32_t)(h >> 32), (uint32_t)q, 0u, key0, key1);
        const uint32_t us[4] = {r.x, r.y, r.z, r.w};
        for (int c = 0; c < 4 && 4 * q + c < p.n; ++c) {
            const int i = 4 * q + c;
            row[i] = (uint8_t)state_from_uniform(us[c], p.thr + (size_t)i * p.km1, p.km1);
        }
    }
}

// Gradient correction: unclassified samples that Phi resolved to S <= m' join
// the failure set; their states are regenerated from Philox and counted.
// First pass: every listed index is checked, and one outside [0, N) sets the
// call's flag; the counting pass then changes nothing.
__global__ void grad_index_check_kernel(const int64_t *__restrict__ idx, int64_t m, int64_t N, int32_t *bad) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t hl = idx[j];
        if (hl < 0 || hl >= N) *bad = 1;
    }
}

__global__ void __launch_bounds__(256) grad_correction_kernel(const ClassifyParams p, const int64_t *__restrict__ idx,
                                                               int64_t m) {
    if (*((volatile const int32_t *)&p.hdr->grad_bad) != 0) return;   // rejected by the check pass
    // one warp per listed sample, lanes over its components (one Philox block each);
    // per-(component, state) counts gathered in shared memory, flushed once per block
    __shared__ unsigned int s_hist[kMaxCorrHist];
    const int nk = p.n * p.K;
    for (int i = threadIdx.x; i < nk; i += blockDim.x) s_hist[i] = 0u;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    for (int64_t j = (int64_t)blockIdx.x * nwarps + warp; j < m; j += (int64_t)gridDim.x * nwarps) {
        const int64_t hl = idx[j];   // in [0, N): checked by the first pass
        const uint64_t h = p.offset + (uint64_t)hl;
        for (int q = lane; 4 * q < p.n; q += 32) {
            const U32x4 r = philox4x32_10((uint32_t)h, (uint32_t)(h >> 32), (uint32_t)q, 0u, key0, key1);
            const uint32_t us[4] = {r.x, r.y, r.z, r.w};
            for (int c = 0; c < 4 && 4 * q + c < p.n; ++c) {
                const int i = 4 * q + c;
                const uint32_t x = state_from_uniform(us[c], p.thr + (size_t)i * p.km1, p.km1);
                atomicAdd(&s_hist[i * p.K + (int)x], 1u);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nk; i += blockDim.x)
        if (s_hist[i]) atomicAdd(&p.grad_counts[i], (unsigned long long)s_hist[i]);
}

}  // namespace

cudaError_t launch_encode_popc(const uint8_t *refs, int64_t R, int n, int km1, int words_b, bool complement,
                               uint32_t *out, cudaStream_t s, const int32_t *perm) {
    const int64_t total = R * words_b;
    if (total <= 0) return cudaSuccess;
    encode_popc_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(refs, perm, R, n, km1, words_b,
                                                                        complement ? 1 : 0, out);
    return cudaGetLastError();
}

cudaError_t launch_score_refs(const uint8_t *refs, int64_t R, int n, int K, const float *table, float *score,
                              cudaStream_t s) {
    if (R <= 0) return cudaSuccess;
    score_refs_kernel<<<(unsigned)((R + 255) / 256), 256, 0, s>>>(refs, R, n, K, table, score);
    return cudaGetLastError();
}

cudaError_t launch_encode_index(const uint32_t *popc_U, const int32_t *perm, int64_t R_U, int words_b, int kenc,
                                uint32_t *out_index, uint32_t *out_and, cudaStream_t s) {
    if (R_U <= 0) return cudaSuccess;
    const int64_t nchunks = (R_U + 255) / 256;
    const int64_t nw_idx = nchunks * 8 * words_b, nw_and = nchunks * words_b;   // warps
    encode_index_kernel<<<(unsigned)((nw_idx + 7) / 8), 256, 0, s>>>(popc_U, perm, R_U, words_b, kenc, nw_idx,
                                                                     out_index);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    chunk_and_kernel<<<(unsigned)((nw_and + 7) / 8), 256, 0, s>>>(popc_U, perm, R_U, words_b, nw_and, out_and);
    return cudaGetLastError();
}

cudaError_t launch_cluster_keys(const uint32_t *popc_U, int64_t R_U, int words_b, const KeyBits &kb, uint32_t *keys,
                                cudaStream_t s) {
    if (R_U <= 0) return cudaSuccess;
    cluster_keys_kernel<<<(unsigned)((R_U + 255) / 256), 256, 0, s>>>(popc_U, R_U, words_b, kb, keys);
    return cudaGetLastError();
}

cudaError_t launch_overlap(const uint32_t *popc_L, int64_t R_L, const uint32_t *popc_U, int64_t R_U, int words_b,
                           WsHeader *hdr, cudaStream_t s) {
    if (R_L <= 0 || R_U <= 0) return cudaSuccess;
    switch (words_b) {
        case 1: return launch_overlap_wb<1>(popc_L, R_L, popc_U, R_U, hdr, s);
        case 2: return launch_overlap_wb<2>(popc_L, R_L, popc_U, R_U, hdr, s);
        case 4: return launch_overlap_wb<4>(popc_L, R_L, popc_U, R_U, hdr, s);
        case 6: return launch_overlap_wb<6>(popc_L, R_L, popc_U, R_U, hdr, s);
        case 8: return launch_overlap_wb<8>(popc_L, R_L, popc_U, R_U, hdr, s);
        case 10: return launch_overlap_wb<10>(popc_L, R_L, popc_U, R_U, hdr, s);
        case 12: return launch_overlap_wb<12>(popc_L, R_L, popc_U, R_U, hdr, s);
        case 16: return launch_overlap_wb<16>(popc_L, R_L, popc_U, R_U, hdr, s);
        case 24: return launch_overlap_wb<24>(popc_L, R_L, popc_U, R_U, hdr, s);
        case 32: return launch_overlap_wb<32>(popc_L, R_L, popc_U, R_U, hdr, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sample(const ClassifyParams &p, uint8_t *states, cudaStream_t s) {
    if (p.N <= 0) return cudaSuccess;
    sample_kernel<<<(unsigned)((p.N + 255) / 256), 256, 0, s>>>(p, states);
    return cudaGetLastError();
}

cudaError_t launch_grad_correction(const ClassifyParams &p, const int64_t *idx, int64_t m, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    const int64_t cgrid = std::min<int64_t>((m + 255) / 256, (int64_t)device_sm_count() * 4);
    grad_index_check_kernel<<<(unsigned)cgrid, 256, 0, s>>>(idx, m, p.N, &p.hdr->grad_bad);
    const int64_t grid = std::min<int64_t>((m + 7) / 8, (int64_t)device_sm_count() * 4);
    grad_correction_kernel<<<(unsigned)grid, 256, 0, s>>>(p, idx, m);
    return cudaGetLastError();
}

}  // namespace rsr
