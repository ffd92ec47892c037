// tc_common.cuh -- the parts shared by the tensor-core classifiers
// (classify_tc.cu: one CTA per MMA; classify_tc2.cu: a CTA pair per MMA):
// sampling a block of 128 samples into the FP8 A tile, the per-bit counts of
// I^L rows for the gradient, and the final flush of counts.
//
// Encoding (an equivalent re-encoding of Sec. 3.2, thermometer instead of
// one-hot for the sample): column j < n(K-1) is (component i, level k), the
// sample row holds A_{h,j} = [x_{h,i} >= k] followed by constant-one bias
// columns; references are encoded by encode_tc_kernel (classify_tc.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rsr_internal.cuh"
#include "tc_ptx.cuh"

namespace rsr {
namespace tc {

constexpr int kTcThreads = 256;  // threads per CTA of both tensor-core kernels
constexpr int kTcRows = 128;     // samples per CTA per block: one A tile of 128 rows

// 4 bits -> 4 bytes of e4m3 {0, 1.0 = 0x38}.
__device__ __forceinline__ uint32_t nibble_to_fp8(uint32_t x) {
    return ((x * 0x00204081u) & 0x01010101u) * 0x38u;
}

// Appends runs of bits to a column of 32-bit words in shared memory (word w of
// thread t at col[w * kTcThreads]).
struct Bits {
    uint32_t *col;
    int w, pos;
    uint32_t cur;
    __device__ __forceinline__ void put(uint32_t bits, int len) {  // len <= 16
        cur |= bits << pos;
        const int np = pos + len;
        if (np >= 32) {
            col[w * kTcThreads] = cur;
            ++w;
            cur = (np > 32) ? (bits >> (32 - pos)) : 0u;
            pos = np - 32;
        } else {
            pos = np;
        }
    }
    __device__ __forceinline__ void finish(int words) {
        if (pos > 0) {
            col[w * kTcThreads] = cur;
            ++w;
        }
        for (; w < words; ++w) col[w * kTcThreads] = 0u;
    }
};

// Samples row0 .. row0 + 127 of the launch (sample h = offset + row, or the
// given states) into the thermometer scratch sTw and the FP8 A tile sA (KP-byte
// rows in the tile_off layout).  Threads t and t + 128 (t < 128) each draw half
// of row t's components (whole Philox blocks); threads from 256 on only take
// part in the barrier.  Rows at or beyond N are all zero.  Every thread of the
// CTA calls it: it contains one __syncthreads (between the bits and their
// expansion); the caller fences the A tile for the async proxy.
__device__ __forceinline__ void sample_a_tile(const ClassifyParams &p, int64_t row0, const unsigned long long *sThr,
                                              uint32_t *sTw, uint8_t *sA, int kp) {
    const int tid = threadIdx.x;
    const bool sampler = tid < kTcThreads;
    const int kwords = kp / 32;
    const int bias_cols = (p.kenc + 15) / 16;
    const int n_half = ((p.n + 7) / 8) * 4;   // a multiple of 4: whole Philox blocks per half
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    if (sampler) {
        const int row = tid & (kTcRows - 1), half = tid >> 7;
        const int64_t hl = row0 + row;
        const int i_lo = half ? (n_half < p.n ? n_half : p.n) : 0;
        const int i_hi = half ? p.n : (n_half < p.n ? n_half : p.n);
        // this thread's bits start at bit i_lo*(K-1) of the row; earlier words stay zero
        const int start = i_lo * p.km1;
        Bits bw{sTw + tid, start >> 5, start & 31, 0u};
        for (int w = 0; w < (start >> 5); ++w) sTw[w * kTcThreads + tid] = 0u;
        if (hl < p.N) {
            if (p.samples) {
                const uint8_t *srow = p.samples + hl * (int64_t)p.n;
                for (int i = i_lo; i < i_hi; ++i) bw.put((1u << srow[i]) - 1u, p.km1);
            } else {
                const uint64_t h = p.offset + (uint64_t)hl;
                // two independent Philox blocks per iteration (instruction-level parallelism)
                for (int q = i_lo / 4; 4 * q < i_hi; q += 2) {
                    const U32x4 ra = philox4x32_10((uint32_t)h, (uint32_t)(h >> 32), (uint32_t)q, 0u, key0, key1);
                    const U32x4 rb =
                        philox4x32_10((uint32_t)h, (uint32_t)(h >> 32), (uint32_t)(q + 1), 0u, key0, key1);
                    const uint32_t us[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const int i = 4 * q + c;
                        if (i < i_hi) {
                            const uint32_t x = state_from_uniform(us[c], sThr + (size_t)i * p.km1, p.km1);
                            bw.put((1u << x) - 1u, p.km1);
                        }
                    }
                }
            }
            if (half) {  // the constant-one bias columns follow the last component
                for (int b = bias_cols; b > 0; b -= 16) {
                    const int len = b < 16 ? b : 16;
                    bw.put((1u << len) - 1u, len);
                }
            }
        }
        bw.finish(kwords);
    }
    __syncthreads();
    if (sampler) {
        // expand the row's bits (the OR of its two halves) to FP8 bytes in the MMA layout;
        // thread t does chunks [0, kp/32) of row t, thread t + 128 the rest
        const int row = tid & (kTcRows - 1), half = tid >> 7;
        const int c_lo = half ? kp / 32 : 0, c_hi = half ? kp / 16 : kp / 32;
        for (int c = c_lo; c < c_hi; ++c) {
            const int w = c >> 1;
            const uint32_t word = sTw[w * kTcThreads + row] | sTw[w * kTcThreads + row + kTcRows];
            const uint32_t b16 = (word >> ((c & 1) * 16)) & 0xFFFFu;
            uint4 v;
            v.x = nibble_to_fp8(b16 & 0xF);
            v.y = nibble_to_fp8((b16 >> 4) & 0xF);
            v.z = nibble_to_fp8((b16 >> 8) & 0xF);
            v.w = nibble_to_fp8((b16 >> 12) & 0xF);
            *reinterpret_cast<uint4 *>(sA + tile_off(row, c, kp)) = v;
        }
    }
}

// Per-bit counts of the I^L rows of one epilogue warp (row = the lane's sample
// row of the A tile), from the thermometer scratch (OR of the two halves),
// added to the block's shared counters sCum.  Called by all 32 lanes.
__device__ __forceinline__ void count_lower_bits(bool isL, int row, int lane, const uint32_t *sTw, uint32_t *sCum,
                                                 int kenc) {
    if (!__ballot_sync(0xffffffffu, isL)) return;
    const int kw = (kenc + 31) / 32;
    for (int w = 0; w < kw; ++w) {
        const uint32_t tw = isL ? (sTw[w * kTcThreads + row] | sTw[w * kTcThreads + row + kTcRows]) : 0u;
        uint32_t mine = 0;
#pragma unroll 4
        for (int b = 0; b < 32; ++b) {
            const uint32_t mm = __ballot_sync(0xffffffffu, (tw >> b) & 1u);
            if (lane == b) mine = __popc(mm);
        }
        if (mine) atomicAdd(&sCum[w * 32 + lane], mine);
    }
}

// Adds the CTA's label counts, executed tests and per-state I^L counts to the
// caller's outputs: C[i][k] = cum_k - cum_{k+1} with cum_0 = |I^L| and
// cum_k = #{I^L rows with x_i >= k} (the thermometer bit counts).
__device__ __forceinline__ void flush_counts(const ClassifyParams &p, const unsigned long long *cnt,
                                             unsigned long long exec, const uint32_t *sCum) {
    const int tid = threadIdx.x;
    if (tid < 3 && cnt[tid]) atomicAdd(&p.counts3[tid], cnt[tid]);
    if (tid == 0 && p.exec_tests && exec) atomicAdd(p.exec_tests, exec);
    if (p.grad_counts && cnt[0]) {
        for (int i = tid; i < p.n; i += blockDim.x) {
            long long prev = (long long)cnt[0];
            for (int k = 1; k <= p.km1; ++k) {
                const long long cum = (long long)sCum[i * p.km1 + (k - 1)];
                const long long dd = prev - cum;
                if (dd) atomicAdd(&p.grad_counts[(size_t)i * p.K + (k - 1)], (unsigned long long)dd);
                prev = cum;
            }
            if (prev) atomicAdd(&p.grad_counts[(size_t)i * p.K + p.km1], (unsigned long long)prev);
        }
    }
}

}  // namespace tc
}  // namespace rsr
