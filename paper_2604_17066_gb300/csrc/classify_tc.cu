// classify_tc.cu -- reference-state classification as a tensor-core
// contraction on sm_103a (tcgen05 + TMEM + bulk async copies).
//
// What it computes (Sec. 3.3, Eq. for the violation matrix, Algorithm 1):
//     V_{h,r} = sum_j A_{h,j} B_{r,j},  sample h classified by r iff V_{h,r} = 0,
// and, exactly as the paper's two products, a sample is in I^L if some lower
// reference gives 0, else in I^U if some upper reference gives 0.  V is never
// written: each 128 x 128 accumulator tile is reduced to "any zero per row" in
// the epilogue straight out of tensor memory.
//
// Encoding (an equivalent re-encoding of Sec. 3.2, thermometer instead of
// one-hot for the sample): j < n(K-1) indexes (component i, level k = 1..K-1).
//   sample row:       A_{h,j} = [x_{h,i} >= k], then `bias` columns equal to 1
//   lower reference:  B_{r,j} = [r_i < k]   (complement), bias columns 0
//                     -> V = #{(i,k): x_i >= k > r_i} >= 0, zero iff x <= r
//   upper reference:  B_{r,j} = [r_i >= k], bias columns sum to -sum_i r_i
//                     -> V = -#{(i,k): r_i >= k > x_i} <= 0, zero iff x >= r
// All values are integers of magnitude <= 16 in FP8 e4m3 and every partial sum
// is an integer far below 2^24, so FP32 accumulation is exact.  Padding
// references carry +1 (lower tiles) or -1 (upper tiles) in the first bias
// column and never give 0.
//
// Kernel structure (one CTA per SM, persistent over 128-sample blocks):
//   all 8 warps : Philox-sample the block's 128 states (two threads per row,
//                 half of the components each) into the FP8 A tile (128 x KP)
//   warp 0      : producer, one cp.async.bulk per B tile of BN references
//                 (BN = 256, the MMA's N; 128 for rows wider than 320 bytes)
//                 into a ring of shared-memory stages; references are
//                 pre-encoded in global memory in the MMA's shared-memory
//                 layout, so BN/128 consecutive encoded tiles are one copy
//   warp 1      : TMEM owner and MMA issuer (KP/32 MMAs of 128 x BN x 32 per
//                 stage into one of two accumulator buffers of BN columns)
//   warps 4-7   : epilogue, the thread of TMEM lane r owns sample row r
// Early exit: the epilogue raises a flag once every row of the block is
// resolved; the producer stops issuing and closes the block with an in-band
// sentinel that walks through the same rings, so every barrier phase stays
// consistent.  Every wait is bounded; on timeout the kernel records
// RSR_ERR_TIMEOUT in the workspace header, frees its TMEM and returns.
#include <algorithm>

#include <cuda_runtime.h>
#include <stdint.h>

#include "rsr_internal.cuh"
#include "rsr_launch.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace rsr {

namespace {

constexpr int kThreads = 256;
constexpr int kRows = 128;           // samples per block: one A tile, the MMA's M
constexpr int kEncTile = kTcRefTile; // rows per encoded reference tile in global memory (128)
constexpr int kMaxStages = 4;
constexpr int kSmemLimit = 232448;   // 227 KB opt-in per CTA
// tensor memory: two FP32 accumulator buffers of BN columns each (BN = MMA N)
using namespace tc;

struct TcSmem {
    // offsets (bytes) from the dynamic shared memory base
    uint32_t a, stages, tw, thr, cum, total;
    int nstages;
};

__host__ __device__ inline TcSmem tc_smem_plan(int kp, int nthr, int bn, int stages_cap) {
    TcSmem s{};
    uint32_t off = 0;
    s.a = off;
    off += (uint32_t)kRows * kp;
    s.tw = off;
    off += (uint32_t)(kp / 32) * kThreads * 4;
    s.thr = off;
    off += (uint32_t)((nthr * 8 + 127) / 128 * 128);
    s.cum = off;
    off += (uint32_t)kp * 4;
    off = (off + 1023) & ~1023u;
    s.stages = off;
    const uint32_t stage_bytes = (uint32_t)bn * kp;
    int ns = 0;
    while (ns < stages_cap && off + (ns + 1) * stage_bytes + 1024 <= (uint32_t)kSmemLimit) ++ns;
    s.nstages = ns;
    s.total = off + ns * stage_bytes;
    return s;
}

struct TcCtl {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t drain;      // after an abort: completion of every MMA issued so far
    int stage_tile[kMaxStages];
    int acc_tile[2];
    uint32_t tmem_base;
    int done;
    int nres;
    int abort_flag;
    unsigned long long exec;
    unsigned long long cnt[3];
};

// BN = references per B tile = MMA N (256, or 128 for rows too wide for two
// 256-row stages).  A block is 128 samples: thread t and t + 128 each sample
// half of row t's components (Philox blocks are independent), so all 8 warps
// generate; the epilogue thread of TMEM lane r owns sample row r.
template <int BN>
__global__ void __launch_bounds__(kThreads, 1) classify_tc_kernel(const ClassifyParams p) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ TcCtl ctl;
    constexpr uint32_t kTmemCols = 2 * BN;
    constexpr uint32_t kIdesc = idesc_f8<kRows, BN>();
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const int kp = p.tc_kpad;
    const int nthr = p.n * p.km1;
    const TcSmem plan = tc_smem_plan(kp, nthr, BN, kMaxStages);
    const int S = plan.nstages;
    uint8_t *sA = smem + plan.a;
    uint8_t *sStage = smem + plan.stages;
    uint32_t *sTw = reinterpret_cast<uint32_t *>(smem + plan.tw);
    unsigned long long *sThr = reinterpret_cast<unsigned long long *>(smem + plan.thr);
    uint32_t *sCum = reinterpret_cast<uint32_t *>(smem + plan.cum);
    volatile int *abort_flag = &ctl.abort_flag;
    int32_t *err = &p.hdr->error;
    const long long budget = p.test_stall ? kTestWaitCycles : kWaitCycles;

    for (int i = tid; i < nthr; i += kThreads) sThr[i] = p.thr[i];
    for (int j = tid; j < kp; j += kThreads) sCum[j] = 0u;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&ctl.full[s], 1);
            mbar_init(&ctl.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ctl.tfull[b], 2);    // MMA completion + the issuer's release arrive
            mbar_init(&ctl.tempty[b], 4);   // one arrive per epilogue warp
        }
        mbar_init(&ctl.drain, 1);
        ctl.done = 0;
        ctl.abort_flag = 0;
        ctl.exec = 0ull;
        ctl.cnt[0] = ctl.cnt[1] = ctl.cnt[2] = 0ull;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(&ctl.tmem_base, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl.tmem_base;

    const bool overlap = *((volatile const int32_t *)&p.hdr->overlap) != 0;
    // tile order: chunk_at() (alternating without overlapping pairs, lower first with them)
    const int64_t tiles_U = (p.R_U + BN - 1) / BN;
    const int64_t tiles_L = (p.R_L + BN - 1) / BN;
    const int64_t T = tiles_U + tiles_L;
    const uint32_t tile_bytes = (uint32_t)BN * kp;   // BN/128 consecutive encoded tiles

    // ring state (continuous across blocks)
    int st_stage = 0;
    uint32_t st_phase = 0;
    // producer: full-barrier phase of the last copy into each stage (bit s set = a copy was issued)
    uint32_t copy_phase = 0u, copy_made = 0u;
    int acc_buf = 0;
    uint32_t acc_phase = 0;

    // epilogue per-thread totals
    unsigned long long c0 = 0, c1 = 0, c2 = 0;

    const int64_t nblocks = (p.N + kRows - 1) / kRows;
    for (int64_t blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
        // ---- 1. sample the block into the thermometer scratch and the A tile -----
        sample_a_tile(p, blk * kRows, sThr, sTw, sA, kp);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (tid == 0) {
            ctl.done = 0;
            ctl.nres = 0;
        }
        __syncthreads();

        // ---- 2. roles -----------------------------------------------------------
        if (warp == 0) {
            if (lane == 0 && !p.test_stall) {
                for (int64_t j = 0; j <= T; ++j) {
                    const bool stop = (j == T) || (!p.dense && *((volatile int *)&ctl.done));
                    if (!mbar_wait(&ctl.empty[st_stage], st_phase ^ 1u, abort_flag, err, budget)) break;
                    if (stop) {
                        ctl.stage_tile[st_stage] = -1;
                        copy_made &= ~(1u << st_stage);   // the stage's last copy was consumed (empty wait)
                        mbar_arrive(&ctl.full[st_stage]);
                    } else {
                        ctl.stage_tile[st_stage] = (int)j;
                        bool up;
                        int64_t ti;
                        chunk_at(j, tiles_U, tiles_L, overlap, &up, &ti);
                        const uint8_t *src = (up ? p.tc_U : p.tc_L) + (size_t)ti * tile_bytes;
                        mbar_arrive_expect_tx(&ctl.full[st_stage], tile_bytes);
                        bulk_g2s(sStage + (size_t)st_stage * tile_bytes, src, tile_bytes, &ctl.full[st_stage]);
                        copy_made |= 1u << st_stage;
                        copy_phase = (copy_phase & ~(1u << st_stage)) | (st_phase << st_stage);
                    }
                    if (++st_stage == S) {
                        st_stage = 0;
                        st_phase ^= 1u;
                    }
                    if (stop) break;
                }
            }
        } else if (warp == 1) {
            if (lane == 0) {
                const uint32_t a_base = smem_u32(sA);
                const uint32_t sbo = (uint32_t)kp * 8u;
                unsigned long long issued = 0;
                while (true) {
                    if (!mbar_wait(&ctl.full[st_stage], st_phase, abort_flag, err, budget)) break;
                    const int j = ctl.stage_tile[st_stage];
                    if (!mbar_wait(&ctl.tempty[acc_buf], acc_phase ^ 1u, abort_flag, err, budget)) break;
                    ctl.acc_tile[acc_buf] = j;
                    if (j < 0) {
                        mbar_arrive(&ctl.empty[st_stage]);
                        mbar_arrive(&ctl.tfull[acc_buf], 2);
                    } else {
                        tc_fence_after();
                        const uint32_t b_base = smem_u32(sStage + (size_t)st_stage * tile_bytes);
                        const uint32_t d = tmem + (uint32_t)(acc_buf * BN);
#pragma unroll 1
                        for (int kk = 0; kk < kp / 32; ++kk) {
                            const uint64_t ad = smem_desc(a_base + kk * 256, 128, sbo);
                            const uint64_t bd = smem_desc(b_base + kk * 256, 128, sbo);
                            mma_f8(d, ad, bd, kIdesc, kk > 0 ? 1u : 0u);
                        }
                        mma_commit(&ctl.empty[st_stage]);
                        mma_commit(&ctl.tfull[acc_buf]);
                        mbar_arrive(&ctl.tfull[acc_buf]);  // release of acc_tile
                        ++issued;
                    }
                    if (++st_stage == S) {
                        st_stage = 0;
                        st_phase ^= 1u;
                    }
                    if (++acc_buf == 2) {
                        acc_buf = 0;
                        acc_phase ^= 1u;
                    }
                    if (j < 0) break;
                }
                ctl.exec += issued * (unsigned long long)(BN * kRows);
            }
        } else if (warp >= 4) {
            const int q = warp & 3;              // TMEM lane quarter
            const int row = q * 32 + lane;       // sample row of this thread
            const int64_t h = blk * kRows + row;
            const bool v = h < p.N;
            bool mL = false, mU = false;
            bool warp_resolved = false;
            while (true) {
                if (!mbar_wait(&ctl.tfull[acc_buf], acc_phase, abort_flag, err, budget)) break;
                const int j = ctl.acc_tile[acc_buf];
                if (j >= 0) {
                    tc_fence_after();
                    bool is_upper;
                    int64_t ti;
                    chunk_at(j, tiles_U, tiles_L, overlap, &is_upper, &ti);
                    float m = 1.0f;
                    const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc_buf * BN);
#pragma unroll 1
                    for (int c = 0; c < BN / 64; ++c) {
                        uint32_t va[32], vb[32];
                        tmem_ld32(tbase + c * 64, va);
                        tmem_ld32(tbase + c * 64 + 32, vb);
                        tmem_ld_wait();
#pragma unroll
                        for (int e = 0; e < 32; ++e)
                            m = fminf(m, fminf(fabsf(__uint_as_float(va[e])), fabsf(__uint_as_float(vb[e]))));
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&ctl.tempty[acc_buf]);
                    const bool z = m < 0.5f;
                    if (is_upper) mU |= z; else mL |= z;
                    if (!p.dense && !warp_resolved) {
                        // resolved: any lower match, or an upper match that precedence cannot
                        // overturn (with overlaps the lower tiles come first)
                        const bool l_done = overlap ? (j + 1 >= tiles_L) : true;
                        const bool r = !v || mL || (mU && (!overlap || l_done));
                        // resolution is monotone: each warp reports once; the fourth report ends the block
                        if (__all_sync(0xffffffffu, r)) {
                            warp_resolved = true;
                            if (lane == 0 && atomicAdd(&ctl.nres, 1) == 3) *((volatile int *)&ctl.done) = 1;
                        }
                    }
                } else {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&ctl.tempty[acc_buf]);
                }
                if (++acc_buf == 2) {
                    acc_buf = 0;
                    acc_phase ^= 1u;
                }
                if (j < 0) break;
            }
            const int lab = mL ? 0 : (mU ? 1 : 2);
            if (v) {
                if (p.labels) p.labels[h] = (uint8_t)lab;
                c0 += lab == 0; c1 += lab == 1; c2 += lab == 2;
            }
            if (p.grad_counts) count_lower_bits(v && lab == 0, row, lane, sTw, sCum, p.kenc);
        }
        // Each role advanced its private copy of the ring positions by the same
        // number of entries (issued tiles + the sentinel), so the copies agree.
        if (*abort_flag && lane == 0) {
            if (warp == 0) {
                // every copy issued into a stage completes its full barrier's phase:
                // wait for the last one of each stage before shared memory is released
                for (int s = 0; s < S; ++s)
                    if (copy_made & (1u << s)) (void)mbar_wait_drain(&ctl.full[s], (copy_phase >> s) & 1u);
            } else if (warp == 1) {
                // a commit tracks every MMA this thread issued before it
                mma_commit(&ctl.drain);
                (void)mbar_wait_drain(&ctl.drain, 0u);
            }
        }
        __syncthreads();
        if (*abort_flag) break;
    }

    // ---- totals -------------------------------------------------------------
    if (warp >= 4) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c0 += __shfl_xor_sync(0xffffffffu, c0, o);
            c1 += __shfl_xor_sync(0xffffffffu, c1, o);
            c2 += __shfl_xor_sync(0xffffffffu, c2, o);
        }
        if (lane == 0) {
            atomicAdd(&ctl.cnt[0], c0);
            atomicAdd(&ctl.cnt[1], c1);
            atomicAdd(&ctl.cnt[2], c2);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);   // after an abort, the drain above waited for the MMAs
    }
    flush_counts(p, ctl.cnt, ctl.exec, sCum);
}

// Reference rows in the MMA layout: tile t = r / 128 holds rows r in
// [128 t, 128 t + 128), each KP bytes, core-matrix blocked (tile_off).
__global__ void encode_tc_kernel(const uint8_t *__restrict__ refs, const int32_t *__restrict__ perm, int64_t R,
                                 int64_t rows, int n, int km1, int kp, int upper, uint8_t *__restrict__ out) {
    const int chunks = kp / 16;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= rows * chunks) return;
    const int64_t r = gid / chunks;                                        // slot (row of the tile matrix)
    const int64_t src = (r < R && perm) ? (int64_t)perm[r] : r;            // reference stored in it
    const int c = (int)(gid % chunks);
    const int kenc = n * km1;
    const int bias_cols = (kenc + 15) / 16;
    int total = 0;  // sum_i r_i, the number of thermometer ones of an upper reference
    if (r < R && upper)
        for (int i = 0; i < n; ++i) total += refs[src * n + i];
    uint8_t bytes[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int j = c * 16 + e;
        float v = 0.0f;
        if (r >= R) {
            // padding: never zero, and of the sign of the set's real values (lower
            // V >= 0, upper V <= 0) so that a min / max reduction ignores it
            v = (j == kenc) ? (upper ? -1.0f : 1.0f) : 0.0f;
        } else if (j < kenc) {
            const int i = j / km1, k = j % km1 + 1;
            const bool a = refs[src * n + i] >= k;
            v = upper ? (a ? 1.0f : 0.0f) : (a ? 0.0f : 1.0f);
        } else if (j < kenc + bias_cols && upper) {
            const int used = (j - kenc) * 16;
            const int rem = total - used;
            v = rem <= 0 ? 0.0f : -(float)(rem < 16 ? rem : 16);
        }
        // e4m3 encodings of the integers -16..1 used here
        uint8_t b = 0;
        if (v == 1.0f) b = 0x38;
        else if (v < 0.0f) {
            const int m = (int)(-v);  // 1..16
            // exponent e, mantissa f: m = (1 + f/8) 2^e
            int e2 = 0;
            while ((m >> (e2 + 1)) != 0) ++e2;
            const int f = ((m << 3) >> e2) & 7;
            b = (uint8_t)(0x80 | ((e2 + 7) << 3) | f);
        }
        bytes[e] = b;
    }
    const int64_t t = r / kEncTile;
    const int rr = (int)(r % kEncTile);
    uint8_t *dst = out + (size_t)t * kEncTile * kp + tile_off(rr, c, kp);
    uint4 v;
    v.x = (uint32_t)bytes[0] | ((uint32_t)bytes[1] << 8) | ((uint32_t)bytes[2] << 16) | ((uint32_t)bytes[3] << 24);
    v.y = (uint32_t)bytes[4] | ((uint32_t)bytes[5] << 8) | ((uint32_t)bytes[6] << 16) | ((uint32_t)bytes[7] << 24);
    v.z = (uint32_t)bytes[8] | ((uint32_t)bytes[9] << 8) | ((uint32_t)bytes[10] << 16) | ((uint32_t)bytes[11] << 24);
    v.w = (uint32_t)bytes[12] | ((uint32_t)bytes[13] << 8) | ((uint32_t)bytes[14] << 16) | ((uint32_t)bytes[15] << 24);
    *reinterpret_cast<uint4 *>(dst) = v;
}

}  // namespace

bool tc_supported() {
    static int cached = -1;
    if (cached < 0) {
        int dev = 0, major = 0, minor = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        cached = (major == 10 && minor == 3) ? 1 : 0;
    }
    return cached == 1;
}

int tc_max_kpad() { return 512; }  // widest row whose A tile and two 128-wide B stages fit

cudaError_t launch_encode_tc(const uint8_t *refs, int64_t R, int64_t rows_padded, int n, int km1, int kpad,
                             bool upper, uint8_t *out, cudaStream_t s, const int32_t *perm) {
    if (rows_padded <= 0) return cudaSuccess;
    const int64_t total = rows_padded * (kpad / 16);
    encode_tc_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(refs, perm, R, rows_padded, n, km1, kpad,
                                                                     upper ? 1 : 0, out);
    return cudaGetLastError();
}

namespace {

template <int BN>
cudaError_t launch_tc_bn(const ClassifyParams &p, cudaStream_t s) {
    // dynamic shared memory up to the opt-in limit minus the kernel's static
    // shared memory; set once per device so that captured launches issue nothing else
    static size_t max_dyn[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (max_dyn[dev] == 0) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, classify_tc_kernel<BN>);
        if (e != cudaSuccess) return e;
        int optin = 0;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        const size_t lim = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
        e = cudaFuncSetAttribute(classify_tc_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
        if (e != cudaSuccess) return e;
        max_dyn[dev] = lim;
    }
    const TcSmem plan = tc_smem_plan(p.tc_kpad, p.n * p.km1, BN, kMaxStages);
    if (plan.nstages < 2) return cudaErrorNotSupported;
    // at least 120 KB so that two CTAs never share an SM (each takes 2*BN TMEM columns)
    const size_t smem = plan.total > 122880u ? plan.total : 122880u;
    if (smem > max_dyn[dev]) return cudaErrorNotSupported;
    const int64_t nblocks = (p.N + kRows - 1) / kRows;
    const int64_t grid = std::min<int64_t>(nblocks, (int64_t)device_sm_count());
    if (grid <= 0) return cudaSuccess;
    classify_tc_kernel<BN><<<(unsigned)grid, kThreads, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

// MMA N = 256 (one instruction covers 256 references) whenever two 256-row
// B stages fit next to the A tile; narrower 128-row tiles for wider rows.
cudaError_t launch_classify_tc(const ClassifyParams &p, cudaStream_t s) {
    if (p.tc_kpad > tc_max_kpad() || p.tc_kpad % 32 != 0) return cudaErrorNotSupported;
    // dense mode: the CTA-pair kernel (classify_tc2.cu) halves the shared-memory
    // traffic per MMA; early exit stays here (its blocks stop at different tiles)
    if (p.dense && tc2_available(p.tc_kpad)) return launch_classify_tc2(p, s);
    if (tc_smem_plan(p.tc_kpad, p.n * p.km1, 256, kMaxStages).nstages >= 2) return launch_tc_bn<256>(p, s);
    return launch_tc_bn<128>(p, s);
}

}  // namespace rsr
