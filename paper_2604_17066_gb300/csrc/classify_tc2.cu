// classify_tc2.cu -- dense reference-state classification on a CTA pair
// (tcgen05 cta_group::2, M = 256) on sm_103a.
//
// What it computes is the violation product of Sec. 3.3 and the first-match
// labels of Algorithm 1, exactly as classify_tc.cu: V_{h,r} = sum_j A_{h,j}
// B_{r,j} over the thermometer encoding, a sample is classified by r iff
// V_{h,r} = 0, lower before upper, and V is never written.  This kernel runs
// the dense mode (every sample against every reference).
//
// Why a pair: one CTA issuing M = 128 x N = 256 x K = 32 FP8 MMAs reads 12 KB
// of operands from its shared memory per instruction and receives the whole
// 256-reference B tile by bulk copy, about 160 bytes per cycle at the full MMA
// rate against the 128 bytes per cycle that shared memory delivers.  Here two
// CTAs of a cluster share each MMA (M = 256 = 128 samples per CTA): each CTA
// holds its own A tile and HALF of every B tile (128 references), so both the
// B operand read and the B tile copy per SM are halved (96 bytes per cycle).
//
// Roles (256 threads per CTA, one CTA per SM, rank 0 = leader, 1 = peer):
//   all 8 warps : Philox-sample the CTA's 128 rows of the pair block into its
//                 FP8 A tile (tc_common.cuh), then a cluster barrier
//   warp 0      : producer in each CTA: one cp.async.bulk per stage, its half
//                 (one encoded 128-row tile) of B tile j, into its own ring
//   warps 1, 2  : both CTAs' warp 1 allocates the pair's tensor memory
//                 (cta_group::2); in the leader, warps 1 and 2 issue the MMAs
//                 of the even and odd tiles (one accumulator each), which write
//                 each CTA's 128 rows of D into that CTA's tensor memory; in the
//                 peer, warp 1 forwards the completion of its stages to the
//                 leader (remote arrive)
//   warps 4-7   : epilogue in each CTA, the thread of TMEM lane r owns sample
//                 row r; it reduces "some V = 0" over the 256 columns (a min
//                 on lower tiles, where V >= 0; a max on upper tiles, where
//                 V <= 0) and arrives on the leader's accumulator-empty barrier
// Barriers: full[s] (own copy), pfull[s] (leader: the peer's copy of stage s
// landed), empty[s] and tfull[b] (the leader's commits, multicast to both
// CTAs), tempty[b] (leader: the eight epilogue warps of the pair have read
// accumulator b).
// Every wait is bounded.  After a timeout the copies and MMAs already issued
// are waited for (bounded), both CTAs meet at a cluster barrier, decide to
// stop together (each reads the other's abort flag), free the tensor memory
// and return; RSR_ERR_TIMEOUT is left in the workspace header.
#include <algorithm>

#include <cuda_runtime.h>
#include <stdint.h>

#include "rsr_internal.cuh"
#include "rsr_launch.h"
#include "tc_common.cuh"
#include "tc_ptx.cuh"

namespace rsr {

namespace {

using namespace tc;

constexpr int kThreads = kTcThreads;   // 8 warps
constexpr int kProducerWarp = 0;
constexpr int kMmaWarp = 1;            // leader: issues the even tiles; peer: forwards stage completions
constexpr int kMmaWarp2 = 2;           // leader: issues the odd tiles
constexpr int kEpiWarp0 = 4;           // warps 4-7: one per TMEM lane quarter
constexpr int kRows = kTcRows;       // samples per CTA per pair block (the pair: 256)
constexpr int kHalfRefs = 128;       // references per CTA per B tile: one encoded 128-row tile
constexpr int kPairRefs = 256;       // references per B tile: the MMA's N
constexpr int kMaxStages = 6;
constexpr int kSmemLimit = 232448;   // 227 KB opt-in per CTA
constexpr uint32_t kTmemCols = 2 * kPairRefs;   // two FP32 accumulators of N = 256 columns
constexpr uint16_t kBoth = 0x3;      // cluster ranks 0 and 1
static_assert(kTcRefTile == kHalfRefs, "a CTA's half of a B tile is one encoded reference tile");

struct PairSmem {
    uint32_t a, tw, thr, cum, stages, total;   // byte offsets from the dynamic shared memory base
    int nstages;
};

__host__ __device__ inline PairSmem pair_smem_plan(int kp, int nthr) {
    PairSmem s{};
    uint32_t off = 0;
    s.a = off;
    off += (uint32_t)kRows * kp;
    s.tw = off;
    off += (uint32_t)(kp / 32) * kTcThreads * 4;   // thermometer words of the 256 sampling threads
    s.thr = off;
    off += (uint32_t)((nthr * 8 + 127) / 128 * 128);
    s.cum = off;
    off += (uint32_t)kp * 4;
    off = (off + 1023) & ~1023u;
    s.stages = off;
    const uint32_t stage_bytes = (uint32_t)kHalfRefs * kp;
    int ns = 0;
    while (ns < kMaxStages && off + (ns + 1) * stage_bytes + 1024 <= (uint32_t)kSmemLimit) ++ns;
    s.nstages = ns;
    s.total = off + ns * stage_bytes;
    return s;
}

struct PairCtl {
    uint64_t full[kMaxStages];    // this CTA's copy of stage s landed (expect_tx + complete_tx)
    uint64_t empty[kMaxStages];   // the MMAs reading stage s completed (leader's commit, both CTAs)
    uint64_t pfull[kMaxStages];   // leader: the peer's copy of stage s landed (peer's remote arrive)
    uint64_t tfull[2];            // accumulator b holds a finished tile (leader's commit, both CTAs)
    uint64_t tempty[2];           // leader: the 8 epilogue warps of the pair have read accumulator b
    uint64_t drain;               // leader, after an abort: every MMA issued so far completed (2 issuers)
    uint32_t tmem_base;
    int abort_flag;
    unsigned long long exec;
    unsigned long long cnt[3];
};

// What one launch classifies.  One problem: p0, in pair blocks of 256
// samples.  A batch (the tensor-core scenarios of rsr_batch): descs[s] per
// scenario, items [begin[s], begin[s+1]) are its pair blocks, and scenario s
// classifies samples offset + round*N .. of its stream.
struct PairWork {
    const ClassifyParams *descs;           // device, or NULL for one problem
    const int64_t *begin;                  // device [S+1]
    const unsigned long long *round;       // device, the batch's round counter
    int S;
    int kp_max, nthr_max;                  // widest row and largest threshold table of the launch
    int64_t total_items;
};

template <bool kBatch>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
    classify_tc2_kernel(const ClassifyParams p0, const PairWork wk) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ PairCtl ctl;
    __shared__ ClassifyParams sp;   // batch: the current scenario (offset moved to its round)
    __shared__ int s_scen;
    __shared__ int s_changed;
    __shared__ long long s_item0;   // batch: first item of the current scenario
    constexpr uint32_t kIdesc = idesc_f8<2 * kRows, kPairRefs>();
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const uint32_t rank = cluster_ctarank();
    const bool leader = rank == 0;
    const PairSmem plan = pair_smem_plan(wk.kp_max, wk.nthr_max);
    const int S = plan.nstages;
    const uint32_t stage_stride = (uint32_t)kHalfRefs * wk.kp_max;
    uint8_t *sA = smem + plan.a;
    uint8_t *sStage = smem + plan.stages;
    uint32_t *sTw = reinterpret_cast<uint32_t *>(smem + plan.tw);
    unsigned long long *sThr = reinterpret_cast<unsigned long long *>(smem + plan.thr);
    uint32_t *sCum = reinterpret_cast<uint32_t *>(smem + plan.cum);
    volatile int *abort_flag = &ctl.abort_flag;
    const ClassifyParams &p = kBatch ? sp : p0;

    if (!kBatch)
        for (int i = tid; i < p0.n * p0.km1; i += kThreads) sThr[i] = p0.thr[i];
    for (int j = tid; j < wk.kp_max; j += kThreads) sCum[j] = 0u;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&ctl.full[s], 1);
            mbar_init(&ctl.empty[s], 1);
            mbar_init(&ctl.pfull[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ctl.tfull[b], 1);
            mbar_init(&ctl.tempty[b], 8);   // four epilogue warps per CTA
        }
        mbar_init(&ctl.drain, 2);   // one commit from each issuing thread
        ctl.abort_flag = 0;
        ctl.exec = 0ull;
        ctl.cnt[0] = ctl.cnt[1] = ctl.cnt[2] = 0ull;
        s_scen = -1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        tmem_alloc_pair(&ctl.tmem_base, kTmemCols);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();   // both CTAs' barriers are initialised before any remote arrive
    tc_fence_after();
    const uint32_t tmem = ctl.tmem_base;
    const unsigned long long round = kBatch ? *((volatile const unsigned long long *)wk.round) : 0ull;

    // the leader's barriers as the peer reaches them
    const uint32_t pfull_at_leader = cluster_map(&ctl.pfull[0], 0);
    const uint32_t tempty_at_leader = cluster_map(&ctl.tempty[0], 0);
    const uint32_t partner_abort = cluster_map(&ctl.abort_flag, rank ^ 1u);

    // ring state (continuous across blocks; every role advances T entries per block)
    int st_stage = 0;
    uint32_t st_phase = 0;
    int acc_buf = 0;
    uint32_t acc_phase = 0;
    uint32_t copy_phase = 0u, copy_made = 0u;   // producer: phase of the last copy into each stage
    int64_t g_base = 0;                         // tiles of the earlier blocks (tile g uses stage g mod S, accumulator g mod 2)

    const int64_t n_items = kBatch ? wk.total_items : (p0.N + 2 * kRows - 1) / (2 * kRows);
    for (int64_t item = cluster_id_x(); item < n_items; item += cluster_count_x()) {
        int64_t pb = item;
        if (kBatch) {
            // the scenario of this item (the same in both CTAs: both walk the same items)
            if (tid == 0) {
                int lo = 0, hi = wk.S - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (wk.begin[mid] <= item) lo = mid; else hi = mid - 1;
                }
                s_changed = lo != s_scen;
                if (s_changed) {
                    s_scen = lo;
                    sp = wk.descs[lo];
                    sp.offset += round * (unsigned long long)sp.N;
                    s_item0 = wk.begin[lo];
                }
            }
            __syncthreads();
            if (s_changed) {
                for (int i = tid; i < sp.n * sp.km1; i += kThreads) sThr[i] = sp.thr[i];
                __syncthreads();   // the sampler reads the table before its own barrier
            }
            pb = item - s_item0;
        }
        const int kp = p.tc_kpad;
        const bool overlap = *((volatile const int32_t *)&p.hdr->overlap) != 0;
        const int64_t tiles_U = (p.R_U + kPairRefs - 1) / kPairRefs;
        const int64_t tiles_L = (p.R_L + kPairRefs - 1) / kPairRefs;
        const int64_t T = tiles_U + tiles_L;
        // Every other item of a pair walks the B tiles backwards.  The pairs take their
        // items in step, so at any time they read about the same tiles, and the tiles a
        // sweep read last are still in L2 when the next sweep starts on them.  Dense
        // labels do not depend on the order of the tiles.
        const bool rev = (((item - (int64_t)cluster_id_x()) / (int64_t)cluster_count_x()) & 1) != 0;
        const uint32_t half_bytes = (uint32_t)kHalfRefs * kp;
        int32_t *err = &p.hdr->error;
        const long long budget = p.test_stall ? kTestWaitCycles : kWaitCycles;
        const int64_t row0 = pb * (2 * kRows) + (int64_t)rank * kRows;
        sample_a_tile(p, row0, sThr, sTw, sA, kp);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        cluster_sync();   // both A tiles are written before the leader's first MMA of the block

        if (warp == kProducerWarp) {
            if (lane == 0 && !p.test_stall) {
                for (int64_t j = 0; j < T; ++j) {
                    if (!mbar_wait(&ctl.empty[st_stage], st_phase ^ 1u, abort_flag, err, budget)) break;
                    bool up;
                    int64_t ti;
                    chunk_at(rev ? T - 1 - j : j, tiles_U, tiles_L, overlap, &up, &ti);
                    const uint8_t *src = (up ? p.tc_U : p.tc_L) + (size_t)(2 * ti + rank) * half_bytes;
                    mbar_arrive_expect_tx(&ctl.full[st_stage], half_bytes);
                    bulk_g2s(sStage + (size_t)st_stage * stage_stride, src, half_bytes, &ctl.full[st_stage]);
                    copy_made |= 1u << st_stage;
                    copy_phase = (copy_phase & ~(1u << st_stage)) | (st_phase << st_stage);
                    if (++st_stage == S) {
                        st_stage = 0;
                        st_phase ^= 1u;
                    }
                }
            }
        } else if (warp == kMmaWarp || warp == kMmaWarp2) {
            if (lane == 0 && leader) {
                // Two issuing threads, one per accumulator (tile parity): while one is
                // blocked in the MMA queue the other commits and waits for its next tile,
                // so the tensor pipe is not left idle between tiles.
                const int64_t parity = warp == kMmaWarp ? 0 : 1;
                const uint32_t a_base = smem_u32(sA);
                const uint32_t sbo = (uint32_t)kp * 8u;
                unsigned long long issued = 0;
                for (int64_t j = 0; j < T; ++j) {
                    if (((g_base + j) & 1) == parity) {
                        if (!mbar_wait(&ctl.full[st_stage], st_phase, abort_flag, err, budget)) break;
                        if (!mbar_wait(&ctl.pfull[st_stage], st_phase, abort_flag, err, budget)) break;
                        if (!mbar_wait(&ctl.tempty[acc_buf], acc_phase ^ 1u, abort_flag, err, budget)) break;
                        tc_fence_after();
                        const uint32_t b_base = smem_u32(sStage + (size_t)st_stage * stage_stride);
                        const uint32_t d = tmem + (uint32_t)(acc_buf * kPairRefs);
#pragma unroll 1
                        for (int kk = 0; kk < kp / 32; ++kk)
                            mma_f8_pair(d, smem_desc(a_base + kk * 256, 128, sbo),
                                        smem_desc(b_base + kk * 256, 128, sbo), kIdesc, kk > 0 ? 1u : 0u);
                        mma_commit_pair(&ctl.empty[st_stage], kBoth);
                        mma_commit_pair(&ctl.tfull[acc_buf], kBoth);
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
                }
                if (issued) atomicAdd(&ctl.exec, issued * (unsigned long long)(kPairRefs * 2 * kRows));
            } else if (lane == 0 && warp == kMmaWarp) {
                // peer: tell the leader when each stage of this CTA has landed
                for (int64_t j = 0; j < T; ++j) {
                    if (!mbar_wait(&ctl.full[st_stage], st_phase, abort_flag, err, budget)) break;
                    mbar_arrive_cluster(pfull_at_leader + 8u * (uint32_t)st_stage);
                    if (++st_stage == S) {
                        st_stage = 0;
                        st_phase ^= 1u;
                    }
                }
            }
        } else if (warp >= kEpiWarp0) {
            const int q = warp & 3;          // TMEM lane quarter
            const int row = q * 32 + lane;   // sample row of this thread in the CTA's A tile
            const int64_t h = row0 + row;
            const bool v = h < p.N;
            bool mL = false, mU = false;
            for (int64_t j = 0; j < T; ++j) {
                if (!mbar_wait(&ctl.tfull[acc_buf], acc_phase, abort_flag, err, budget)) break;
                tc_fence_after();
                bool is_upper;
                int64_t ti;
                chunk_at(rev ? T - 1 - j : j, tiles_U, tiles_L, overlap, &is_upper, &ti);
                // V >= 0 against lower references and V <= 0 against upper ones (padding
                // rows give +1 / -1), so "some V = 0" is min V < 0.5 on a lower tile and
                // max V > -0.5 on an upper tile
                float m = is_upper ? -1.0f : 1.0f;
                const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc_buf * kPairRefs);
                // 128 columns per load round trip (the latency of a tensor-memory load,
                // not the arithmetic, sets the epilogue's time)
#pragma unroll 1
                for (int c = 0; c < kPairRefs / 128; ++c) {
                    uint32_t va[64], vb[64];
                    tmem_ld64(tbase + c * 128, va);
                    tmem_ld64(tbase + c * 128 + 64, vb);
                    tmem_ld_wait();
                    if (is_upper) {
#pragma unroll
                        for (int e = 0; e < 64; ++e) m = fmax3(m, __uint_as_float(va[e]), __uint_as_float(vb[e]));
                    } else {
#pragma unroll
                        for (int e = 0; e < 64; ++e) m = fmin3(m, __uint_as_float(va[e]), __uint_as_float(vb[e]));
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(tempty_at_leader + 8u * (uint32_t)acc_buf);
                const bool z = is_upper ? (m > -0.5f) : (m < 0.5f);
                if (is_upper) mU |= z; else mL |= z;
                if (++acc_buf == 2) {
                    acc_buf = 0;
                    acc_phase ^= 1u;
                }
            }
            const int lab = mL ? 0 : (mU ? 1 : 2);
            if (v && p.labels) p.labels[h] = (uint8_t)lab;
            if (p.grad_counts) count_lower_bits(v && lab == 0, row, lane, sTw, sCum, p.kenc);
            // the item's label counts
            unsigned long long c0 = __popc(__ballot_sync(0xffffffffu, v && lab == 0));
            unsigned long long c1 = __popc(__ballot_sync(0xffffffffu, v && lab == 1));
            unsigned long long c2 = __popc(__ballot_sync(0xffffffffu, v && lab == 2));
            if (lane == 0) {
                if (c0) atomicAdd(&ctl.cnt[0], c0);
                if (c1) atomicAdd(&ctl.cnt[1], c1);
                if (c2) atomicAdd(&ctl.cnt[2], c2);
            }
        }
        if (*abort_flag && lane == 0) {
            if (warp == kProducerWarp) {
                // every copy issued into a stage completes that stage's full barrier
                for (int s = 0; s < S; ++s)
                    if (copy_made & (1u << s)) (void)mbar_wait_drain(&ctl.full[s], (copy_phase >> s) & 1u);
                copy_made = 0u;
            } else if ((warp == kMmaWarp || warp == kMmaWarp2) && leader) {
                mma_commit_pair(&ctl.drain, 0x1);   // tracks every MMA this thread issued before it
                (void)mbar_wait_drain(&ctl.drain, 0u);
            }
        }
        g_base += T;
        __syncthreads();
        // the item's counts (label counts, executed tests, per-state I^L counts from the
        // bit counts) go to its problem, and the shared totals start again at zero
        flush_counts(p, ctl.cnt, ctl.exec, sCum);
        __syncthreads();
        if (tid < 3) ctl.cnt[tid] = 0ull;
        if (tid == 0) ctl.exec = 0ull;
        for (int j = tid; j < kp; j += kThreads) sCum[j] = 0u;
        cluster_sync();
        // Every role of both CTAs has finished this block, so both abort flags
        // are final here; both CTAs take the same decision.
        if (*abort_flag || ld_cluster_s32(partner_abort)) break;
    }

    if (warp == kProducerWarp && lane == 0) {
        // the leader's last commits to this CTA's empty barriers have arrived
        for (int s = 0; s < S; ++s)
            if (copy_made & (1u << s)) (void)mbar_wait_drain(&ctl.empty[s], (copy_phase >> s) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();   // neither CTA touches the other's barriers or tensor memory any more
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, kTmemCols);
    }
}

}  // namespace

// Pairs that can be resident at once (one CTA per SM, both CTAs of a pair in
// one GPC), cached per device together with the shared-memory attributes so
// that a launch issues nothing but the kernel.
template <bool kBatch>
static cudaError_t pair_limits_of(int *max_pairs) {
    static int cached[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (cached[dev] == 0) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, classify_tc2_kernel<kBatch>);
        if (e != cudaSuccess) return e;
        int optin = 0;
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) return e;
        const size_t lim = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
        e = cudaFuncSetAttribute(classify_tc2_kernel<kBatch>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * (unsigned)device_sm_count(), 1, 1);
        cfg.blockDim = dim3(kThreads, 1, 1);
        cfg.dynamicSmemBytes = lim;
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, classify_tc2_kernel<kBatch>, &cfg);
        if (e != cudaSuccess) return e;
        cached[dev] = n > 0 ? n : -1;
    }
    *max_pairs = cached[dev];
    return cudaSuccess;
}

bool tc2_available(int kpad) {
    if (!tc_supported() || kpad > 512 || kpad % 32 != 0) return false;
    int pairs = 0, pairs_b = 0;
    if (pair_limits_of<false>(&pairs) != cudaSuccess || pair_limits_of<true>(&pairs_b) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return pairs > 0 && pairs_b > 0 && pair_smem_plan(kpad, 1024).nstages >= 2;
}

// more than half of an SM's shared memory: one CTA per SM
static size_t pair_smem_bytes(const PairSmem &plan) { return plan.total > 122880u ? plan.total : 122880u; }

cudaError_t launch_classify_tc2(const ClassifyParams &p, cudaStream_t s) {
    if (p.tc_kpad > 512 || p.tc_kpad % 32 != 0) return cudaErrorNotSupported;
    int pairs = 0;
    cudaError_t e = pair_limits_of<false>(&pairs);
    if (e != cudaSuccess) return e;
    if (pairs <= 0) return cudaErrorNotSupported;
    const PairSmem plan = pair_smem_plan(p.tc_kpad, p.n * p.km1);
    if (plan.nstages < 2) return cudaErrorNotSupported;
    const int64_t npb = (p.N + 2 * kRows - 1) / (2 * kRows);
    const int64_t grid_pairs = std::min<int64_t>(npb, (int64_t)pairs);
    if (grid_pairs <= 0) return cudaSuccess;
    PairWork wk{};
    wk.kp_max = p.tc_kpad;
    wk.nthr_max = p.n * p.km1;
    classify_tc2_kernel<false><<<(unsigned)(2 * grid_pairs), kThreads, pair_smem_bytes(plan), s>>>(p, wk);
    return cudaGetLastError();
}

cudaError_t launch_classify_tc2_batch(const ClassifyParams *descs, const int64_t *begin, int S, int64_t total_items,
                                      const unsigned long long *round, int kp_max, int nthr_max, cudaStream_t s) {
    if (kp_max > 512 || kp_max % 32 != 0) return cudaErrorNotSupported;
    int pairs = 0;
    cudaError_t e = pair_limits_of<true>(&pairs);
    if (e != cudaSuccess) return e;
    if (pairs <= 0) return cudaErrorNotSupported;
    const PairSmem plan = pair_smem_plan(kp_max, nthr_max);
    if (plan.nstages < 2) return cudaErrorNotSupported;
    const int64_t grid_pairs = std::min<int64_t>(total_items, (int64_t)pairs);
    if (grid_pairs <= 0) return cudaSuccess;
    PairWork wk{descs, begin, round, S, kp_max, nthr_max, total_items};
    ClassifyParams none{};
    classify_tc2_kernel<true><<<(unsigned)(2 * grid_pairs), kThreads, pair_smem_bytes(plan), s>>>(none, wk);
    return cudaGetLastError();
}

}  // namespace rsr
