// batch.cu -- many classification problems (hazard scenarios) in one
// persistent launch.
//
// Each scenario s has its own n, K, pmf thresholds, reference sets, sample
// count N_s, seed and offset.  Work items are (scenario, 256-sample tile),
// enumerated scenario by scenario in the order the host chose (longest
// scenarios first); a persistent grid pulls items from an atomic counter, so
// short and long scenarios share the machine without per-scenario launch
// tails.  Per item the block runs the same bit-packed test as classify_popc.cu
// (Sec. 3.3, Algorithm 1) for the scenario's word count.  Counts go to the
// scenario's counts3; I^L per-bit counts go to a scenario scratch counter, and
// the last block to finish converts them into the per-state gradient counts,
// zeroes the scratch, resets the work counter and advances the round, so the
// same launch can be replayed (e.g. from a CUDA graph) on the next N_s samples
// of every scenario without any host work.  Scenarios whose upper set has a
// component-major index (popc_index.cuh) test their upper chunks through it,
// after a direct test of their kHot most probable upper references.
#include <cuda_runtime.h>

#include "popc_index.cuh"
#include "rsr_batch.h"
#include "rsr_internal.cuh"
#include "rsr_launch.h"

namespace rsr {

namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 256;
constexpr int kMaxWB = 16;  // batch path: n*(K-1) <= 512
constexpr int kCoopLanes = 16; // at most this many unresolved lanes: cooperative warp scan
constexpr int kHot = 16;        // upper references tried one by one before the index
constexpr int kCoopIdx = 1;     // at most this many lanes needing the index test: cooperative test
constexpr int kZeroLanes = 32;  // at most this many I^L lanes in a warp: count their zero bits (all: measured fastest)

struct Shared {
    BatchDesc d;
    int scenario;
    long long item;
    unsigned long long cnt[3];
    unsigned int fz;   // I^L samples of the item counted by their zero bits
    int last;
};

template <int WB>
__device__ void classify_item(const BatchDesc &d, int64_t tile, uint64_t round, const unsigned long long *s_thr,
                              uint32_t *s_tw, uint32_t *s_buf, uint32_t *s_cum, const uint32_t *s_hot,
                              const uint32_t *s_first, const uint32_t *s_zero, uint32_t *s_and, Shared &sh) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int64_t hl = tile * kThreads + tid;
    const bool valid = hl < d.N;
    const uint32_t key0 = (uint32_t)d.seed, key1 = (uint32_t)(d.seed >> 32);
    // chunk walk; chunk 0 is copied (cp.async) while the item is sampled.  Every
    // thread is past the item's set-up barrier, so both buffers are free.
    const bool overlap = *((volatile const int32_t *)d.overlap) != 0;
    const bool use_idx = d.popc_UT != nullptr;
    const int kenc = d.n * d.km1;
    const int64_t nU = (d.R_U + kChunk - 1) / kChunk, nL = (d.R_L + kChunk - 1) / kChunk;
    const int64_t nsteps = nU + nL;
    ChunkWalk walk(nU, nL, overlap, use_idx);
    bool upper = false;
    int64_t ci = 0;
    walk.next(&upper, &ci);   // nsteps >= 1: some reference exists
    auto chunk_refs = [&](bool up, int64_t c, int *cnt_out) {
        const int64_t R = up ? d.R_U : d.R_L;
        const int64_t base = c * kChunk;
        *cnt_out = (int)((R - base) < (int64_t)kChunk ? (R - base) : (int64_t)kChunk);
        return (up ? d.popc_U : d.popc_L) + base * WB;
    };
    auto issue = [&](int buf, bool up, int64_t c) {
        int cnt_c;
        const uint32_t *rows = chunk_refs(up, c, &cnt_c);
        const bool ix = use_idx && up;
        load_chunk_async<WB, kThreads>(s_buf + buf * (kChunk * kMaxWB), ix,
                                       ix ? d.popc_UT + (size_t)c * kIdxChunk * WB : nullptr, kenc,
                                       ix ? d.popc_UA + (size_t)c * WB : nullptr, s_and + buf * kMaxWB, rows, cnt_c,
                                       tid);
    };
    issue(0, upper, ci);
    // ---- sample and encode (thermometer words, one column per thread) ----
    if (d.km1 == 1) {
        // binary: 32-bit thresholds and never-bits (binary_tables_to_smem) in the s_thr region
        const uint32_t *s_t32 = reinterpret_cast<const uint32_t *>(s_thr);
        if (valid)
            sample_binary_words<WB, kThreads>(d.offset + round * (uint64_t)d.N + (uint64_t)hl, key0, key1, d.n,
                                              s_t32, s_t32 + 512, s_tw + tid);
        else
            for (int w = 0; w < WB; ++w) s_tw[w * kThreads + tid] = 0u;
    } else {
        uint32_t *col = s_tw + tid;
        int w = 0, pos = 0;
        uint32_t cur = 0;
        if (valid) {
            const uint64_t h = d.offset + round * (uint64_t)d.N + (uint64_t)hl;
            // two independent Philox blocks per iteration (instruction-level parallelism)
            for (int q = 0; 4 * q < d.n; q += 2) {
                const U32x4 ra = philox4x32_10((uint32_t)h, (uint32_t)(h >> 32), (uint32_t)q, 0u, key0, key1);
                const U32x4 rb = philox4x32_10((uint32_t)h, (uint32_t)(h >> 32), (uint32_t)(q + 1), 0u, key0, key1);
                const uint32_t us[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int i = 4 * q + c;
                    if (i >= d.n) break;
                    const uint32_t x = state_from_uniform(us[c], s_thr + (size_t)i * d.km1, d.km1);
                    const uint32_t bits = (1u << x) - 1u;
                    cur |= bits << pos;
                    const int np = pos + d.km1;
                    if (np >= 32) {
                        col[w * kThreads] = cur;
                        ++w;
                        cur = (np > 32) ? (bits >> (32 - pos)) : 0u;
                        pos = np - 32;
                    } else {
                        pos = np;
                    }
                }
            }
            if (pos > 0) {
                col[w * kThreads] = cur;
                ++w;
            }
        }
        for (; w < WB; ++w) col[w * kThreads] = 0u;
    }
    uint32_t t[WB];
#pragma unroll
    for (int w = 0; w < WB; ++w) t[w] = s_tw[w * kThreads + tid];

    bool mL = false, mU = false, done = !valid;
    // index mode: the most probable upper references first, one by one (not with an
    // overlapping pair, where every lower chunk has to come first)
    if (use_idx && !overlap && !done) {
        const int hotc = (int)(d.R_U < kHot ? d.R_U : kHot);
        for (int r = 0; r < hotc; ++r) {
            uint32_t acc = 0;
#pragma unroll
            for (int w = 0; w < WB; ++w) acc |= s_hot[r * WB + w] & ~t[w];
            if (acc == 0u) {
                mU = true;
                done = true;
                break;
            }
        }
    }
    for (int64_t step = 0; step < nsteps; ++step) {
        cp_async_wait_all();                       // this thread's copies of chunk `step`
        if (__syncthreads_and(done)) break;        // chunk `step` visible; chunk step-1 consumed
        const int cur_buf = (int)(step & 1);
        uint32_t *s_ref = s_buf + cur_buf * (kChunk * kMaxWB);
        int cnt;
        (void)chunk_refs(upper, ci, &cnt);
        const bool idx_chunk = use_idx && upper;
        bool up_next = false;
        int64_t ci_next = 0;
        if (step + 1 < nsteps) {
            walk.next(&up_next, &ci_next);
            issue((int)((step + 1) & 1), up_next, ci_next);
        }
        // per-lane scan while many lanes are unresolved, cooperative warp scan otherwise
        const unsigned active = __ballot_sync(0xffffffffu, !done);
        if (idx_chunk) {
            // a sample lacking a bit of the chunk's AND row dominates none of its references
            const bool ruled = !done && chunk_ruled_out<WB>(t, s_and + cur_buf * kMaxWB);
            const unsigned need = __ballot_sync(0xffffffffu, !done && !ruled);
            if (__popc(need) > kCoopIdx) {
                if (!done && !ruled && idx_match_lane<WB>(t, s_ref, s_first, s_zero, kenc, cnt)) {
                    mU = true;
                    done = true;
                }
            } else {
                unsigned rem = need;
                while (rem) {
                    const int src = __ffs(rem) - 1;
                    rem &= rem - 1;
                    const bool found =
                        idx_match_warp<WB, kThreads>(s_tw + (tid - lane + src), s_ref, s_first, kenc, cnt, lane);
                    if (lane == src && found) {
                        mU = true;
                        done = true;
                    }
                }
                __syncwarp();  // the columns read above are rewritten by their lanes for the next item
            }
        } else if (__popc(active) > kCoopLanes) {
            if (!done) {
                bool m = false;
                if (upper) {
                    for (int r = 0; r < cnt; ++r) {
                        uint32_t acc = 0;
#pragma unroll
                        for (int w = 0; w < WB; ++w) acc |= s_ref[r * WB + w] & ~t[w];
                        if (acc == 0u) { m = true; break; }
                    }
                } else {
                    for (int r = 0; r < cnt; ++r) {
                        uint32_t acc = 0;
#pragma unroll
                        for (int w = 0; w < WB; ++w) acc |= t[w] & s_ref[r * WB + w];
                        if (acc == 0u) { m = true; break; }
                    }
                }
                if (m) {
                    if (upper) mU = true; else mL = true;
                    done = true;
                }
            }
        } else {
            unsigned rem = active;
            while (rem) {
                const int src = __ffs(rem) - 1;
                rem &= rem - 1;
                uint32_t ts[WB];
#pragma unroll
                for (int w = 0; w < WB; ++w) ts[w] = __shfl_sync(0xffffffffu, t[w], src);
                bool found = false;
                for (int r0 = 0; r0 < cnt && !found; r0 += 32) {
                    const int r = r0 + lane;
                    bool m = false;
                    if (r < cnt) {
                        uint32_t acc = 0;
                        if (upper) {
#pragma unroll
                            for (int w = 0; w < WB; ++w) acc |= s_ref[r * WB + w] & ~ts[w];
                        } else {
#pragma unroll
                            for (int w = 0; w < WB; ++w) acc |= ts[w] & s_ref[r * WB + w];
                        }
                        m = (acc == 0u);
                    }
                    found = __any_sync(0xffffffffu, m);
                }
                if (lane == src && found) {
                    if (upper) mU = true; else mL = true;
                    done = true;
                }
            }
        }
        upper = up_next;
        ci = ci_next;
    }
    const int label = mL ? 0 : (mU ? 1 : 2);
    if (valid && d.labels) d.labels[hl] = (uint8_t)label;
    // counts
    const unsigned b0 = __ballot_sync(0xffffffffu, valid && label == 0);
    const unsigned b1 = __ballot_sync(0xffffffffu, valid && label == 1);
    const unsigned b2 = __ballot_sync(0xffffffffu, valid && label == 2);
    if (lane == 0) {
        if (b0) atomicAdd(&sh.cnt[0], (unsigned long long)__popc(b0));
        if (b1) atomicAdd(&sh.cnt[1], (unsigned long long)__popc(b1));
        if (b2) atomicAdd(&sh.cnt[2], (unsigned long long)__popc(b2));
    }
    // per-bit counts of I^L samples: zero bits with shared atomics for a warp with
    // at most kZeroLanes I^L samples (every warp at 32), 32 ballots per word (one
    // bits) otherwise
    if (d.bitcnt && b0 && __popc(b0) <= kZeroLanes) {
        if (valid && label == 0) {
            const int kenc = d.n * d.km1;
#pragma unroll
            for (int w = 0; w < WB; ++w) {
                uint32_t z = ~t[w] & enc_valid_bits(kenc, w);
                while (z) {
                    const int b = __ffs(z) - 1;
                    z &= z - 1u;
                    atomicSub(&s_cum[w * 32 + b], 1u);   // ones = (zero-route samples) - zeros
                }
            }
        }
        if (lane == 0) atomicAdd(&sh.fz, (unsigned)__popc(b0));
    } else if (d.bitcnt && b0) {
        const bool isL = valid && label == 0;
#pragma unroll
        for (int w = 0; w < WB; ++w) {
            const uint32_t tw = isL ? t[w] : 0u;
            uint32_t mine = 0;
#pragma unroll 4
            for (int b = 0; b < 32; ++b) {
                const uint32_t m = __ballot_sync(0xffffffffu, (tw >> b) & 1u);
                if (lane == b) mine = __popc(m);
            }
            if (mine) atomicAdd(&s_cum[w * 32 + lane], mine);
        }
    }
}

__global__ void __launch_bounds__(kThreads, 4) batch_kernel(const BatchDesc *__restrict__ descs,
                                                             const int64_t *__restrict__ item_begin, int S,
                                                             int64_t total_items, BatchHeader *hdr) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared sh;
    __shared__ __align__(16) uint32_t s_zero[kIdxWords];
    __shared__ uint32_t s_and[2 * kMaxWB];   // AND rows of the staged index chunks
    const int tid = threadIdx.x;
    unsigned long long *s_thr = reinterpret_cast<unsigned long long *>(smem);        // [512]
    uint32_t *s_tw = reinterpret_cast<uint32_t *>(smem + 512 * 8);                     // [kMaxWB][256]
    uint32_t *s_buf = s_tw + kMaxWB * kThreads;                                         // [2][kChunk * kMaxWB]
    uint32_t *s_cum = s_buf + 2 * kChunk * kMaxWB;                                      // [kMaxWB * 32]
    uint32_t *s_hot = s_cum + kMaxWB * 32;                                              // [kHot * kMaxWB]
    uint32_t *s_first = s_hot + kHot * kMaxWB;                                          // [kMaxWB]
    const uint64_t round = *((volatile unsigned long long *)&hdr->round);
    if (tid == 0) sh.scenario = -1;
    if (tid < kIdxWords) s_zero[tid] = 0u;
    __syncthreads();
    while (true) {
        if (tid == 0) sh.item = (long long)atomicAdd(&hdr->next_item, 1ull);
        __syncthreads();
        const long long item = sh.item;
        if (item >= total_items) break;
        // scenario of this item: last s with item_begin[s] <= item
        if (tid == 0) {
            int lo = 0, hi = S - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (item_begin[mid] <= item) lo = mid; else hi = mid - 1;
            }
            if (lo != sh.scenario) {
                sh.scenario = lo;
                sh.d = descs[lo];
            }
            sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0ull;
            sh.fz = 0u;
        }
        __syncthreads();
        const BatchDesc &d = sh.d;
        const int nthr = d.n * d.km1;
        if (d.km1 == 1) {
            uint32_t *s_t32 = reinterpret_cast<uint32_t *>(s_thr);   // [512] + never-words [16]
            binary_tables_to_smem(d.thr, d.n, s_t32, s_t32 + 512, tid, kThreads);
        } else {
            for (int i = tid; i < nthr; i += kThreads) s_thr[i] = d.thr[i];
        }
        for (int j = tid; j < d.words_b * 32; j += kThreads) s_cum[j] = 0u;
        if (d.popc_UT) {
            const int hotw = (int)(d.R_U < kHot ? d.R_U : kHot) * d.words_b;
            for (int i = tid; i < hotw; i += kThreads) s_hot[i] = d.popc_U[i];
            for (int w = tid; w < d.words_b; w += kThreads) s_first[w] = component_first_bits(d.km1, nthr, w);
        }
        __syncthreads();
        const int64_t tile = item - item_begin[sh.scenario];
        switch (d.words_b) {
            case 1: classify_item<1>(d, tile, round, s_thr, s_tw, s_buf, s_cum, s_hot, s_first, s_zero, s_and, sh); break;
            case 2: classify_item<2>(d, tile, round, s_thr, s_tw, s_buf, s_cum, s_hot, s_first, s_zero, s_and, sh); break;
            case 4: classify_item<4>(d, tile, round, s_thr, s_tw, s_buf, s_cum, s_hot, s_first, s_zero, s_and, sh); break;
            case 6: classify_item<6>(d, tile, round, s_thr, s_tw, s_buf, s_cum, s_hot, s_first, s_zero, s_and, sh); break;
            case 8: classify_item<8>(d, tile, round, s_thr, s_tw, s_buf, s_cum, s_hot, s_first, s_zero, s_and, sh); break;
            case 10: classify_item<10>(d, tile, round, s_thr, s_tw, s_buf, s_cum, s_hot, s_first, s_zero, s_and, sh); break;
            case 12: classify_item<12>(d, tile, round, s_thr, s_tw, s_buf, s_cum, s_hot, s_first, s_zero, s_and, sh); break;
            default: classify_item<16>(d, tile, round, s_thr, s_tw, s_buf, s_cum, s_hot, s_first, s_zero, s_and, sh); break;
        }
        __syncthreads();
        if (tid < 3 && sh.cnt[tid]) atomicAdd(&d.counts3[tid], sh.cnt[tid]);
        if (d.bitcnt && sh.cnt[0]) {
            if (tid == 0) atomicAdd(d.lcount, sh.cnt[0]);
            for (int j = tid; j < nthr; j += kThreads) {
                const uint32_t ones = s_cum[j] + sh.fz;   // one bits of the item's I^L samples (mod 2^32)
                if (ones) atomicAdd(&d.bitcnt[j], ones);
            }
        }
        __syncthreads();
    }
    // ---- the last block converts bit counts to per-state counts and re-arms ----
    __threadfence();
    __syncthreads();
    if (tid == 0) sh.last = (atomicAdd(&hdr->blocks_done, 1u) == gridDim.x - 1) ? 1 : 0;
    __syncthreads();
    if (!sh.last) return;
    __threadfence();
    for (int s = 0; s < S; ++s) {
        const BatchDesc &d = descs[s];
        if (!d.bitcnt) continue;
        const unsigned long long F = *((volatile unsigned long long *)d.lcount);
        if (F) {
            for (int i = tid; i < d.n; i += kThreads) {
                long long prev = (long long)F;
                for (int k = 1; k <= d.km1; ++k) {
                    const long long cum = (long long)((volatile uint32_t *)d.bitcnt)[i * d.km1 + (k - 1)];
                    const long long delta = prev - cum;
                    if (delta) atomicAdd(&d.grad_counts[(size_t)i * d.K + (k - 1)], (unsigned long long)delta);
                    prev = cum;
                }
                if (prev) atomicAdd(&d.grad_counts[(size_t)i * d.K + d.km1], (unsigned long long)prev);
            }
        }
        __syncthreads();
        for (int j = tid; j < d.n * d.km1; j += kThreads) d.bitcnt[j] = 0u;
        if (tid == 0) *d.lcount = 0ull;
    }
    if (tid == 0) {
        hdr->next_item = 0ull;
        hdr->blocks_done = 0u;
        hdr->round = round + 1ull;
    }
}

}  // namespace

size_t batch_kernel_smem() {
    return 512 * 8 + sizeof(uint32_t) * ((size_t)kMaxWB * kThreads + 2 * (size_t)kChunk * kMaxWB + (size_t)kMaxWB * 32 +
                                         (size_t)kHot * kMaxWB + (size_t)kMaxWB);
}

int batch_max_words() { return kMaxWB; }

cudaError_t batch_max_grid(int *blocks_per_sm) {
    const size_t smem = batch_kernel_smem();
    cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, batch_kernel, kThreads, smem);
}

// The shared-memory attribute is set by batch_max_grid() (called when a batch
// is prepared), so a launch issues nothing but the kernel and can be captured.
cudaError_t launch_batch(const BatchDesc *descs, const int64_t *item_begin, int S, int64_t total_items,
                         BatchHeader *hdr, int grid, cudaStream_t s) {
    const size_t smem = batch_kernel_smem();
    if (grid <= 0 || total_items <= 0) return cudaSuccess;
    batch_kernel<<<grid, kThreads, smem, s>>>(descs, item_begin, S, total_items, hdr);
    return cudaGetLastError();
}

}  // namespace rsr
