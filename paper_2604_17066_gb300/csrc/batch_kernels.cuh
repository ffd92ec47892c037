// batch_kernels.cuh -- the batched persistent kernels (see batch.cu for the
// scheme), as templates in an unnamed namespace: batch.cu instantiates them
// without the cycle profile (kProf = false) and batch_prof.cu with it, so the
// two variants compile in parallel and the plain kernels keep their code.
#pragma once

#include <algorithm>

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
    int changed;                 // the item's scenario differs from the block's previous one
    long long deep_pos;          // the item's reservation in its scenario's deep queue
    unsigned int warp_pend[kThreads / 32];
    long long tile;                          // the tile (first pass) or queued group (later stage) run now
    int left;                                // the item's tiles still to run after this one
    int fresh;                               // this tile starts an item (counts and bit counts zeroed)
    long long t_start, t_ready, t_sampled;   // cycle profile marks: tile start, tables ready, warp 0's samples written
};

// The multi-state sampler as a call: inlined, its registers would add to the
// walk's in this one kernel for every scenario (spills 180 -> 400 bytes in
// batch_kernel); called, it keeps its own (224 bytes).
template <int WB>
__device__ __noinline__ void sample_multi_call(uint64_t h, uint32_t key0, uint32_t key1, int n, int km1,
                                               const uint32_t *s_t32k, uint32_t *col) {
    sample_multi_words_k<WB, kThreads, 0>(h, key0, key1, n, km1, s_t32k, col);   // level loop at run time: fewer spills here
}

// One item.  First pass (deep == nullptr): samples tile*256 + tid.  A later
// stage: the sample whose local index is deep[tid] (none if tid >= n_deep or
// the entry is negative).  Chunk steps [step0, lim); the samples still
// unresolved at lim go to queue q_sel (0 or 1; -1: lim is the end).  kProf:
// thread 0 marks the time warp 0's samples are written (sh.t_sampled).
template <int WB, bool kProf>
__device__ void classify_item(const BatchDesc &d, int64_t tile, const int64_t *deep, int n_deep, int step0_in,
                              int lim_in, int q_sel, uint64_t round,
                              const unsigned long long *s_thr, uint32_t *s_tw, uint32_t *s_buf, uint32_t *s_cum,
                              const uint32_t *s_hot, const uint32_t *s_first, const uint32_t *s_zero,
                              uint32_t *s_and, Shared &sh) {
    const int tid = threadIdx.x, lane = tid & 31;
    const bool second = deep != nullptr;
    int64_t hl;
    if (second) hl = tid < n_deep ? deep[tid] : -1;
    else hl = tile * kThreads + tid;
    const bool valid = hl >= 0 && hl < d.N;
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
    // steps [step0, lim): a later stage replays the walk up to its first step
    const int64_t step0 = step0_in;
    int64_t lim = lim_in;
    for (int64_t i = 0; i < step0; ++i) walk.next(&upper, &ci);
    walk.next(&upper, &ci);   // step0 < nsteps: some reference exists, and a later stage only runs below nsteps
    auto chunk_refs = [&](bool up, int64_t c, int *cnt_out) {
        const int64_t R = up ? d.R_U : d.R_L;
        const int64_t base = c * kChunk;
        *cnt_out = (int)((R - base) < (int64_t)kChunk ? (R - base) : (int64_t)kChunk);
        return (up ? d.popc_U : d.popc_L) + base * WB;
    };
    const bool use_lg = d.popc_LG != nullptr;
    auto issue = [&](int buf, bool up, int64_t c) {
        int cnt_c;
        const uint32_t *rows = chunk_refs(up, c, &cnt_c);
        const bool ix = use_idx && up, lg = use_lg && !up;
        const uint32_t *skip = ix ? d.popc_UA + (size_t)c * WB : (lg ? d.popc_LG + (size_t)c * 2 * WB : nullptr);
        load_chunk_async<WB, kThreads>(s_buf + buf * (kChunk * kMaxWB), ix,
                                       ix ? d.popc_UT + (size_t)c * kIdxChunk * WB : nullptr, kenc, skip,
                                       ix ? WB : 2 * WB, s_and + buf * 2 * kMaxWB, rows, cnt_c, tid);
    };
    issue((int)(step0 & 1), upper, ci);
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
        // multi-state: 32-bit tables and never words (multi_tables_to_smem) in the s_thr region
        const uint32_t *s_t32k = reinterpret_cast<const uint32_t *>(s_thr);
        if (valid)
            sample_multi_call<WB>(d.offset + round * (uint64_t)d.N + (uint64_t)hl, key0, key1, d.n, d.km1, s_t32k,
                                  s_tw + tid);
        else
            for (int w = 0; w < WB; ++w) s_tw[w * kThreads + tid] = 0u;
    }
    if (kProf && tid == 0) sh.t_sampled = clock64();
    uint32_t t[WB];
#pragma unroll
    for (int w = 0; w < WB; ++w) t[w] = s_tw[w * kThreads + tid];

    bool mL = false, mU = false, done = !valid, deferred = false;
    // index mode: the most probable upper references first, one by one (not with an
    // overlapping pair, where every lower chunk has to come first); first pass only
    if (!second && use_idx && !overlap && !done) {
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
    for (int64_t step = step0; step < nsteps; ++step) {
        cp_async_wait_all();                       // this thread's copies of chunk `step`
        if (__syncthreads_and(done)) break;        // chunk `step` visible; chunk step-1 consumed
        if (step == lim) {
            // The stage's steps are spent: queue the unresolved samples for the next stage.
            // (An unresolved sample has no match so far: with an overlapping pair a lower
            // match is final and upper chunks only follow the lower ones.)
            const bool pend = !done;
            const unsigned wb = __ballot_sync(0xffffffffu, pend);
            if (lane == 0) sh.warp_pend[tid >> 5] = (unsigned)__popc(wb);
            __syncthreads();
            int before = 0, total = 0;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) {
                const int c = (int)sh.warp_pend[w];
                before += (w < (tid >> 5)) ? c : 0;
                total += c;
            }
            int64_t *q_out = d.deep + (size_t)q_sel * d.deep_cap;
            if (tid == 0) sh.deep_pos = (long long)atomicAdd(d.deep_count + q_sel, (unsigned long long)total);
            __syncthreads();
            const long long pos = sh.deep_pos;
            if (pos + total <= (long long)d.deep_cap) {
                if (pend) {
                    q_out[pos + before + __popc(wb & ((1u << lane) - 1u))] = hl;
                    deferred = true;
                }
                break;
            }
            // the queue is full: void this reservation's slots below the capacity and walk on here
            for (long long k = tid; k < total && pos + k < (long long)d.deep_cap; k += kThreads) q_out[pos + k] = -1;
            lim = nsteps;
        }
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
        // per-lane scan while many lanes are unresolved, cooperative warp scan otherwise;
        // in a lower chunk only the lanes its skip rows do not rule out
        const bool skip = !done && !upper && use_lg && lower_chunk_ruled_out<WB>(t, s_and + cur_buf * 2 * kMaxWB);
        const unsigned active = __ballot_sync(0xffffffffu, !done && !skip);
        if (idx_chunk) {
            // a sample lacking a bit of the chunk's AND row dominates none of its references
            const bool ruled = !done && chunk_ruled_out<WB>(t, s_and + cur_buf * 2 * kMaxWB);
            const unsigned need = __ballot_sync(0xffffffffu, !done && !ruled);
            if (__popc(need) > kCoopIdx) {
                unsigned long long ops_unused = 0;
                if (!done && !ruled && idx_match_lane<WB>(t, s_ref, s_first, s_zero, kenc, cnt, &ops_unused)) {
                    mU = true;
                    done = true;
                }
            } else {
                unsigned rem = need;
                while (rem) {
                    const int src = __ffs(rem) - 1;
                    rem &= rem - 1;
                    unsigned long long ops_unused = 0;
                    const bool found = idx_match_warp<WB, kThreads>(s_tw + (tid - lane + src), s_ref, s_first, kenc,
                                                                    cnt, lane, &ops_unused);
                    if (lane == src && found) {
                        mU = true;
                        done = true;
                    }
                }
                __syncwarp();  // the columns read above are rewritten by their lanes for the next item
            }
        } else if (__popc(active) > kCoopLanes) {
            if (!done && !skip) {
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
    cp_async_wait_all();   // the copy of a chunk that a finished walk did not reach
    const bool final_ = valid && !deferred;   // resolved here (a deferred sample is counted by a later stage)
    const int label = mL ? 0 : (mU ? 1 : 2);
    if (final_ && d.labels) d.labels[hl] = (uint8_t)label;
    // counts
    const unsigned b0 = __ballot_sync(0xffffffffu, final_ && label == 0);
    const unsigned b1 = __ballot_sync(0xffffffffu, final_ && label == 1);
    const unsigned b2 = __ballot_sync(0xffffffffu, final_ && label == 2);
    if (lane == 0) {
        if (b0) atomicAdd(&sh.cnt[0], (unsigned long long)__popc(b0));
        if (b1) atomicAdd(&sh.cnt[1], (unsigned long long)__popc(b1));
        if (b2) atomicAdd(&sh.cnt[2], (unsigned long long)__popc(b2));
    }
    // per-bit counts of I^L samples: zero bits with shared atomics for a warp with
    // at most kZeroLanes I^L samples (every warp at 32), 32 ballots per word (one
    // bits) otherwise
    if (d.bitcnt && b0 && __popc(b0) <= kZeroLanes) {
        if (final_ && label == 0) {
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
        const bool isL = final_ && label == 0;
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

// Shared-memory carve-up of every pass.
struct BatchSmem {
    unsigned long long *thr;   // [512] thresholds (or 32-bit binary tables and never-words)
    uint32_t *tw, *buf, *cum, *hot, *first;
};

__device__ __forceinline__ BatchSmem batch_smem(unsigned char *smem) {
    BatchSmem m;
    m.thr = reinterpret_cast<unsigned long long *>(smem);          // [512]
    m.tw = reinterpret_cast<uint32_t *>(smem + 512 * 8);            // [kMaxWB][256]
    m.buf = m.tw + kMaxWB * kThreads;                               // [2][kChunk * kMaxWB]
    m.cum = m.buf + 2 * kChunk * kMaxWB;                            // [kMaxWB * 32]
    m.hot = m.cum + kMaxWB * 32;                                    // [kHot * kMaxWB]
    m.first = m.hot + kHot * kMaxWB;                                // [kMaxWB]
    return m;
}

// The chunk steps of stage `stage` of a scenario (0: the first pass): the first
// pass walks [0, k0) (everything if k0 = 0), each later stage from where the
// previous one stopped to next_stage_end() (d.staged) or to the end; empty
// (lo = nsteps) once done.
__device__ __forceinline__ void stage_steps(const BatchDesc &d, int stage, int64_t *lo, int64_t *hi) {
    const int64_t nsteps = (d.R_U + kChunk - 1) / kChunk + (d.R_L + kChunk - 1) / kChunk;
    int64_t a = 0, b = (d.k0 > 0 && (int64_t)d.k0 < nsteps) ? (int64_t)d.k0 : nsteps;
    for (int st = 0; st < stage; ++st) {
        a = b;
        b = (b >= nsteps || !d.staged) ? nsteps : next_stage_end(b, nsteps);
    }
    *lo = a;
    *hi = b;
}

// The persistent item loop of one pass: items [begin[s], begin[s+1]) belong to
// scenario s.  A first-pass item is d.tiles consecutive 256-sample tiles of
// its scenario (one work-counter atomic, scenario lookup, table load and count
// flush for all of them); a later-stage item is one group of 256 queued
// samples.  The loop runs one tile per iteration and keeps its state (item,
// tile, tiles left) in shared memory, so nothing of it is live across the
// chunk walk.  With a cycle profile (prof: [S][8]), thread 0 adds to its
// scenario's row, at [0] for the first pass and [4] for a later stage: tiles
// (groups), then SM cycles from a tile's start to its tables being ready (work
// counter, scenario lookup, table loads), from there to warp 0's samples being
// written (sampling), and from there to the tile's end (the chunk walk; an
// item's last tile includes its count flush).
template <bool kSecond, bool kProf>
__device__ void item_loop(const BatchDesc *__restrict__ descs, const int64_t *__restrict__ begin, int S,
                          int64_t total_items, unsigned long long *counter, uint64_t round, int stage,
                          const BatchSmem &m, const uint32_t *s_zero, uint32_t *s_and, Shared &sh,
                          unsigned long long *prof) {
    const int tid = threadIdx.x;
    if (tid == 0) sh.left = 0;
    while (true) {
        if (kProf && tid == 0) sh.t_start = clock64();
        if (tid == 0 && sh.left == 0) sh.item = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long item = sh.item;
        if (item >= total_items) break;
        if (tid == 0) {
            const int fresh = sh.left == 0;
            if (fresh) {
                // scenario of this item: last s with begin[s] <= item
                int lo = 0, hi = S - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (begin[mid] <= item) lo = mid; else hi = mid - 1;
                }
                sh.changed = lo != sh.scenario;
                if (sh.changed) {
                    sh.scenario = lo;
                    sh.d = descs[lo];
                }
                sh.cnt[0] = sh.cnt[1] = sh.cnt[2] = 0ull;
                sh.fz = 0u;
                const int64_t k = item - begin[lo];
                if (kSecond) {
                    sh.tile = k;
                    sh.left = 1;
                } else {
                    const int64_t ntiles = (sh.d.N + kThreads - 1) / kThreads;
                    const int tiles = sh.d.tiles > 1 ? sh.d.tiles : 1;   // the host writes >= 1
                    sh.tile = k * tiles;
                    sh.left = (int)min((int64_t)tiles, ntiles - (int64_t)sh.tile);
                }
            } else {
                sh.changed = 0;
                sh.tile += 1;
            }
            sh.fresh = fresh;
            sh.left -= 1;
        }
        __syncthreads();
        const BatchDesc &d = sh.d;
        const int nthr = d.n * d.km1;
        // the scenario's tables stay in shared memory while the block's items stay in it
        // (items only read them)
        if (sh.changed) {
            if (d.km1 == 1) {
                uint32_t *s_t32 = reinterpret_cast<uint32_t *>(m.thr);   // [512] + never-words [16]
                binary_tables_to_smem(d.thr, d.n, s_t32, s_t32 + 512, tid, kThreads);
            } else {
                // 32-bit tables: at most 512 + 7 * 15 + 16 words of the 1024 in the region
                multi_tables_to_smem(d.thr, d.n, d.km1, reinterpret_cast<uint32_t *>(m.thr), tid, kThreads);
            }
            if (d.popc_UT) {
                const int hotw = (int)(d.R_U < kHot ? d.R_U : kHot) * d.words_b;
                for (int i = tid; i < hotw; i += kThreads) m.hot[i] = d.popc_U[i];
                for (int w = tid; w < d.words_b; w += kThreads) m.first[w] = component_first_bits(d.km1, nthr, w);
            }
        }
        if (sh.fresh)
            for (int j = tid; j < d.words_b * 32; j += kThreads) m.cum[j] = 0u;
        __syncthreads();
        if (kProf && tid == 0) sh.t_ready = clock64();
        const int64_t k = sh.tile;   // tile, or group of queued samples
        const int64_t *deep = nullptr;
        int n_deep = 0;
        if (kSecond) {
            // this stage reads the queue the previous one filled
            const int q_in = (stage - 1) & 1;
            const int64_t queued = (int64_t)min(*((volatile unsigned long long *)(d.deep_count + q_in)),
                                                (unsigned long long)d.deep_cap);
            deep = d.deep + (size_t)q_in * d.deep_cap + k * kThreads;
            n_deep = (int)min((int64_t)kThreads, queued - k * kThreads);
        }
        int64_t step_lo, step_hi;
        stage_steps(d, stage, &step_lo, &step_hi);
        const int64_t nsteps_d = (d.R_U + kChunk - 1) / kChunk + (d.R_L + kChunk - 1) / kChunk;
        // chunk steps stay below 2^24 (R < 2^31): 32 bits carry them
        const int step0 = kSecond ? (int)(step_lo < nsteps_d ? step_lo : nsteps_d) : 0;
        const int q_sel = step_hi < nsteps_d ? (stage & 1) : -1;
        const int lim = (int)(q_sel >= 0 ? step_hi : nsteps_d);
#define RSR_ITEM(WBV)                                                                                           \
    classify_item<WBV, kProf>(d, k, deep, n_deep, step0, lim, q_sel, round, m.thr, m.tw, m.buf, m.cum, m.hot, \
                              m.first, s_zero, s_and, sh)
        switch (d.words_b) {
            case 1: RSR_ITEM(1); break;
            case 2: RSR_ITEM(2); break;
            case 4: RSR_ITEM(4); break;
            case 6: RSR_ITEM(6); break;
            case 8: RSR_ITEM(8); break;
            case 10: RSR_ITEM(10); break;
            case 12: RSR_ITEM(12); break;
            default: RSR_ITEM(16); break;
        }
#undef RSR_ITEM
        __syncthreads();
        if (sh.left == 0) {   // the item's last tile: flush its counts
            if (tid < 3 && sh.cnt[tid]) atomicAdd(&d.counts3[tid], sh.cnt[tid]);
            if (d.bitcnt && sh.cnt[0]) {
                if (tid == 0) atomicAdd(d.lcount, sh.cnt[0]);
                for (int j = tid; j < nthr; j += kThreads) {
                    const uint32_t ones = m.cum[j] + sh.fz;   // one bits of the item's I^L samples (mod 2^32)
                    if (ones) atomicAdd(&d.bitcnt[j], ones);
                }
            }
        }
        __syncthreads();
        if (kProf && tid == 0) {
            const long long t_end = clock64();
            unsigned long long *row = prof + (size_t)sh.d.id * 8 + (kSecond ? 4 : 0);
            atomicAdd(row + 0, 1ull);
            atomicAdd(row + 1, (unsigned long long)(sh.t_ready - sh.t_start));
            atomicAdd(row + 2, (unsigned long long)(sh.t_sampled - sh.t_ready));
            atomicAdd(row + 3, (unsigned long long)(t_end - sh.t_sampled));
        }
    }
}

// True in exactly one thread block, the last of the grid to get here (its
// threads see every other block's writes).
__device__ __forceinline__ bool last_block(unsigned int *done_counter, Shared &sh) {
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh.last = (atomicAdd(done_counter, 1u) == gridDim.x - 1) ? 1 : 0;
    __syncthreads();
    if (!sh.last) return false;
    __threadfence();
    return true;
}

// Items of the next stage (groups of 256 queued samples per scenario) from the
// counts of queue q; one thread.
__device__ void lay_out_stage(const BatchDesc *descs, int S, int q, int64_t *deep_begin, BatchHeader *hdr) {
    int64_t acc = 0;
    for (int s = 0; s < S; ++s) {
        deep_begin[s] = acc;
        const unsigned long long c = *((volatile unsigned long long *)(descs[s].deep_count + q));
        const int64_t queued = (int64_t)(c < (unsigned long long)descs[s].deep_cap ? c : descs[s].deep_cap);
        acc += (queued + kThreads - 1) / kThreads;
    }
    deep_begin[S] = acc;
    hdr->deep_total = acc;
}

// First pass (stage 0).  Its last block lays out stage 1's items and re-arms the
// first pass's counters.
template <bool kProf>
__global__ void __launch_bounds__(kThreads, 4) batch_kernel(const BatchDesc *__restrict__ descs,
                                                             const int64_t *__restrict__ item_begin, int S,
                                                             int64_t total_items, BatchHeader *hdr,
                                                             int64_t *deep_begin, unsigned long long *prof) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared sh;
    __shared__ __align__(16) uint32_t s_zero[kIdxWords];
    __shared__ uint32_t s_and[4 * kMaxWB];   // skip rows of the two staged chunks (AND row, guard row)
    const int tid = threadIdx.x;
    const BatchSmem m = batch_smem(smem);
    const uint64_t round = *((volatile unsigned long long *)&hdr->round);
    if (tid == 0) sh.scenario = -1;
    if (tid < kIdxWords) s_zero[tid] = 0u;
    __syncthreads();
    item_loop<false, kProf>(descs, item_begin, S, total_items, &hdr->next_item, round, 0, m, s_zero, s_and, sh, prof);
    if (!last_block(&hdr->blocks_done, sh)) return;
    if (tid == 0) {
        lay_out_stage(descs, S, 0, deep_begin, hdr);
        hdr->next_item = 0ull;
        hdr->blocks_done = 0u;
        __threadfence();
    }
}

// Stage `stage` >= 1 over the queued samples (queue (stage-1) & 1, filling
// queue stage & 1).  Its last block clears the count of the queue it read; then
// it lays out the next stage's items, or, in the last stage (final != 0),
// converts the I^L bit counts to per-state gradient counts, zeroes the scratch
// and both queue counts, re-arms the counters and advances the round.
template <bool kProf>
__global__ void __launch_bounds__(kThreads, 4) batch_deep_kernel(const BatchDesc *__restrict__ descs,
                                                                  int64_t *deep_begin, int S, BatchHeader *hdr,
                                                                  int stage, int final, unsigned long long *prof) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Shared sh;
    __shared__ __align__(16) uint32_t s_zero[kIdxWords];
    __shared__ uint32_t s_and[4 * kMaxWB];
    const int tid = threadIdx.x;
    const BatchSmem m = batch_smem(smem);
    const uint64_t round = *((volatile unsigned long long *)&hdr->round);
    const int64_t total = *((volatile long long *)&hdr->deep_total);
    if (tid == 0) sh.scenario = -1;
    if (tid < kIdxWords) s_zero[tid] = 0u;
    __syncthreads();
    item_loop<true, kProf>(descs, deep_begin, S, total, &hdr->next_deep, round, stage, m, s_zero, s_and, sh, prof);
    if (!last_block(&hdr->blocks_done2, sh)) return;
    if (!final) {
        if (tid == 0) {
            for (int s = 0; s < S; ++s) descs[s].deep_count[(stage - 1) & 1] = 0ull;   // read by this stage
            lay_out_stage(descs, S, stage & 1, deep_begin, hdr);
            hdr->next_deep = 0ull;
            hdr->blocks_done2 = 0u;
            __threadfence();
        }
        return;
    }
    for (int s = 0; s < S; ++s) {
        const BatchDesc &d = descs[s];
        if (d.bitcnt) {
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
        if (tid == 0) d.deep_count[0] = d.deep_count[1] = 0ull;
    }
    if (tid == 0) {
        hdr->next_deep = 0ull;
        hdr->blocks_done2 = 0u;
        hdr->round = round + 1ull;
    }
}

inline size_t batch_smem_bytes() {
    return 512 * 8 + sizeof(uint32_t) * ((size_t)kMaxWB * kThreads + 2 * (size_t)kChunk * kMaxWB + (size_t)kMaxWB * 32 +
                                         (size_t)kHot * kMaxWB + (size_t)kMaxWB);
}

// One variant's shared-memory attributes; *blocks_per_sm = min(its occupancy, *blocks_per_sm).
template <bool kProf>
cudaError_t batch_variant_attributes(int *blocks_per_sm) {
    const size_t smem = batch_smem_bytes();
    const void *kernels[2] = {(const void *)batch_kernel<kProf>, (const void *)batch_deep_kernel<kProf>};
    for (const void *f : kernels) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int a = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, f, kThreads, smem);
        if (e != cudaSuccess) return e;
        if (a < *blocks_per_sm) *blocks_per_sm = a;
    }
    return cudaSuccess;
}

// One variant's launches: the tile pass, then n_stages later stages (the last closes the round).
template <bool kProf>
cudaError_t batch_variant_launch(const BatchDesc *descs, const int64_t *item_begin, int S, int64_t total_items,
                                 BatchHeader *hdr, int64_t *deep_begin, int n_stages, int grid, cudaStream_t s,
                                 unsigned long long *prof) {
    const size_t smem = batch_smem_bytes();
    batch_kernel<kProf><<<grid, kThreads, smem, s>>>(descs, item_begin, S, total_items, hdr, deep_begin, prof);
    cudaError_t e = cudaGetLastError();
    for (int st = 1; st <= n_stages && e == cudaSuccess; ++st) {
        batch_deep_kernel<kProf><<<grid, kThreads, smem, s>>>(descs, deep_begin, S, hdr, st, st == n_stages ? 1 : 0,
                                                              prof);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace
}  // namespace rsr
