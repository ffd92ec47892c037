// classify_popc.cu -- bit-packed reference-state classifier on the CUDA cores.
//
// What it computes (Sec. 3.3, Algorithm 1): sample h is in I^L if x_h <= r for
// some lower reference r, else in I^U if x_h >= r for some upper reference r,
// else unclassified; lower takes precedence.
//
// How: every state is re-encoded as its thermometer bits t_{i,k} = [x_i >= k],
// k = 1..K-1, packed into 32-bit words (equivalent to the paper's one-hot /
// cumulative encoding of Sec. 3.2: x_i <= r_i iff t(x_i) is a bitwise subset of
// t(r_i)).  Then
//     x <= r^L  iff  OR_w ( t_w(x)  AND NOT t_w(r^L) ) == 0
//     x >= r^U  iff  OR_w ( t_w(r^U) AND NOT t_w(x)  ) == 0
// one LOP3 per word and reference.  The complement of each lower reference is
// stored, so both tests are a single and-or-accumulate.  No violation matrix is
// ever written; each thread keeps its sample's words in registers and streams
// the references through shared memory (broadcast reads).
//
// Fused in the same pass: Philox sampling (or a read of given states), the
// label write, the three counts, and the per-bit counts of I^L samples that the
// score-function gradient needs.  A persistent grid walks 256-sample tiles.
//
// Early-exit mode with the component-major index of the upper set
// (popc_index.cuh, the default): each sample first tries the kHot most
// probable upper references one by one, then the upper chunks are tested
// through the index (one 256-bit OR per decisive zero bit of the sample)
// instead of reference by reference.  Lower chunks are always scanned
// reference by reference.
#include <algorithm>

#include <cuda_runtime.h>

#include "popc_index.cuh"
#include "rsr_internal.cuh"
#include "rsr_launch.h"

namespace rsr {

namespace {

constexpr int kThreads = 256;   // one sample per thread
constexpr int kChunk = 256;     // references per shared-memory chunk
constexpr int kCoopLanes = 16;  // at most this many unresolved lanes: cooperative warp scan
constexpr int kHot = 16;        // upper references tried one by one before the index
constexpr int kCoopIdx = 1;     // at most this many lanes needing the index test: cooperative test
constexpr int kZeroLanes = 32;  // at most this many I^L lanes in a warp: count their zero bits (all: measured fastest)

// Resident blocks per SM the register budget is sized for: four (64 registers a
// thread) while a sample's words fit beside the Philox state, fewer for wide
// encodings, where a tighter budget would spill (C2 at n = 295: 1.30 -> 1.05 ms
// with four instead of two).
constexpr int min_blocks(int wb) { return wb <= 12 ? 4 : (wb <= 16 ? 3 : 2); }
// Chunk buffers: two (the next chunk is copied while the current one is
// tested) unless that would cost a resident block (32 words: one buffer).
template <int WB>
__host__ __device__ constexpr int kBufs() { return WB <= 24 ? 2 : 1; }

struct WordWriter {
    // Appends per-component thermometer runs to a column of 32-bit words in
    // shared memory (word w of thread t at col[w * kThreads]).
    uint32_t *col;
    int w, pos;
    uint32_t cur;
    int km1;
    __device__ __forceinline__ void put(uint32_t x) {
        const uint32_t bits = (1u << x) - 1u;  // x ones, x <= K-1 <= 15
        cur |= bits << pos;
        const int np = pos + km1;
        if (np >= 32) {
            col[w * kThreads] = cur;
            ++w;
            cur = (np > 32) ? (bits >> (32 - pos)) : 0u;
            pos = np - 32;
        } else {
            pos = np;
        }
    }
    __device__ __forceinline__ void flush(int words_b) {
        if (pos > 0) {
            col[w * kThreads] = cur;
            ++w;
        }
        for (; w < words_b; ++w) col[w * kThreads] = 0u;
    }
};

// kDeep: the staged form (a pass that reads the call's tiles or a queue, and may
// queue the samples it leaves unresolved); the one-pass launches run an
// instantiation without it, which keeps the walk's register budget.
template <int WB, bool kDeep>
__global__ void __launch_bounds__(kThreads, min_blocks(WB)) classify_popc_kernel(const ClassifyParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    // smem starts with the sampler's 32-bit threshold tables and never words (kMaxKenc * 8 bytes)
    uint32_t *s_tw = reinterpret_cast<uint32_t *>(smem + (size_t)kMaxKenc * 8);
    uint32_t *s_buf = s_tw + WB * kThreads;           // kBufs chunk buffers of kChunk * WB words
    // per thermometer bit: one bits of I^L samples counted by ballots, minus zero bits
    // of those counted by their zero bits (modulo 2^32; s_fz of them are added at the end)
    uint32_t *s_cum = s_buf + kBufs<WB>() * kChunk * WB;
    uint32_t *s_hot = s_cum + WB * 32;      // the first kHot upper references (index mode)
    uint32_t *s_first = s_hot + kHot * WB;  // component start bits per encoding word (index mode)
    __shared__ __align__(16) uint32_t s_zero[kIdxWords];
    __shared__ uint32_t s_and[2][2 * kMaxWords];   // skip rows of the staged chunks (index AND row; lower AND, guard rows)
    __shared__ unsigned long long s_cnt[3];
    __shared__ unsigned long long s_exec, s_ops;
    __shared__ unsigned int s_fz;           // I^L samples counted by their zero bits
    __shared__ unsigned int s_pend[kThreads / 32];   // unresolved samples per warp at the pass's last step
    __shared__ long long s_deep_pos;                 // the tile's reservation in the output queue

    // a pass over a queue: nothing to do for blocks beyond its groups (before any set-up)
    if (kDeep && p.q_in >= 0) {
        const unsigned long long q = *((volatile const unsigned long long *)(p.deep_count + p.q_in));
        const unsigned long long queued_now = q < (unsigned long long)p.deep_cap ? q : (unsigned long long)p.deep_cap;
        if ((unsigned long long)blockIdx.x * kThreads >= queued_now) return;
    }
    const bool use_idx = p.popc_UT != nullptr && !p.dense && p.R_U > 0;
    const bool use_lg = p.popc_LG != nullptr && !p.dense && p.R_L > 0;   // lower chunk skip rows
    const int hotc = use_idx ? (int)(p.R_U < kHot ? p.R_U : kHot) : 0;
    // 32-bit thresholds and never words: binary (never words at kMaxKenc) or multi-state
    // (multi_tables_to_smem's layout, at most kMaxKenc + 7 (K-1) + 32 words)
    uint32_t *s_t32 = reinterpret_cast<uint32_t *>(smem);
    uint32_t *s_never = s_t32 + kMaxKenc;
    const bool binary = p.km1 == 1;
    if (binary) binary_tables_to_smem(p.thr, p.n, s_t32, s_never, tid, kThreads);
    else multi_tables_to_smem(p.thr, p.n, p.km1, s_t32, tid, kThreads);   // 32-bit tables and never words
    if (use_idx) {
        for (int i = tid; i < hotc * WB; i += kThreads) s_hot[i] = p.popc_U[i];
        for (int w = tid; w < WB; w += kThreads) s_first[w] = component_first_bits(p.km1, p.kenc, w);
        if (tid < kIdxWords) s_zero[tid] = 0u;
    }
    if (p.grad_counts)
        for (int j = tid; j < WB * 32; j += kThreads) s_cum[j] = 0u;
    if (tid == 0) s_fz = 0u;
    if (tid < 3) s_cnt[tid] = 0ull;
    if (tid == 0) s_exec = s_ops = 0ull;
    __syncthreads();

    // Set order: see ChunkWalk (upper bursts between lower chunks without
    // overlapping pairs, lower first with them, as Algorithm 1's precedence requires).
    const bool overlap = *((volatile const int32_t *)&p.hdr->overlap) != 0;
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    unsigned long long my_cnt0 = 0, my_cnt1 = 0, my_cnt2 = 0, my_exec = 0;
    unsigned long long my_ops = 0;   // 32-bit logic operations on reference data (scan words, AND rows, index rows)

    // Staged passes in early-exit mode (kDeep): a pass walks chunk steps
    // [step_lo, step_hi) for the call's tiles (q_in < 0, step_lo = 0) or for the
    // samples queue q_in holds, 256 at a time, and queues the samples still
    // unresolved at step_hi into queue q_out for the next pass (none in the last).
    const bool second = kDeep && p.q_in >= 0;
    const int64_t nU = (p.R_U + kChunk - 1) / kChunk, nL = (p.R_L + kChunk - 1) / kChunk;
    const int64_t nsteps = nU + nL;
    const bool defer = kDeep && !p.dense && p.q_out >= 0 && p.deep != nullptr && p.deep_cap > 0;
    const int64_t step0 = second ? (p.step_lo < nsteps ? p.step_lo : nsteps) : 0;
    const int64_t lim0 = defer && p.step_hi < nsteps ? p.step_hi : nsteps;
    const int64_t *q_in = second ? p.deep + (size_t)p.q_in * p.deep_cap : nullptr;
    int64_t *q_out = defer ? p.deep + (size_t)p.q_out * p.deep_cap : nullptr;
    unsigned long long *q_out_count = defer ? p.deep_count + p.q_out : nullptr;
    const int64_t queued =
        second ? (int64_t)min(*((volatile const unsigned long long *)(p.deep_count + p.q_in)),
                              (unsigned long long)p.deep_cap)
               : 0;
    const int64_t ntiles = second ? (queued + kThreads - 1) / kThreads : (p.N + kThreads - 1) / kThreads;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int64_t hl = tile * kThreads + tid;
        if (second) hl = hl < queued ? q_in[hl] : -1;   // -1: a voided entry or no entry
        const bool valid = hl >= 0 && hl < p.N;
        ChunkWalk walk(nU, nL, overlap, use_idx);
        bool upper = false;
        int64_t ci = 0;
        for (int64_t i = 0; i < step0; ++i) walk.next(&upper, &ci);   // a later pass resumes at step_lo
        walk.next(&upper, &ci);   // step0 < nsteps: some reference exists, and nothing is queued at nsteps
        int64_t lim = lim0;
        bool deferred = false;
        auto chunk_refs = [&](bool up, int64_t c, int *cnt_out) {
            const int64_t R = up ? p.R_U : p.R_L;
            const int64_t base = c * kChunk;
            *cnt_out = (int)((R - base) < (int64_t)kChunk ? (R - base) : (int64_t)kChunk);
            return (up ? p.popc_U : p.popc_L) + base * WB;
        };
        auto issue = [&](int buf, bool up, int64_t c) {
            int cnt_c;
            const uint32_t *rows = chunk_refs(up, c, &cnt_c);
            const bool ix = use_idx && up, lg = use_lg && !up;
            const uint32_t *skip = ix ? p.popc_UA + (size_t)c * WB : (lg ? p.popc_LG + (size_t)c * 2 * WB : nullptr);
            load_chunk_async<WB, kThreads>(s_buf + buf * (kChunk * WB), ix,
                                           ix ? p.popc_UT + (size_t)c * kIdxChunk * WB : nullptr, p.kenc, skip,
                                           ix ? WB : 2 * WB, s_and[buf], rows, cnt_c, tid);
        };
        if (kBufs<WB>() == 2) {
            __syncthreads();                          // every thread is done with the previous tile's buffers
            issue((int)(step0 & 1), upper, ci);       // the first chunk, copied while the tile is sampled
        }

        // ---- sample (or read) and encode this thread's state ----------------
        WordWriter ww{s_tw + tid, 0, 0, 0u, p.km1};
        if (valid && binary && !p.samples) {
            sample_binary_words<WB, kThreads>(p.offset + (uint64_t)hl, key0, key1, p.n, s_t32, s_never, s_tw + tid);
            ww.w = WB;  // every word written
        } else if (valid) {
            if (p.samples) {
                const uint8_t *row = p.samples + hl * (int64_t)p.n;
                for (int i = 0; i < p.n; ++i) ww.put(row[i]);
            } else {
                sample_multi_words<WB, kThreads>(p.offset + (uint64_t)hl, key0, key1, p.n, p.km1, s_t32, s_tw + tid);
                ww.w = WB;  // every word written
            }
        }
        ww.flush(WB);
        uint32_t t[WB];
#pragma unroll
        for (int w = 0; w < WB; ++w) t[w] = s_tw[w * kThreads + tid];

        // ---- classify ---------------------------------------------------------
        bool mL = false, mU = false;
        bool done = !valid;
        // index mode: the most probable upper references first, one by one (with an
        // overlapping pair every lower chunk has to come first: no shortcut then)
        if (hotc > 0 && !overlap && !done && !second) {
            int r = 0;
            for (; r < hotc; ++r) {
                uint32_t acc = 0;
#pragma unroll
                for (int w = 0; w < WB; ++w) acc |= s_hot[r * WB + w] & ~t[w];
                if (acc == 0u) {
                    mU = true;
                    done = true;
                    ++r;
                    break;
                }
            }
            my_exec += (unsigned long long)r;
            my_ops += (unsigned long long)r * WB;
        }
        for (int64_t step = step0; step < nsteps; ++step) {
            if (kBufs<WB>() == 2) cp_async_wait_all();      // this thread's copies of chunk `step`
            const bool all_done = __syncthreads_and(done);  // chunk `step` visible; chunk step-1 consumed
            if (all_done && !p.dense) break;
            if (kDeep && step == lim) {
                // The pass's steps are spent: queue the unresolved samples for the next
                // pass (a block-wide reservation).  An unresolved sample has no match so
                // far: with an overlapping pair a lower match is final and upper chunks
                // come last.
                const bool pend = !done;
                const unsigned wb = __ballot_sync(0xffffffffu, pend);
                if (lane == 0) s_pend[tid >> 5] = (unsigned)__popc(wb);
                __syncthreads();
                int before = 0, total = 0;
#pragma unroll
                for (int w = 0; w < kThreads / 32; ++w) {
                    const int c = (int)s_pend[w];
                    before += (w < (tid >> 5)) ? c : 0;
                    total += c;
                }
                if (tid == 0) s_deep_pos = (long long)atomicAdd(q_out_count, (unsigned long long)total);
                __syncthreads();
                const long long pos = s_deep_pos;
                if (pos + total <= (long long)p.deep_cap) {
                    if (pend) {
                        q_out[pos + before + __popc(wb & ((1u << lane) - 1u))] = hl;
                        deferred = true;
                    }
                    break;
                }
                // the queue is full: void this reservation's slots below the capacity, walk on here
                for (long long k = tid; k < total && pos + k < (long long)p.deep_cap; k += kThreads)
                    q_out[pos + k] = -1;
                lim = nsteps;
            }
            const int cur_buf = kBufs<WB>() == 2 ? (int)(step & 1) : 0;
            uint32_t *s_ref = s_buf + cur_buf * (kChunk * WB);
            int cnt;
            (void)chunk_refs(upper, ci, &cnt);
            const bool idx_chunk = use_idx && upper;
            bool up_next = false;
            int64_t ci_next = 0;
            if (step + 1 < nsteps) walk.next(&up_next, &ci_next);
            if (kBufs<WB>() == 2) {
                if (step + 1 < nsteps) issue((int)((step + 1) & 1), up_next, ci_next);
            } else {
                issue(0, upper, ci);
                cp_async_wait_all();
                __syncthreads();
            }
            if (p.dense) {
                bool m = false;
                if (valid) {
                    if (upper) {
                        for (int r = 0; r < cnt; ++r) {
                            uint32_t acc = 0;
#pragma unroll
                            for (int w = 0; w < WB; ++w) acc |= s_ref[r * WB + w] & ~t[w];
                            m |= (acc == 0u);
                        }
                    } else {
                        for (int r = 0; r < cnt; ++r) {
                            uint32_t acc = 0;
#pragma unroll
                            for (int w = 0; w < WB; ++w) acc |= t[w] & s_ref[r * WB + w];
                            m |= (acc == 0u);
                        }
                    }
                    my_exec += (unsigned long long)cnt;
                    my_ops += (unsigned long long)cnt * WB;
                }
                if (upper) mU |= m; else mL |= m;
            } else if (idx_chunk) {
                // Early exit through the index.  A sample lacking a bit of the chunk's
                // AND row dominates none of its references; the others are tested
                // per lane while several need it, one sample per warp otherwise.
                const bool ruled = !done && chunk_ruled_out<WB>(t, s_and[cur_buf]);
                if (!done) {
                    my_exec += (unsigned long long)cnt;
                    my_ops += WB;   // the AND-row test
                }
                const unsigned need = __ballot_sync(0xffffffffu, !done && !ruled);
                if (__popc(need) > kCoopIdx) {
                    if (!done && !ruled && idx_match_lane<WB>(t, s_ref, s_first, s_zero, p.kenc, cnt, &my_ops)) {
                        mU = true;
                        done = true;
                    }
                } else {
                    unsigned rem = need;
                    while (rem) {
                        const int src_lane = __ffs(rem) - 1;
                        rem &= rem - 1;
                        const bool found = idx_match_warp<WB, kThreads>(s_tw + (tid - lane + src_lane), s_ref,
                                                                        s_first, p.kenc, cnt, lane, &my_ops);
                        if (lane == src_lane && found) {
                            mU = true;
                            done = true;
                        }
                    }
                    __syncwarp();  // the columns read above are rewritten by their lanes for the next tile
                }
            } else {
                // Early-exit mode.  In a lower chunk a lane whose sample the chunk's skip
                // rows rule out passes over it.  While many lanes of the warp are
                // unresolved each lane scans for its own sample; once few remain, the warp
                // scans cooperatively, one unresolved sample at a time, 32 references per step.
                bool skip = false;
                if (!done && !upper && use_lg) {
                    skip = lower_chunk_ruled_out<WB>(t, s_and[cur_buf]);
                    my_ops += 2 * WB;   // the skip-row test
                    if (skip) my_exec += (unsigned long long)cnt;
                }
                const unsigned active = __ballot_sync(0xffffffffu, !done && !skip);
                if (__popc(active) > kCoopLanes) {
                    if (!done && !skip) {
                        int r = 0;
                        bool m = false;
                        if (upper) {
                            for (; r < cnt; ++r) {
                                uint32_t acc = 0;
#pragma unroll
                                for (int w = 0; w < WB; ++w) acc |= s_ref[r * WB + w] & ~t[w];
                                if (acc == 0u) { m = true; ++r; break; }
                            }
                        } else {
                            for (; r < cnt; ++r) {
                                uint32_t acc = 0;
#pragma unroll
                                for (int w = 0; w < WB; ++w) acc |= t[w] & s_ref[r * WB + w];
                                if (acc == 0u) { m = true; ++r; break; }
                            }
                        }
                        my_exec += (unsigned long long)r;
                        my_ops += (unsigned long long)r * WB;
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
                        int tested = 0;
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
                            tested = (cnt < r0 + 32) ? cnt : r0 + 32;
                        }
                        if (lane == src) {
                            my_exec += (unsigned long long)tested;
                            my_ops += (unsigned long long)tested * WB;
                            if (found) {
                                if (upper) mU = true; else mL = true;
                                done = true;
                            }
                        }
                    }
                }
            }
            upper = up_next;
            ci = ci_next;
        }
        const int label = mL ? 0 : (mU ? 1 : 2);
        const bool final_ = valid && !deferred;   // a deferred sample is counted by a later pass
        if (final_) {
            if (p.labels) p.labels[hl] = (uint8_t)label;
            my_cnt0 += label == 0;
            my_cnt1 += label == 1;
            my_cnt2 += label == 2;
        }

        // ---- per-bit counts of I^L samples (gradient) ------------------------
        // A warp with at most kZeroLanes I^L samples counts their zero bits (sparse)
        // with shared atomics; otherwise 32 ballots per word count the one bits of
        // all lanes.  With kZeroLanes = 32 every warp takes the zero bits, which
        // measured faster than the ballots on C2 and C4.
        if (p.grad_counts) {
            const bool isL = final_ && label == 0;
            const unsigned lmask = __ballot_sync(0xffffffffu, isL);
            if (lmask && __popc(lmask) <= kZeroLanes) {
                if (isL) {
#pragma unroll
                    for (int w = 0; w < WB; ++w) {
                        uint32_t z = ~t[w] & enc_valid_bits(p.kenc, w);
                        while (z) {
                            const int b = __ffs(z) - 1;
                            z &= z - 1u;
                            atomicSub(&s_cum[w * 32 + b], 1u);   // ones = (zero-route samples) - zeros
                        }
                    }
                }
                if (lane == 0) atomicAdd(&s_fz, (unsigned)__popc(lmask));
            } else if (lmask) {
#pragma unroll
                for (int w = 0; w < WB; ++w) {
                    uint32_t mine = 0;
                    const uint32_t tw = isL ? t[w] : 0u;
#pragma unroll 4
                    for (int b = 0; b < 32; ++b) {
                        const uint32_t m = __ballot_sync(0xffffffffu, (tw >> b) & 1u);
                        if (lane == b) mine = __popc(m);
                    }
                    if (mine) atomicAdd(&s_cum[w * 32 + lane], mine);
                }
            }
        }
    }

    // ---- block totals -> global -------------------------------------------
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        my_cnt0 += __shfl_xor_sync(0xffffffffu, my_cnt0, o);
        my_cnt1 += __shfl_xor_sync(0xffffffffu, my_cnt1, o);
        my_cnt2 += __shfl_xor_sync(0xffffffffu, my_cnt2, o);
        my_exec += __shfl_xor_sync(0xffffffffu, my_exec, o);
        my_ops += __shfl_xor_sync(0xffffffffu, my_ops, o);
    }
    if (lane == 0) {
        atomicAdd(&s_cnt[0], my_cnt0);
        atomicAdd(&s_cnt[1], my_cnt1);
        atomicAdd(&s_cnt[2], my_cnt2);
        atomicAdd(&s_exec, my_exec);
        atomicAdd(&s_ops, my_ops);
    }
    __syncthreads();
    if (tid < 3 && s_cnt[tid]) atomicAdd(&p.counts3[tid], s_cnt[tid]);
    if (tid == 0 && p.exec_tests && s_exec) atomicAdd(p.exec_tests, s_exec);
    if (tid == 0 && p.exec_tests && s_ops) atomicAdd(p.exec_tests + 1, s_ops);
    if (p.grad_counts && s_cnt[0]) {
        // C[i,0] += F - cum_1 ; C[i,k] += cum_k - cum_{k+1} (cum_K = 0); cum_j = one bits
        // counted by ballots + (samples counted by zero bits - their zero bits)
        for (int i = tid; i < p.n; i += kThreads) {
            long long prev = (long long)s_cnt[0];
            for (int k = 1; k <= p.km1; ++k) {
                const int j = i * p.km1 + (k - 1);
                const long long cum = (long long)(uint32_t)(s_cum[j] + s_fz);
                const long long d = prev - cum;
                if (d) atomicAdd(&p.grad_counts[(size_t)i * p.K + (k - 1)], (unsigned long long)d);
                prev = cum;
            }
            if (prev) atomicAdd(&p.grad_counts[(size_t)i * p.K + p.km1], (unsigned long long)prev);
        }
    }
}

template <int WB, bool kDeep>
cudaError_t launch_wb(const ClassifyParams &p, cudaStream_t s) {
    // dynamic shared memory for the largest threshold table; the attribute and
    // the occupancy are queried once per device so that launches made during
    // stream capture issue nothing but the kernel
    const size_t smem = (size_t)kMaxKenc * 8 +
                        sizeof(uint32_t) * ((size_t)WB * kThreads + (size_t)kBufs<WB>() * kChunk * WB + (size_t)WB * 32 +
                                            (size_t)kHot * WB + (size_t)WB);
    static int occ_cache[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int occ = (dev >= 0 && dev < 64) ? occ_cache[dev] : 0;
    if (occ == 0) {
        e = cudaFuncSetAttribute(classify_popc_kernel<WB, kDeep>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, classify_popc_kernel<WB, kDeep>, kThreads, smem);
        if (e != cudaSuccess) return e;
        if (occ < 1) occ = 1;
        if (dev >= 0 && dev < 64) occ_cache[dev] = occ;
    }
    const int64_t ntiles = (p.N + kThreads - 1) / kThreads;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)device_sm_count() * occ);
    if (grid <= 0) return cudaSuccess;
    classify_popc_kernel<WB, kDeep><<<(unsigned)grid, kThreads, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

int popc_word_bucket(int words) {
    static const int buckets[] = {1, 2, 4, 6, 8, 10, 12, 16, 24, 32};
    for (int b : buckets)
        if (words <= b) return b;
    return -1;
}

namespace {
cudaError_t launch_words(const ClassifyParams &p, cudaStream_t s) {
    const bool deep = p.k0 > 0;   // the staged form (the launcher clears k0 for one pass)
    switch (p.words) {
        case 1: return deep ? launch_wb<1, true>(p, s) : launch_wb<1, false>(p, s);
        case 2: return deep ? launch_wb<2, true>(p, s) : launch_wb<2, false>(p, s);
        case 4: return deep ? launch_wb<4, true>(p, s) : launch_wb<4, false>(p, s);
        case 6: return deep ? launch_wb<6, true>(p, s) : launch_wb<6, false>(p, s);
        case 8: return deep ? launch_wb<8, true>(p, s) : launch_wb<8, false>(p, s);
        case 10: return deep ? launch_wb<10, true>(p, s) : launch_wb<10, false>(p, s);
        case 12: return deep ? launch_wb<12, true>(p, s) : launch_wb<12, false>(p, s);
        case 16: return deep ? launch_wb<16, true>(p, s) : launch_wb<16, false>(p, s);
        case 24: return deep ? launch_wb<24, true>(p, s) : launch_wb<24, false>(p, s);
        case 32: return deep ? launch_wb<32, true>(p, s) : launch_wb<32, false>(p, s);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

// One pass, or in early-exit mode with deep queues, k0 > 0 and at least
// two_pass_min_n samples (kTwoPassMinN) staged passes (staged_passes()): the
// first walks chunk steps [0, k0) of the call's tiles, each later one takes the
// samples the previous one queued, 256 at a time, and walks kDeferGrowth times
// as far as the step it starts at (next_stage_end); the last walks to the end.  Two queues
// alternate; each pass that queues clears its queue's count first (a memset and
// a launch per pass, all on stream s; a pass whose queue is empty returns at
// once).  Below that size the extra launches and memsets cost more than the
// deferral saves (the 256 hazard scenarios at 2e5 samples each: 37.5 ms in two
// passes against 34.2 ms in one).
cudaError_t launch_classify_popc(const ClassifyParams &p, cudaStream_t s) {
    const int64_t nsteps = (p.R_U + kChunk - 1) / kChunk + (p.R_L + kChunk - 1) / kChunk;
    if (p.dense || p.k0 <= 0 || !p.deep || !p.deep_count || p.deep_cap <= 0 || p.N < p.two_pass_min_n ||
        staged_passes(nsteps, p.k0) < 2) {
        ClassifyParams one = p;
        one.k0 = 0;
        one.q_in = one.q_out = -1;
        one.step_lo = 0;
        one.step_hi = nsteps;
        return launch_words(one, s);
    }
    int64_t lo = 0, hi = p.k0;
    int q_in = -1, q_out = 0;
    while (true) {
        const bool last = hi >= nsteps;
        ClassifyParams c = p;
        c.q_in = q_in;
        c.q_out = last ? -1 : q_out;
        c.step_lo = lo;
        c.step_hi = last ? nsteps : hi;
        cudaError_t e;
        if (!last && (e = cudaMemsetAsync(p.deep_count + q_out, 0, sizeof(unsigned long long), s)) != cudaSuccess)
            return e;
        if ((e = launch_words(c, s)) != cudaSuccess) return e;
        if (last) return cudaSuccess;
        lo = hi;
        hi = next_stage_end(hi, nsteps);
        q_in = q_out;
        q_out ^= 1;
    }
}

}  // namespace rsr
