/*
 * rsr.h -- C ABI of the GB300 (sm_103a) RSR hot-path library, librsr.so.
 *
 * Reference-state System Reliability (arXiv 2604.17066): N Monte Carlo samples
 * of n components with K states each are classified against lower (failure,
 * S <= m') and upper (survival, S >= m'+1) reference states; probabilities,
 * coefficients of variation and score-function gradients follow from integer
 * counts.
 *
 * Conventions (all functions):
 *   - Return RSR_OK (0) or a negative rsr_status; no exception crosses the ABI.
 *   - "device" pointers are CUDA global-memory pointers on the current device;
 *     "host" pointers are ordinary CPU memory.  The caller owns every buffer;
 *     the library allocates no device memory (the caller passes a workspace of
 *     rsr_workspace_size() bytes, 256-byte aligned).
 *   - Calls that take a stream are asynchronous on it unless stated otherwise.
 *     Stream 0 is the legacy default stream.
 *   - Component states are uint8 in [0, K).  Reference and sample matrices are
 *     row-major, one row of n states per reference / sample.
 *   - Labels: 0 = I^L (sample lies below a lower reference: S <= m'),
 *             1 = I^U (sample lies above an upper reference: S >= m'+1),
 *             2 = I^u (unclassified).
 *   - Sampler (not specified by the paper, Sec. 3.1 assumes P(X) can be
 *     sampled): thresholds T_{i,k} = min(2^32, floor(2^32 * sum_{j<k} q_{i,j}))
 *     with the fp64 sum taken left to right; component i of sample h
 *     (h = offset + local index) uses u = word (i mod 4) of
 *     Philox4x32-10(key = (seed lo32, seed hi32), ctr = (h lo32, h hi32, i/4, 0))
 *     and takes state x = #{k in 1..K-1 : u >= T_{i,k}}.
 *   - Limits: 1 <= n, 2 <= K <= 16, n*(K-1) <= 1024, R_L + R_U >= 1,
 *     R_L, R_U < 2^31.
 */
#ifndef RSR_H
#define RSR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RSR_API __attribute__((visibility("default")))
#else
#define RSR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *rsr_stream_t;

typedef enum rsr_status {
    RSR_OK = 0,
    RSR_ERR_INVALID_ARG = -1,    /* NULL pointer, size out of range, pmf row not summing to 1 */
    RSR_ERR_CUDA = -2,           /* a CUDA runtime call failed (rsr_last_cuda_error() has it) */
    RSR_ERR_WORKSPACE = -3,      /* workspace too small or not 256-byte aligned */
    RSR_ERR_TIMEOUT = -4,        /* a bounded device wait gave up (the context stays usable) */
    RSR_ERR_UNSUPPORTED = -5,    /* sizes beyond the limits above, or no sm_100-family GPU */
    RSR_ERR_NOT_PREPARED = -6    /* workspace not prepared for this problem / pmf */
} rsr_status;

/* Classifier implementation. */
typedef enum rsr_path {
    RSR_PATH_AUTO = 0,  /* tuned choice (see rsr_autotune) */
    RSR_PATH_POPC = 1,  /* bit-packed AND / OR-reduce on the CUDA cores */
    RSR_PATH_TC = 2     /* tcgen05 FP8 violation contraction on the tensor cores */
} rsr_path;

/* rsr_problem.flags */
#define RSR_FLAG_DENSE 1u  /* test every sample against every reference (no early exit) */
/* Bit-packed path, early-exit mode: scan both sets reference by reference,
 * without the upper set's component-major index and the lower set's chunk
 * skip.  The index (built by rsr_prepare) tests a chunk of 256 upper
 * references with one 256-bit OR per component of the sample below its top
 * state, after a direct test of the 16 most probable upper references.  The
 * chunk skip passes over a chunk of 256 lower references when the sample has a
 * 1 at a thermometer bit that all of them lack, or at every guard bit of the
 * chunk (each lower reference's guard: the bit it lacks that is most likely 1;
 * rsr_prepare groups the lower references after the 256 most probable by
 * guard).  Labels, counts and gradient counts are the same either way. */
#define RSR_FLAG_NO_INDEX 2u
/* Failure-detection test hook (tensor-core path only): the reference producer
 * never starts, so the kernel's bounded waits run out after about 10 ms; the
 * kernel records RSR_ERR_TIMEOUT in the workspace header (rsr_workspace_status),
 * frees its tensor memory and returns, leaving the context usable. */
#define RSR_FLAG_TEST_STALL 0x100u
/* Test hook (batched bit-packed path): the scenario's deep queue holds 1024
 * samples, so that tiles find it full and finish their walk themselves (the
 * fallback a queue of one entry per sample never needs). */
#define RSR_FLAG_TEST_DEEP_CAP 0x200u
/* Test hook (bit-packed path, early exit): staged passes whenever the
 * workspace holds a deep queue, whatever N (without it, calls of fewer than
 * 2^19 samples run one pass). */
#define RSR_FLAG_TEST_TWO_PASS 0x400u
/* Test hook (batched bit-packed path): the scenario's first-pass work items
 * hold three consecutive 256-sample tiles each instead of one, until
 * rsr_batch_autotune picks the tiles per item for every scenario. */
#define RSR_FLAG_TEST_TILES3 0x800u

/*
 * One classification problem for a threshold m' (Sec. 3.2-3.3).
 *   n, K     : components and states per component (paper: N and M).
 *   pmf      : host, n*K fp64, row i = P(X_i = 0..K-1); each row sums to 1 within 1e-9.
 *   R_L, R_U : numbers of lower / upper reference states (paper: R^L, R^U).
 *   ref_L    : device, R_L*n uint8, lower references x^L_r (Eq. (2)); may be NULL if R_L = 0.
 *   ref_U    : device, R_U*n uint8, upper references x^U_r (Eq. (3)); may be NULL if R_U = 0.
 *   path     : rsr_path.
 *   flags    : RSR_FLAG_* bits.
 * The library reads ref_L / ref_U only inside rsr_prepare (it keeps its own
 * encoded copies in the workspace).
 */
typedef struct rsr_problem {
    int32_t n;
    int32_t K;
    const double *pmf;
    int64_t R_L;
    int64_t R_U;
    const uint8_t *ref_L;
    const uint8_t *ref_U;
    int32_t path;
    uint32_t flags;
} rsr_problem;

/* Estimates from integer counts (Sec. 3.3 estimators and c.o.v.; Sec. 3.5). */
typedef struct rsr_estimate_out {
    double pL, pU, pu;   /* |I^L|/H, |I^U|/H, |I^u|/H */
    double P_lower;      /* (|I^L| + n_u_lower)/H : P(S <= m') once I^u is resolved */
    double P_upper;      /* (|I^U| + |I^u| - n_u_lower)/H : P(S >= m'+1) */
    double cov_pL, cov_pU, cov_pu, cov_lower, cov_upper;  /* sqrt((1-p)/(H p)); +inf at p = 0 */
} rsr_estimate_out;

/*
 * Workspace bytes for `problem` with deep queues for calls of up to N
 * samples: the prepared references, then (N > 0) two queues of min(N, 2^22)
 * sample indices each for the bit-packed path's staged passes.  Any workspace
 * of at least rsr_workspace_size(problem, 0) bytes serves calls of any N: the
 * queues are whatever the workspace holds beyond that size (none: one pass),
 * and a tile whose samples would overflow a queue finishes their walk itself.
 * 0 on invalid input (or N < 0).
 */
RSR_API size_t rsr_workspace_size(const rsr_problem *problem, int64_t N);

/*
 * Prepare `ws` for `problem` (Sec. 3.2 encoding, plus the sampler thresholds):
 * computes the thresholds on the host, orders each reference set by the
 * probability of the region its references dominate, encodes both sets
 * (bit-packed thermometer words; FP8 0/1 tiles in the tensor-core
 * shared-memory layout), builds the component-major index of the upper set
 * with one AND row per chunk of 256 references (in a clustered order when a
 * few binary components fail far more often than the rest), orders the lower
 * set's bit-packed rows by guard after its 256 most probable references, with
 * an AND row and a guard row per chunk (RSR_FLAG_NO_INDEX), and runs the
 * precedence pre-check (does any upper reference lie below a lower
 * reference?  Algorithm 1 lets lower win; if no pair overlaps, the kernels may
 * stop at the first match in either set).  None of these orders changes a
 * label.  Synchronises `stream`: reference scores and clustering keys are
 * sorted on the host.  Not capturable in a CUDA graph.
 */
RSR_API int rsr_prepare(const rsr_problem *problem, void *ws, size_t ws_bytes, rsr_stream_t stream);

/*
 * Recompute only the sampler thresholds after `problem->pmf` changed (the
 * references stay valid when component probabilities change, Sec. 5).  `ws`
 * must have been prepared for the same references.  Clears the workspace's
 * device error word (rsr_workspace_status).
 */
RSR_API int rsr_update_pmf(const rsr_problem *problem, void *ws, size_t ws_bytes, rsr_stream_t stream);

/*
 * Classify N samples (Sec. 3.3, Algorithm 1; lower takes precedence).
 *   seed, offset     : sampler key and index of the first sample.
 *   samples_or_null  : device N*n uint8 states to classify instead of sampling; NULL = sample.
 *   labels_or_null   : device N uint8 labels (0/1/2); NULL = do not write labels.
 *   counts3          : device int64[3], |I^L|, |I^U|, |I^u| are ADDED (the caller zeroes it).
 *   grad_counts_or_null : device int64[n*K]; C[i*K+k] += #{h in I^L : x_{h,i} = k}.
 *   exec_tests_or_null  : device int64[2]; [0] += reference tests actually executed
 *                         (tiles issued x tile size on the tensor path; on the
 *                         bit-packed path every reference of an upper chunk that
 *                         the index test visits, and of a lower chunk that the
 *                         chunk skip passes over, counts); [1] += the 32-bit logic
 *                         operations the bit-packed path issued on reference data:
 *                         one per word of each scanned reference test, one per
 *                         word of each chunk AND-row test, two per word of each
 *                         lower chunk-skip test, 4 per index row ORed
 *                         by one lane (8 words, two rows per three-input OR) plus
 *                         8 per encoding word it visits, 1 per index word ORed in
 *                         the warp-cooperative test (0 on the tensor path).
 * `ws` must be prepared for this problem and pmf (else RSR_ERR_NOT_PREPARED).
 * On the bit-packed path in early-exit mode, for N >= 2^19 samples, when `ws`
 * holds deep queues (see rsr_workspace_size), the call runs in stages, one
 * launch each (after a memset of the count of the queue it fills): the first
 * walks k0 reference chunks per 256-sample tile (k0 from rsr_autotune for this
 * problem shape, else 2) and queues the samples still unresolved; each later
 * stage takes the queued samples 256 at a time and walks on to four times the
 * chunk step it starts at, queueing again, and the last walks to the end
 * (rsr_classify_plan gives the count).  Labels, counts and gradient counts are
 * those of one pass.  Capturable in a CUDA graph.
 */
RSR_API int rsr_classify(const rsr_problem *problem, uint64_t seed, uint64_t offset, int64_t N,
                 const uint8_t *samples_or_null, uint8_t *labels_or_null, int64_t *counts3,
                 int64_t *grad_counts_or_null, int64_t *exec_tests_or_null,
                 void *ws, size_t ws_bytes, rsr_stream_t stream);

/*
 * What rsr_classify would run for N samples of `problem` in a prepared
 * workspace of ws_bytes bytes (host only, no device work): out[0] = the path
 * (RSR_PATH_POPC or RSR_PATH_TC, after RSR_PATH_AUTO's decision), out[1] = the
 * kernel launches (0 for N = 0; one per stage when the bit-packed path runs in stages),
 * out[2] = the first pass's chunk-step budget k0 (0: one pass).
 */
RSR_API int rsr_classify_plan(const rsr_problem *problem, int64_t N, size_t ws_bytes, int32_t out[3]);

/*
 * Estimates on the host from counts3 (host int64[3]) and H = N (Sec. 3.3):
 * p_hat = count/H and delta_hat = sqrt((1 - p)/(H p)); n_u_lower = number of
 * unclassified samples that Phi resolved to S <= m' (Sec. 3.5 Stage 2; pass 0
 * before Stage 2).  Synchronous, no CUDA.
 */
RSR_API int rsr_estimate(const int64_t counts3[3], int64_t N, int64_t n_u_lower, rsr_estimate_out *out);

/*
 * Score-function gradient of P(S <= m') with respect to every q_{i,k} (not in
 * the paper).  dP/dq_{i,k} = E[1_F 1{X_i = k}]/q_{i,k} = P(F | X_i = k), F = S <= m'.
 *   grad_counts : device int64[n*K] from rsr_classify over samples offset..offset+N-1;
 *                 the states of the listed unclassified samples are ADDED to it in place.
 *   u_lower_idx : device int64[n_u_lower], local indices (0..N-1) of unclassified samples
 *                 that Phi resolved to S <= m'; may be NULL if n_u_lower = 0.
 *   grad_out, se_out : host fp64[n*K]: g = (C/H)/q, se = sqrt(p(1-p)/H)/q with p = C/H.
 * Synchronises `stream` (reads the counts back).  Uses the thresholds in `ws`.
 * Errors: RSR_ERR_INVALID_ARG if a listed index lies outside [0, N); the
 * indices are checked on the device before any count changes, so grad_counts
 * is then left as it was.  Each call checks only its own indices: a device
 * error recorded in the workspace by an earlier call (rsr_workspace_status)
 * does not make rsr_grad fail.
 */
RSR_API int rsr_grad(const rsr_problem *problem, uint64_t seed, uint64_t offset, int64_t N,
             int64_t *grad_counts, const int64_t *u_lower_idx, int64_t n_u_lower,
             double *grad_out, double *se_out, void *ws, size_t ws_bytes, rsr_stream_t stream);

/*
 * Materialise samples offset..offset+N-1 as device N*n uint8 states (the same
 * states rsr_classify draws).  `ws` must hold this problem's thresholds.
 */
RSR_API int rsr_sample(const rsr_problem *problem, uint64_t seed, uint64_t offset, int64_t N,
               uint8_t *states, void *ws, size_t ws_bytes, rsr_stream_t stream);

/*
 * Device-side results of the precedence pre-check and error flag, copied to
 * host int32[2] = {overlapping pairs > 0, device error code}.  Synchronises
 * `stream`.  The error word records problems that kernels find while they run
 * (RSR_ERR_TIMEOUT from a bounded wait; 2 = a node index out of range; 3 = a
 * broken flow path; 4 = the Stage-2 index list was full) and keeps the first
 * or largest code: it is sticky until rsr_prepare or rsr_update_pmf clears it.
 */
RSR_API int rsr_workspace_status(const void *ws, int32_t out[2], rsr_stream_t stream);

/*
 * Batched launch (many problems, e.g. hazard scenarios, in persistent
 * kernels).  Arrays of length S describe the scenarios; scenario s classifies
 * samples offsets[s] + r*Ns[s] .. offsets[s] + (r+1)*Ns[s] - 1 of its own
 * Philox stream (key seeds[s]) on the r-th rsr_batch call after
 * rsr_batch_prepare (r = 0 first), with the test of Algorithm 1 (Sec. 3.3):
 * on the tensor cores (the CTA-pair FP8 contraction, one persistent launch
 * over every dense tensor-core scenario's 256-sample blocks) for scenarios in
 * dense mode whose path is RSR_PATH_TC, or RSR_PATH_AUTO when timing (or,
 * before rsr_batch_autotune, the reference-count rule of RSR_PATH_AUTO)
 * picks the tensor cores; on the bit-packed path otherwise (early-exit
 * scenarios always).
 *   labels_or_null       : host array of S device pointers (N_s uint8 each, NULL entries
 *                          allowed), or NULL.
 *   counts3xS            : device int64[S*3]; counts are ADDED.
 *   grad_counts_or_null  : host array of S device pointers (n_s*K_s int64 each, NULL entries
 *                          allowed), or NULL; per-state I^L counts are ADDED.
 * Limits: every scenario within the rsr_problem limits and n*(K-1) <= 512.
 *
 * rsr_batch_workspace_size : bytes of the batch workspace for these problems and sample counts
 *                            Ns (host int64[S]; 0 on invalid input).  It includes a deep queue of
 *                            min(Ns[s], 2^22) sample indices per scenario.
 * rsr_batch_prepare        : thresholds, reference encodings, precedence pre-checks and the work
 *                            list (longest scenarios first) into `ws`; not capturable.
 * rsr_batch                : the pair-kernel launch (if any scenario runs on the tensor cores),
 *                            then the bit-packed persistent launches: every (scenario, 256-sample
 *                            tile) walks at most k0 reference chunks, and the samples still
 *                            unresolved then are queued and taken 256 at a time by the later
 *                            launches, one stage to the last chunk or (staged) stages that each
 *                            walk four times as far as they start and queue again (same labels
 *                            and counts as one walk; a tile that would overflow a queue of more
 *                            than 2^22 samples finishes its walk itself).  The arguments must
 *                            equal those given to rsr_batch_prepare (else RSR_ERR_NOT_PREPARED).
 *                            The launches re-arm their own counters, so they can be captured
 *                            once in a CUDA graph and replayed.
 * rsr_batch_profile        : rsr_batch (the same outputs, and it advances the round) with a cycle
 *                            profile of the bit-packed launches: cycles is a device uint64[S*8],
 *                            zeroed by the call (stream-ordered), then per scenario s, at
 *                            [8s + 0..3] for the tile pass and [8s + 4..7] for the later stages:
 *                            tiles (groups of queued samples), and SM clock cycles (clock64 of
 *                            the tile's block, summed over tiles) spent from a tile's start to
 *                            its tables being ready (for an item's first tile: the work counter,
 *                            scenario lookup and table loads), from there to the block's first
 *                            warp having written its samples (Philox sampling and encoding), and
 *                            from there to the tile's end (the reference-chunk walk; an item's
 *                            last tile includes its count flush).  Scenarios on the tensor cores keep zeros.
 *                            Blocks share their SM, so the cycles measure where a block's time
 *                            goes, not SM time; the three parts give the split.
 * rsr_batch_autotune       : first picks the path of every dense RSR_PATH_AUTO scenario by timing
 *                            the pair kernel and the bit-packed kernel on a slice of its samples
 *                            (scenarios of one shape share the timing), then times the first
 *                            pass's chunk budget k0 (0 = no later stage, 2, 4, 8, 16, 32) with
 *                            either one later stage to the end or stages that each walk four
 *                            times as far as they start (staged), then work orders and grid
 *                            sizes, then the first pass's tiles per work item (1, 2, 4, 8
 *                            consecutive 256-sample tiles of a scenario: one work-counter
 *                            atomic, scenario lookup, table load and count flush for all of
 *                            them), on the prepared batch (writing only into the workspace's
 *                            scratch, never the caller's outputs), keeps the fastest for later
 *                            rsr_batch calls and resets the round to 0; chosen (host
 *                            int32[6]): chosen[0] = grid, chosen[1] = order (0 = longest first,
 *                            1 = as given), chosen[2] = k0 (8 until tuned), chosen[3] =
 *                            scenarios on the tensor cores, chosen[4] = staged (0 until tuned),
 *                            chosen[5] = tiles per first-pass item (1 until tuned).
 *                            Synchronises `stream`.  With RSR_TUNE_CACHE set (see rsr_autotune)
 *                            the choices are read from and written to the tuning cache.
 */
RSR_API size_t rsr_batch_workspace_size(const rsr_problem *problems, int32_t S, const int64_t *Ns);
RSR_API int rsr_batch_prepare(const rsr_problem *problems, int32_t S, const uint64_t *seeds,
                              const uint64_t *offsets, const int64_t *Ns, uint8_t *const *labels_or_null,
                              int64_t *counts3xS, int64_t *const *grad_counts_or_null, void *ws,
                              size_t ws_bytes, rsr_stream_t stream);
RSR_API int rsr_batch(const rsr_problem *problems, int32_t S, const uint64_t *seeds, const uint64_t *offsets,
                      const int64_t *Ns, uint8_t *const *labels_or_null, int64_t *counts3xS,
                      int64_t *const *grad_counts_or_null, void *ws, size_t ws_bytes, rsr_stream_t stream);
RSR_API int rsr_batch_profile(const rsr_problem *problems, int32_t S, const uint64_t *seeds,
                              const uint64_t *offsets, const int64_t *Ns, uint8_t *const *labels_or_null,
                              int64_t *counts3xS, int64_t *const *grad_counts_or_null, void *ws, size_t ws_bytes,
                              rsr_stream_t stream, uint64_t *cycles);
RSR_API int rsr_batch_autotune(const rsr_problem *problems, int32_t S, const uint64_t *seeds,
                               const uint64_t *offsets, const int64_t *Ns, uint8_t *const *labels_or_null,
                               int64_t *counts3xS, int64_t *const *grad_counts_or_null, void *ws,
                               size_t ws_bytes, rsr_stream_t stream, int32_t chosen[5]);

/*
 * Gradients of every scenario of a batch from its per-state I^L counts (the
 * same arithmetic as rsr_grad, without Stage-2 corrections): grad_counts[s]
 * (device int64[n_s*K_s], e.g. filled by rsr_batch), Ns[s] samples;
 * grad_out[s], se_out[s] host fp64[n_s*K_s].  One device->host transfer per
 * scenario on `stream`, one synchronisation for the whole batch.
 */
RSR_API int rsr_batch_grad(const rsr_problem *problems, int32_t S, const int64_t *Ns, int64_t *const *grad_counts,
                           double *const *grad_out, double *const *se_out, rsr_stream_t stream);

/*
 * Time both classifier paths on a slice of `problem` (prepared in `ws`; 2^18
 * samples in dense mode, 2^20 in early-exit mode) and remember the faster one
 * for RSR_PATH_AUTO on problems with the same n, K, density flag and
 * reference-count bucket (power of two).  *chosen_path receives it.  When the
 * bit-packed path wins in early-exit mode and `ws` holds a deep queue, its
 * first-pass budget k0 in {0 (one pass), 2, 4, 8, 16} is timed too and
 * remembered for the same shapes (used by rsr_classify whatever the path).
 * Synchronises `stream`.
 * Tuning cache: when the environment variable RSR_TUNE_CACHE names a file,
 * decisions (this one, and those of rsr_batch_autotune) are also kept there as
 * a JSON object {"key": [integers]}, keyed by the device (name and SM count)
 * and the problem shape, read at the first lookup and rewritten on every new
 * decision; RSR_PATH_AUTO then uses a cached decision without timing.
 */
RSR_API int rsr_autotune(const rsr_problem *problem, void *ws, size_t ws_bytes, rsr_stream_t stream,
                         int32_t *chosen_path);

/*
 * Classification for callers that cannot allocate device memory: for example
 * a plugin inside a host application that owns all device memory through its
 * own pool and does not let libraries allocate, a real-time loop whose
 * allocations are fixed at start-up, or a foreign-language caller that reaches
 * this library only through the C ABI and has no device allocator.  The
 * paper has no counterpart: this is a deployment variant of rsr_prepare +
 * rsr_classify on RSR_PATH_POPC (same arguments, same results; problem->path
 * is ignored, problem->flags honoured), not a step of the method.
 * The workspace is a library-owned device array of RSR_STATIC_SCRATCH_BYTES
 * (4 MiB) that every GPU loading librsr holds until the process exits.
 * Problems whose header + thresholds + bit-packed references exceed it are
 * rejected with RSR_ERR_WORKSPACE before any GPU work.  The first call on a
 * device looks up the array's device address once (cudaGetSymbolAddress, with
 * that device current), so make that first call before any stream capture.
 * Asynchronous on `stream`: the sampler thresholds reach the array as a kernel
 * argument, not through a host-to-device copy, so no step waits for it.
 * Every call shares the array and re-initialises what it needs; calls whose
 * GPU work overlaps (other streams, other host threads) race on it, so
 * serialise them.  The library itself calls no allocation routine here.
 */
#define RSR_STATIC_SCRATCH_BYTES (4u << 20)
RSR_API int rsr_classify_static(const rsr_problem *problem, uint64_t seed, uint64_t offset, int64_t N,
                                const uint8_t *samples_or_null, uint8_t *labels_or_null, int64_t *counts3,
                                int64_t *grad_counts_or_null, rsr_stream_t stream);

/*
 * Stage 2 on the device (Sec. 3.5): evaluate the system function Phi for the
 * unclassified samples so that P(S <= m') is estimated without the host.
 * Built-in system functions (the families of the paper's experiments):
 *   RSR_PHI_ST_CONNECTIVITY   K = 2; component i is the undirected edge
 *                             (src[i], dst[i]), working when x_i = 1;
 *                             Phi = 1 iff s reaches t over working edges.
 *   RSR_PHI_ST_MAXFLOW_LEVELS component i is the directed arc src[i] -> dst[i]
 *                             with capacity x_i; Phi = #{l : maxflow(s->t) >= level_thr[l]}
 *                             (level_thr ascending, n_levels <= 8).
 *   RSR_PHI_GLOBAL_CONNECTIVITY  K = 2; edges as for s-t connectivity; Phi = 1 iff
 *                             the working edges connect all n_nodes nodes (Sec. 4.3).
 *   RSR_PHI_GLOBAL_CONN_LEVEL K = 2; Phi = 0 if the working edges leave the nodes
 *                             disconnected, 1 if connected but some working edge is
 *                             a bridge (some pair of nodes has a single
 *                             edge-disjoint path), 2 otherwise (Sec. 4.6).
 * s and t are read by the s-t kinds only but must lie in [0, n_nodes) for every
 * kind.  Limits: n_nodes <= 1024.  src/dst: device int32[n].
 */
#define RSR_PHI_ST_CONNECTIVITY 0
#define RSR_PHI_ST_MAXFLOW_LEVELS 1
#define RSR_PHI_GLOBAL_CONNECTIVITY 2
#define RSR_PHI_GLOBAL_CONN_LEVEL 3

typedef struct rsr_system {
    int32_t kind;
    int32_t n_nodes;
    const int32_t *src;
    const int32_t *dst;
    int32_t s, t;
    int32_t n_levels;
    int32_t level_thr[8];
    int32_t m_prime;
} rsr_system;

/*
 * For every sample with label 2 in labels[0..N) (device, from rsr_classify on
 * samples offset..offset+N-1 of `seed`), regenerate its states, evaluate Phi
 * and relabel it 3 (Phi <= m', i.e. S <= m') or 4 (S >= m'+1).
 *   u_lower_idx : device int64[cap]; the local indices of the 3s are appended in
 *                 no particular order (pass them to rsr_grad).  If more than cap
 *                 samples resolve lower, the extra indices are dropped and the
 *                 workspace error word is set (rsr_workspace_status); counts stay exact.
 *   counts2     : device int64[2], += (#3, #4); n_u_lower for rsr_estimate is counts2[0].
 * Bad node indices in src/dst are dropped and flagged in the error word.
 * Asynchronous on `stream`; `ws` must be prepared for `problem`.
 */
RSR_API int rsr_resolve(const rsr_problem *problem, const rsr_system *system, uint64_t seed, uint64_t offset,
                        int64_t N, uint8_t *labels, int64_t *u_lower_idx, int64_t cap, int64_t *counts2,
                        void *ws, size_t ws_bytes, rsr_stream_t stream);

/*
 * System-state pmf over all levels in one call (Sec. 3.5 applied at every
 * boundary; the multi-state examples of Sec. 4.5-4.6): counts of S = m for
 * m = 0..n_boundaries over samples offset..offset+N-1 of `seed`.
 * Each boundary b (m' = b) classifies every sample against its own reference
 * sets: a lower match bounds S <= b, an upper match S >= b+1.  A sample whose
 * bounds meet is counted directly; for the others Phi is evaluated on the
 * device (decisions Phi <= m' for the open boundaries, lowest first).
 *   problems        : host array[n_boundaries]; problem b holds the references
 *                     of boundary m' = b; all share n, K and the pmf.
 *   ws, ws_bytes    : host arrays[n_boundaries]; ws[b] prepared for problems[b].
 *   system          : Phi (system->m_prime is ignored).  The number of
 *                     boundaries must match Phi: 1 for the binary kinds, 2 for
 *                     RSR_PHI_GLOBAL_CONN_LEVEL, n_levels for max-flow levels.
 *   labels_scratch  : device uint8[n_boundaries*N] (per-boundary labels, 0/1/2).
 *   levels_or_null  : device uint8[N], S of every sample.
 *   counts3_per_boundary : device int64[3*n_boundaries], += the classification
 *                     counts (I^L, I^U, I^u) of each boundary.
 *   level_counts    : device int64[n_boundaries+1], += #{h : S_h = m}.
 *   n_phi_or_null   : device int64[1], += samples that needed Phi.
 * Asynchronous on `stream`.  Inconsistent references (a lower bound below an
 * upper bound for one sample) set the error word of ws[0]; the sample is not counted.
 */
RSR_API int rsr_level_pmf(const rsr_problem *problems, int32_t n_boundaries, void *const *ws,
                          const size_t *ws_bytes, const rsr_system *system, uint64_t seed, uint64_t offset,
                          int64_t N, uint8_t *labels_scratch, uint8_t *levels_or_null,
                          int64_t *counts3_per_boundary, int64_t *level_counts, int64_t *n_phi_or_null,
                          rsr_stream_t stream);

/*
 * Stage 1 building block (Sec. 3.4): componentwise boundary search.  For each
 * j < n_starts, sample offset + starts[j] of `seed` is regenerated (same
 * sampler as rsr_classify).  If Phi(x) <= m' its components are raised one at a
 * time in the visiting order, one state at a time with Phi re-evaluated after
 * each step, until the top state or until a step makes Phi > m' (that step is
 * undone); otherwise they are lowered in the same way while Phi >= m'+1 holds.
 * The final state is a boundary reference state.
 *   order     : RSR_SEARCH_INDEX_ORDER visits components 0, 1, ..., n-1, as the
 *               paper does; RSR_SEARCH_PERMUTED visits them in a per-start
 *               pseudo-random order (not in the paper): a Fisher-Yates shuffle,
 *               for i = n-1 down to 1 swapping i with j = (u*(i+1)) >> 32, u = word
 *               (i mod 4) of Philox4x32-10(key = seed, counter = (h lo, h hi,
 *               floor(i/4), 1)), h = offset + starts[j].  Searches from different
 *               samples then spread over the boundary instead of concentrating on
 *               the states that are extreme in index order.
 *   problem   : n, K, pmf are read (references are not).
 *   starts    : device int64[n_starts], sample indices relative to offset.
 *   refs_out  : device uint8[n_starts*n], row j = the reference found from start j.
 *   side_out  : device uint8[n_starts], 0 = lower reference (S <= m'), 1 = upper.
 *   phi_evals : device int64[1], += number of Phi evaluations (NULL: not counted).
 *   ws        : device, rsr_search_workspace_size(problem) bytes, 256-byte aligned;
 *               the call writes the sampler thresholds into it (not prepared).
 * Asynchronous on `stream`.  Bad node indices set the error word of `ws`.
 */
RSR_API size_t rsr_search_workspace_size(const rsr_problem *problem);
#define RSR_SEARCH_INDEX_ORDER 0
#define RSR_SEARCH_PERMUTED 1
RSR_API int rsr_boundary_search(const rsr_problem *problem, const rsr_system *system, uint64_t seed,
                                uint64_t offset, const int64_t *starts, int64_t n_starts, uint8_t *refs_out,
                                uint8_t *side_out, int64_t *phi_evals, int32_t order, void *ws, size_t ws_bytes,
                                rsr_stream_t stream);

/*
 * Reference-set maintenance (Sec. 2.2, Eqs. (2)-(3): reference sets hold only
 * non-dominated states).  keep[j] = 1 iff no other reference of the set
 * dominates refs[j]: for a lower set (upper = 0) no r_i with r_j <= r_i
 * componentwise, for an upper set no r_i with r_j >= r_i.  Of equal references
 * only the first (lowest index) is kept.
 *   refs    : device uint8[R*n], states in [0, K).
 *   keep    : device uint8[R].   n_keep : device int64[1], += number kept.
 *   scratch : device, rsr_nondominated_scratch_size(n, K, R) bytes, 256-byte aligned.
 * Asynchronous on `stream`.
 */
RSR_API size_t rsr_nondominated_scratch_size(int32_t n, int32_t K, int64_t R);
RSR_API int rsr_nondominated(int32_t n, int32_t K, int64_t R, const uint8_t *refs, int32_t upper, uint8_t *keep,
                             int64_t *n_keep, void *scratch, size_t scratch_bytes, rsr_stream_t stream);

/*
 * Stage 1 on the device (Sec. 3.5, with many searches per round).  Round r
 * classifies samples r*N .. r*N+N-1 of `seed` against the current references
 * and stops when (double)n_u < eps_u * (double)N (n_u = unclassified count),
 * else when R_L + R_U >= R_max, else after max_rounds rounds.  Otherwise the
 * first min(max_starts, n_u, R_max - R_L - R_U) unclassified samples in index
 * order start boundary searches (rsr_boundary_search); the references found are
 * appended to their set in start order and each set is reduced to its
 * non-dominated elements, order kept (rsr_nondominated).
 */
typedef struct rsr_stage1_opts {
    uint64_t seed;          /* Philox stream of the rounds                          */
    int64_t N;              /* samples per round (the paper's H)                     */
    int64_t max_starts;     /* boundary searches per round, >= 1                     */
    double eps_u;           /* target unclassified fraction                          */
    int64_t R_max;          /* reference limit; each buffer holds R_max rows         */
    int32_t max_rounds;     /* >= 1                                                  */
    int32_t search_order;   /* RSR_SEARCH_INDEX_ORDER or RSR_SEARCH_PERMUTED         */
} rsr_stage1_opts;

typedef struct rsr_stage1_result {
    int32_t rounds;         /* rounds classified                                     */
    int32_t stop;           /* 0 = eps_u reached, 1 = R_max reached, 2 = max_rounds  */
    int64_t R_L, R_U;       /* rows now held in ref_L_buf / ref_U_buf                */
    int64_t n_u_last;       /* unclassified samples of the last round                */
    int64_t phi_evals;      /* Phi evaluations of all searches                       */
} rsr_stage1_result;

/*
 *   problem   : n, K, pmf, path, flags; R_L / R_U = rows already in the buffers
 *               (initial references, may be 0); problem->ref_L / ref_U are ignored.
 *   system    : Phi and m' (system->m_prime).
 *   ref_L_buf, ref_U_buf : device uint8[R_max*n] each, updated in place.
 *   history_or_null : host int64[4*max_rounds]; row r = (n_u, R_L, R_U, starts)
 *               at the start of round r.
 *   ws        : device, rsr_stage1_workspace_size(problem, opts) bytes, 256-aligned.
 * Synchronous: returns when Stage 1 has stopped.  Returns RSR_ERR_TIMEOUT if a
 * classification round reported a device timeout, RSR_ERR_INVALID_ARG if a system
 * kernel reported bad input (error word of the workspace).
 */
RSR_API size_t rsr_stage1_workspace_size(const rsr_problem *problem, const rsr_stage1_opts *opts);
RSR_API int rsr_stage1(const rsr_problem *problem, const rsr_system *system, const rsr_stage1_opts *opts,
                       uint8_t *ref_L_buf, uint8_t *ref_U_buf, int64_t *history_or_null,
                       rsr_stage1_result *result, void *ws, size_t ws_bytes, rsr_stream_t stream);

/*
 * Measured integer throughput of the current GPU, for the roofline of the
 * bit-packed classifiers (not a step of the method; the paper has no
 * counterpart).  Runs two short kernels on a full grid, each with eight
 * independent chains per thread: three-input logic ops (LOP3, the classifiers'
 * and-or test) and 32x32->64 multiply-adds (the products of Philox4x32-10).
 *   lop3_ops_per_s, imad_ops_per_s : host double[1] each, set to thread-ops per second.
 * Synchronous (waits for its own kernels on `stream`); allocates nothing.
 */
RSR_API int rsr_measure_int_peak(double *lop3_ops_per_s, double *imad_ops_per_s, rsr_stream_t stream);

/*
 * Measured rate of the samplers' generator on the current GPU (not a step of
 * the method): Philox4x32-10 blocks per second on a full grid (8 blocks of 256
 * threads per SM, eight independent counters per thread), the library's own
 * implementation, timed on the second of two launches.
 *   blocks_per_s : host double[1].
 * Synchronous (waits for its own kernels on `stream`); allocates nothing.
 */
RSR_API int rsr_measure_philox_rate(double *blocks_per_s, rsr_stream_t stream);

/*
 * Measured dense FP8 tensor-core rate of the current GPU, for the roofline of
 * the tensor-core classifiers (not a step of the method; the paper has no
 * counterpart).  One CTA per SM issues tcgen05.mma.kind::f8f6f4 (K = 32, E4M3
 * operands resident in shared memory, FP32 accumulators in tensor memory)
 * back to back, with no copies and no epilogue.
 *   cta_pair          : 0 = cta_group::1, M = 128 x N = 256 per CTA (as the
 *                       early-exit classifier); 1 = cta_group::2 on clusters
 *                       of two CTAs, M = 256 x N = 256 per pair (as the dense
 *                       classifier).  Either way 2*128*256*32 flop per CTA per
 *                       instruction.
 *   seconds           : length of the sustained run, in [0, 60]; 0 skips it.
 *   burst_flops_per_s : host double[1], the fastest of five single launches of
 *                       about 16 ms each (after one warm-up launch).
 *   sustained_flops_per_s : host double[1], launches back to back for about
 *                       `seconds` (0.0 when skipped).
 * Synchronous (waits for its own kernels on `stream`); allocates nothing.
 * RSR_ERR_UNSUPPORTED on a GPU without tcgen05; RSR_ERR_TIMEOUT if a final
 * bounded wait for the issued MMAs ran out.
 */
RSR_API int rsr_measure_fp8_peak(int32_t cta_pair, double seconds, double *burst_flops_per_s,
                                 double *sustained_flops_per_s, rsr_stream_t stream);

/* Message for a status code (static storage). */
RSR_API const char *rsr_status_string(int status);

/* Text of the last CUDA error seen by this thread inside the library. */
RSR_API const char *rsr_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RSR_H */
