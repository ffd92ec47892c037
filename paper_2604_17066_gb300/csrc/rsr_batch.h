// rsr_batch.h -- device-visible structures of the batched launch (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rsr {

// One scenario of a batch, as the persistent kernel sees it.
struct BatchDesc {
    int32_t n, K, km1, words_b;
    int64_t R_L, R_U;
    uint64_t seed, offset;
    int64_t N;
    const unsigned long long *thr;       // [n*(K-1)]
    const uint32_t *popc_L, *popc_U;     // [R][words_b]
    const uint32_t *popc_UT;             // component-major index of the upper set, or NULL
    const uint32_t *popc_UA;             // per index chunk: AND of its references
    const uint32_t *popc_LG;             // per lower chunk: AND row and guard row ([2][words_b]), or NULL
    const int32_t *overlap;              // precedence pre-check result
    uint8_t *labels;                     // [N] or NULL
    unsigned long long *counts3;         // [3]
    unsigned long long *grad_counts;     // [n*K] or NULL
    uint32_t *bitcnt;                    // [n*(K-1)] I^L per-bit scratch, or NULL
    unsigned long long *lcount;          // I^L count scratch
    int64_t *deep;                       // [2][deep_cap] two queues: local indices of deferred samples
    unsigned long long *deep_count;      // [2] samples appended to each queue (may exceed deep_cap)
    int64_t deep_cap;                    // entries per queue
    int32_t k0;                          // chunk steps of the first pass (0 = all)
    int32_t staged;                      // later stages grow by kDeferGrowth (0: one stage to the end)
    int32_t path;                        // RSR_PATH_POPC, or RSR_PATH_TC: the scenario runs on the pair kernel
    int32_t id;                          // the scenario's index in the caller's arrays (descriptors are in work order)
    int32_t tiles;                       // first pass: consecutive 256-sample tiles per work item (>= 1)
    int32_t pad_;
};

// Work counter and round of a batch workspace (256 bytes at its start).
struct BatchHeader {
    unsigned long long next_item;   // first pass: work counter
    unsigned int blocks_done;       // first pass: finished blocks
    unsigned int blocks_done2;      // later stages: finished blocks
    unsigned long long round;       // launch sets since prepare: sample window index
    unsigned long long next_deep;   // later stages: work counter
    long long deep_total;           // the next stage's items (groups of 256 queued samples)
    unsigned long long reserved[27];
};
static_assert(sizeof(BatchHeader) == 256, "batch header is one 256-byte line");

size_t batch_kernel_smem();
int batch_max_words();
cudaError_t batch_max_grid(int *blocks_per_sm);
// The tile pass, then n_stages stages over the queued deep samples (deep_begin:
// workspace int64[S+1], written by the launch before each stage).  prof: null,
// or a device [S][8] cycle profile the launches add to (per scenario: first
// pass items, set-up, sampling and walk cycles, then the same for later stages).
cudaError_t launch_batch(const BatchDesc *descs, const int64_t *item_begin, int S, int64_t total_items,
                         BatchHeader *hdr, int64_t *deep_begin, int n_stages, int grid, cudaStream_t s,
                         unsigned long long *prof = nullptr);
// The profiled variant (batch_prof.cu): its shared-memory attributes (lowering
// *blocks_per_sm to its occupancy) and its launches (prof non-null).
cudaError_t batch_prof_attributes(int *blocks_per_sm);
cudaError_t launch_batch_prof(const BatchDesc *descs, const int64_t *item_begin, int S, int64_t total_items,
                              BatchHeader *hdr, int64_t *deep_begin, int n_stages, int grid, cudaStream_t s,
                              unsigned long long *prof);
// Stages after the tile pass for these descriptors (host copies): the most any
// bit-packed scenario needs (staged_passes() - 1), at least one.
int batch_stages(const BatchDesc *descs, int S);
constexpr int64_t kBatchDeepCap = int64_t(1) << 22;   // deep-queue entries per scenario at most (32 MB)
constexpr int64_t kBatchTestDeepCap = 1024;           // with RSR_FLAG_TEST_DEEP_CAP (test hook)
constexpr int kBatchMaxTiles = 8;          // first-pass tiles per work item that rsr_batch_autotune tries (1, 2, 4, 8)
constexpr int kBatchDefaultK0 = 8;         // first-pass chunk steps before rsr_batch_autotune picks them

}  // namespace rsr
