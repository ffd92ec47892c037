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
    const int32_t *overlap;              // precedence pre-check result
    uint8_t *labels;                     // [N] or NULL
    unsigned long long *counts3;         // [3]
    unsigned long long *grad_counts;     // [n*K] or NULL
    uint32_t *bitcnt;                    // [n*(K-1)] I^L per-bit scratch, or NULL
    unsigned long long *lcount;          // I^L count scratch
};

// Work counter and round of a batch workspace (256 bytes at its start).
struct BatchHeader {
    unsigned long long next_item;
    unsigned int blocks_done;
    unsigned int pad;
    unsigned long long round;       // launches since prepare: sample window index
    unsigned long long reserved[29];
};
static_assert(sizeof(BatchHeader) == 256, "batch header is one 256-byte line");

size_t batch_kernel_smem();
int batch_max_words();
cudaError_t batch_max_grid(int *blocks_per_sm);
cudaError_t launch_batch(const BatchDesc *descs, const int64_t *item_begin, int S, int64_t total_items,
                         BatchHeader *hdr, int grid, cudaStream_t s);

}  // namespace rsr
