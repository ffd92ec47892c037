// batch_prof.cu -- the batched persistent kernels with the cycle profile
// (rsr_batch_profile): the same kernels as batch.cu, with thread 0 of each
// block reading clock64 at an item's start, when its tables are ready, when
// warp 0 has written its samples and when the item's counts are flushed, and
// adding the three spans to its scenario's row.  A translation unit of its own
// so that it compiles beside batch.cu.
#include "batch_kernels.cuh"

namespace rsr {

cudaError_t batch_prof_attributes(int *blocks_per_sm) { return batch_variant_attributes<true>(blocks_per_sm); }

cudaError_t launch_batch_prof(const BatchDesc *descs, const int64_t *item_begin, int S, int64_t total_items,
                              BatchHeader *hdr, int64_t *deep_begin, int n_stages, int grid, cudaStream_t s,
                              unsigned long long *prof) {
    return batch_variant_launch<true>(descs, item_begin, S, total_items, hdr, deep_begin, n_stages, grid, s, prof);
}

}  // namespace rsr
