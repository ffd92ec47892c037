// batch.cu -- many classification problems (hazard scenarios) in one
// persistent launch per pass (the kernels are in batch_kernels.cuh; this file
// launches them without the cycle profile).
//
// Each scenario s has its own n, K, pmf thresholds, reference sets, sample
// count N_s, seed and offset.  First-pass work items are (scenario, run of
// d.tiles consecutive 256-sample tiles), enumerated scenario by scenario in the
// order the host chose (longest scenarios first); a persistent grid pulls items
// from an atomic counter, so short and long scenarios share the machine without
// per-scenario launch tails.  Per tile the block runs the same bit-packed test as classify_popc.cu
// (Sec. 3.3, Algorithm 1) for the scenario's word count.  Scenarios whose upper
// set has a component-major index (popc_index.cuh) test their upper chunks
// through it, after a direct test of their kHot most probable upper references.
//
// Staged passes.  The 256 samples of a tile walk the reference chunks together
// (one shared copy of each chunk), so a tile costs as many chunk steps as its
// deepest sample needs, and in scenarios with partial reference sets every
// tile holds a few samples that match nothing and visit every chunk while the
// other lanes idle.  The first pass (batch_kernel) therefore walks at most k0
// chunks per tile; samples still unresolved then are appended to their
// scenario's deep queue (a block-wide reservation; a tile whose reservation
// would overflow the queue keeps walking itself).  The later stages
// (batch_deep_kernel) take the queued samples 256 at a time, regenerate their
// states from Philox, and resume the walk where the previous stage stopped
// with every lane busy: either one stage to the last chunk, or (a staged
// scenario) stages that each walk four times as far as they start and queue
// again into the other of the scenario's two queues.  Labels, counts and
// gradient counts are the same as one pass would give: the visiting order of
// the chunks is the same, and a sample is counted once, in the pass that
// resolves it.  k0 = 0 runs everything in the first pass.  I^L per-bit counts
// go to a scenario scratch counter; the last block of the final stage converts
// them into the per-state gradient counts, zeroes the scratch and the queues,
// resets the work counters and advances the round, so the same launches can be
// replayed (e.g. from a CUDA graph) on the next N_s samples of every scenario
// without any host work.
#include "batch_kernels.cuh"

namespace rsr {

size_t batch_kernel_smem() { return batch_smem_bytes(); }

int batch_max_words() { return kMaxWB; }

cudaError_t batch_max_grid(int *blocks_per_sm) {
    int occ = 1 << 30;
    cudaError_t e = batch_variant_attributes<false>(&occ);
    if (e == cudaSuccess) e = batch_prof_attributes(&occ);
    if (e != cudaSuccess) return e;
    *blocks_per_sm = occ;
    return cudaSuccess;
}

// The shared-memory attributes are set by batch_max_grid() (called when a
// batch is prepared), so a launch issues nothing but the kernels and can be
// captured.  The final stage always runs: it also closes the round.
cudaError_t launch_batch(const BatchDesc *descs, const int64_t *item_begin, int S, int64_t total_items,
                         BatchHeader *hdr, int64_t *deep_begin, int n_stages, int grid, cudaStream_t s,
                         unsigned long long *prof) {
    if (grid <= 0) grid = 1;   // every launch runs even without bit-packed items: the last closes the round
    if (n_stages < 1) n_stages = 1;
    if (prof) return launch_batch_prof(descs, item_begin, S, total_items, hdr, deep_begin, n_stages, grid, s, prof);
    return batch_variant_launch<false>(descs, item_begin, S, total_items, hdr, deep_begin, n_stages, grid, s,
                                       nullptr);
}

int batch_stages(const BatchDesc *descs, int S) {
    int stages = 1;
    for (int k = 0; k < S; ++k) {
        if (descs[k].path == RSR_PATH_TC) continue;   // on the pair kernel
        const int64_t nsteps = (descs[k].R_U + kChunk - 1) / kChunk + (descs[k].R_L + kChunk - 1) / kChunk;
        stages = std::max(stages, descs[k].staged ? staged_passes(nsteps, descs[k].k0) - 1 : 1);
    }
    return stages;
}

}  // namespace rsr
