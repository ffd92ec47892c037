// rsr_launch.h -- host-side launchers of librsr's kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rsr_internal.cuh"

namespace rsr {

// Word bucket used by the bit-packed kernels for `words` 32-bit words.
int popc_word_bucket(int words);

// Preparation (prep_kernels.cu).
cudaError_t launch_encode_popc(const uint8_t *refs, int64_t R, int n, int km1, int words_b,
                               bool complement, uint32_t *out, cudaStream_t s, const int32_t *perm = nullptr);
// Component-major index of the upper set (popc_index.cuh) from its bit-packed rows,
// slot r taking row perm[r] (identity if perm is NULL), and the per-chunk AND rows.
cudaError_t launch_encode_index(const uint32_t *popc_U, const int32_t *perm, int64_t R_U, int words_b, int kenc,
                                uint32_t *out_index, uint32_t *out_and, cudaStream_t s);
// Clustering keys of the upper references (bits at the positions of kb, most significant first).
struct KeyBits {
    int32_t nbits;
    int16_t pos[32];
};
cudaError_t launch_cluster_keys(const uint32_t *popc_U, int64_t R_U, int words_b, const KeyBits &kb, uint32_t *keys,
                                cudaStream_t s);
cudaError_t launch_score_refs(const uint8_t *refs, int64_t R, int n, int K, const float *table, float *score,
                              cudaStream_t s);
cudaError_t launch_overlap(const uint32_t *popc_L, int64_t R_L, const uint32_t *popc_U, int64_t R_U,
                           int words_b, WsHeader *hdr, cudaStream_t s);
cudaError_t launch_sample(const ClassifyParams &p, uint8_t *states, cudaStream_t s);
cudaError_t launch_grad_correction(const ClassifyParams &p, const int64_t *idx, int64_t m,
                                   cudaStream_t s);

// Classification (classify_popc.cu, classify_tc.cu).
cudaError_t launch_classify_popc(const ClassifyParams &p, cudaStream_t s);
cudaError_t launch_encode_tc(const uint8_t *refs, int64_t R, int64_t rows_padded, int n, int km1,
                             int kpad, bool upper, uint8_t *out, cudaStream_t s, const int32_t *perm = nullptr);
cudaError_t launch_classify_tc(const ClassifyParams &p, cudaStream_t s);   // dense: the pair kernel below
cudaError_t launch_classify_tc2(const ClassifyParams &p, cudaStream_t s);  // dense, CTA pairs (cta_group::2)
bool tc2_available(int kpad);   // the pair kernel runs on this device for rows of kpad bytes
// The tensor-core scenarios of a batch on the pair kernel: items [begin[s], begin[s+1]) are
// scenario s's pair blocks of 256 samples; descs[s].offset is moved by round*N.
cudaError_t launch_classify_tc2_batch(const ClassifyParams *descs, const int64_t *begin, int S, int64_t total_items,
                                      const unsigned long long *round, int kp_max, int nthr_max, cudaStream_t s);
bool tc_supported();
int tc_max_kpad();

// Stage 2 (resolve.cu).
cudaError_t launch_resolve(const ClassifyParams &p, const rsr_system &sys, uint8_t *labels, int64_t *u_lower_idx,
                           int64_t cap, unsigned long long *counts2, cudaStream_t s);
int resolve_max_nodes();
cudaError_t launch_levels(const ClassifyParams &p, const rsr_system &sys, int nb, const uint8_t *labels,
                          uint8_t *levels_out, unsigned long long *level_counts, unsigned long long *n_phi,
                          cudaStream_t s);
cudaError_t launch_search(const ClassifyParams &p, const rsr_system &sys, const int64_t *starts, int64_t n_starts,
                          uint8_t *refs_out, uint8_t *side_out, unsigned long long *evals, int order_mode,
                          cudaStream_t s);

// Reference-set maintenance and order-preserving selection (maintain.cu).
cudaError_t launch_nondominated(const uint32_t *enc, int64_t R, int words_b, bool upper, uint8_t *keep,
                                unsigned long long *n_keep, cudaStream_t s);
// The same keep mask when rows [0, R_old) are already non-dominated among themselves.
cudaError_t launch_nondominated_appended(const uint32_t *enc, int64_t R_old, int64_t R, int words_b, bool upper,
                                         uint8_t *keep, unsigned long long *n_keep, cudaStream_t s);
size_t select_scratch_bytes(int64_t N);
cudaError_t launch_select(const uint8_t *flags, uint8_t value, int64_t N, int64_t limit, int64_t *out_idx,
                          int64_t *n_out, int64_t *scratch, cudaStream_t s);
cudaError_t launch_gather_rows(const uint8_t *src, const int64_t *idx, int64_t count, int n, uint8_t *dst,
                               cudaStream_t s);

// Host helpers of the C ABI (rsr_capi.cu).
int validate_problem(const rsr_problem *p);              // every rsr_problem check; RSR_OK or an error code
int validate_states(int n, int K, const double *pmf);   // sizes and pmf rows; RSR_OK or an error code
int validate_system(const rsr_system *system, int K);    // built-in Phi arguments
void host_thresholds(int n, int K, const double *pmf, unsigned long long *T);   // n*(K-1) values
int cuda_fail(cudaError_t e, const char *where);          // records the error, returns RSR_ERR_CUDA

int device_sm_count();

}  // namespace rsr
