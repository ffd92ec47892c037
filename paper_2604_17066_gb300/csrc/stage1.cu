// stage1.cu -- Stage 1 of the RSR workflow on the device (Sec. 3.4-3.5):
// rsr_boundary_search (the componentwise search from chosen samples),
// rsr_nondominated (reference-set maintenance, Eqs. (2)-(3)) and rsr_stage1,
// the round loop that alternates classification and search until the
// unclassified fraction falls below eps_u or the reference limit is reached.
//
// The paper draws one unclassified sample per iteration; here a round starts
// up to max_starts searches at once (the first unclassified samples in index
// order, which are a uniform random choice because the samples are i.i.d.),
// so references found in the same round can coincide and each set is reduced
// to its non-dominated elements after the round.  Every step runs in kernels;
// the host only moves counts (a few int64 per round) and makes decisions.
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "rsr.h"
#include "rsr_internal.cuh"
#include "rsr_launch.h"

namespace rsr {
namespace {

#define S1_CUDA(call)                                          \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
    } while (0)

constexpr size_t kAlign = 256;

size_t up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int words_bucket(int n, int K) { return popc_word_bucket((n * (K - 1) + 31) / 32); }

// Search workspace: header (error word), an evaluation counter, thresholds.
constexpr size_t kSearchOffEvals = sizeof(WsHeader);
constexpr size_t kSearchOffThr = 512;

size_t search_ws_bytes(int n, int K) { return kSearchOffThr + up((size_t)n * (K - 1) * sizeof(unsigned long long)); }

struct S1Layout {
    size_t cls_bytes = 0;   // classification workspace sized for R_max rows per set, at offset 0
    size_t off_search = 0, search_bytes = 0;
    size_t off_labels = 0, off_counts = 0, off_starts = 0, off_side = 0, off_new = 0, off_sel = 0, off_keep = 0,
           off_tmp = 0, off_enc = 0, off_selscr = 0, off_scal = 0;
    size_t total = 0;
};

S1Layout s1_layout(const rsr_problem *p, const rsr_stage1_opts *o) {
    S1Layout L;
    rsr_problem q = *p;
    static const uint8_t dummy = 0;
    q.R_L = o->R_max;
    q.R_U = o->R_max;
    q.ref_L = &dummy;
    q.ref_U = &dummy;
    L.cls_bytes = up(rsr_workspace_size(&q, o->N));
    if (L.cls_bytes == 0) return L;
    const int n = p->n, K = p->K;
    const int64_t B = o->max_starts, R = o->R_max, N = o->N;
    size_t off = L.cls_bytes;
    L.off_search = off;
    L.search_bytes = search_ws_bytes(n, K);
    off += up(L.search_bytes);
    L.off_labels = off;
    off += up((size_t)N);
    L.off_counts = off;
    off += up(3 * sizeof(int64_t));
    L.off_starts = off;
    off += up((size_t)B * sizeof(int64_t));
    L.off_side = off;
    off += up((size_t)B);
    L.off_new = off;
    off += up((size_t)B * n);
    L.off_sel = off;
    off += up((size_t)std::max(B, R) * sizeof(int64_t));
    L.off_keep = off;
    off += up((size_t)R);
    L.off_tmp = off;
    off += up((size_t)R * n);
    L.off_enc = off;
    off += up((size_t)R * words_bucket(n, K) * sizeof(uint32_t));
    L.off_selscr = off;
    off += up(select_scratch_bytes(std::max(std::max(N, R), B)));
    L.off_scal = off;
    off += up(4 * sizeof(int64_t));
    L.total = off;
    return L;
}

int check_opts(const rsr_problem *p, const rsr_stage1_opts *o) {
    if (!p || !o) return RSR_ERR_INVALID_ARG;
    if (o->N < 1 || o->max_starts < 1 || o->R_max < 1 || o->max_rounds < 1 || !(o->eps_u >= 0.0))
        return RSR_ERR_INVALID_ARG;
    if (o->search_order != RSR_SEARCH_INDEX_ORDER && o->search_order != RSR_SEARCH_PERMUTED)
        return RSR_ERR_INVALID_ARG;
    if (o->R_max >= (int64_t(1) << 31)) return RSR_ERR_UNSUPPORTED;
    if (p->R_L < 0 || p->R_U < 0 || p->R_L > o->R_max || p->R_U > o->R_max) return RSR_ERR_INVALID_ARG;
    if (p->path < RSR_PATH_AUTO || p->path > RSR_PATH_TC) return RSR_ERR_INVALID_ARG;
    return validate_states(p->n, p->K, p->pmf);
}

}  // namespace
}  // namespace rsr

using namespace rsr;

extern "C" {

size_t rsr_search_workspace_size(const rsr_problem *problem) {
    if (!problem || validate_states(problem->n, problem->K, problem->pmf) != RSR_OK) return 0;
    return search_ws_bytes(problem->n, problem->K);
}

int rsr_boundary_search(const rsr_problem *problem, const rsr_system *system, uint64_t seed, uint64_t offset,
                        const int64_t *starts, int64_t n_starts, uint8_t *refs_out, uint8_t *side_out,
                        int64_t *phi_evals, int32_t order, void *ws, size_t ws_bytes, rsr_stream_t stream) {
    if (!problem) return RSR_ERR_INVALID_ARG;
    if (order != RSR_SEARCH_INDEX_ORDER && order != RSR_SEARCH_PERMUTED) return RSR_ERR_INVALID_ARG;
    int st = validate_states(problem->n, problem->K, problem->pmf);
    if (st != RSR_OK) return st;
    if ((st = validate_system(system, problem->K)) != RSR_OK) return st;
    if (n_starts < 0 || (n_starts > 0 && (!starts || !refs_out || !side_out))) return RSR_ERR_INVALID_ARG;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < search_ws_bytes(problem->n, problem->K))
        return RSR_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(ws);
    std::vector<unsigned long long> T((size_t)problem->n * (problem->K - 1));
    host_thresholds(problem->n, problem->K, problem->pmf, T.data());
    S1_CUDA(cudaMemsetAsync(base, 0, kSearchOffThr, s));
    // pageable source: staged before the call returns
    S1_CUDA(cudaMemcpyAsync(base + kSearchOffThr, T.data(), T.size() * sizeof(T[0]), cudaMemcpyHostToDevice, s));
    if (n_starts == 0) return RSR_OK;
    ClassifyParams c{};
    c.n = problem->n;
    c.K = problem->K;
    c.km1 = problem->K - 1;
    c.thr = reinterpret_cast<const unsigned long long *>(base + kSearchOffThr);
    c.hdr = reinterpret_cast<WsHeader *>(base);
    c.seed = seed;
    c.offset = offset;
    unsigned long long *ev = phi_evals ? reinterpret_cast<unsigned long long *>(phi_evals)
                                       : reinterpret_cast<unsigned long long *>(base + kSearchOffEvals);
    S1_CUDA(launch_search(c, *system, starts, n_starts, refs_out, side_out, ev, order, s));
    return RSR_OK;
}

size_t rsr_nondominated_scratch_size(int32_t n, int32_t K, int64_t R) {
    if (n < 1 || K < 2 || K > kMaxK || (int64_t)n * (K - 1) > kMaxKenc || R < 0) return 0;
    return up((size_t)std::max<int64_t>(R, 1) * words_bucket(n, K) * sizeof(uint32_t));
}

int rsr_nondominated(int32_t n, int32_t K, int64_t R, const uint8_t *refs, int32_t upper, uint8_t *keep,
                     int64_t *n_keep, void *scratch, size_t scratch_bytes, rsr_stream_t stream) {
    if (n < 1 || K < 2 || R < 0 || !n_keep || (R > 0 && (!refs || !keep))) return RSR_ERR_INVALID_ARG;
    if (K > kMaxK || (int64_t)n * (K - 1) > kMaxKenc) return RSR_ERR_UNSUPPORTED;
    if (!scratch || (reinterpret_cast<uintptr_t>(scratch) & 255u) != 0 ||
        scratch_bytes < rsr_nondominated_scratch_size(n, K, R))
        return RSR_ERR_WORKSPACE;
    if (R == 0) return RSR_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int wb = words_bucket(n, K);
    uint32_t *enc = static_cast<uint32_t *>(scratch);
    S1_CUDA(launch_encode_popc(refs, R, n, K - 1, wb, false, enc, s));
    S1_CUDA(launch_nondominated(enc, R, wb, upper != 0, keep, reinterpret_cast<unsigned long long *>(n_keep), s));
    return RSR_OK;
}

size_t rsr_stage1_workspace_size(const rsr_problem *problem, const rsr_stage1_opts *opts) {
    if (check_opts(problem, opts) != RSR_OK) return 0;
    return s1_layout(problem, opts).total;
}

int rsr_stage1(const rsr_problem *problem, const rsr_system *system, const rsr_stage1_opts *opts,
               uint8_t *ref_L_buf, uint8_t *ref_U_buf, int64_t *history_or_null, rsr_stage1_result *result,
               void *ws, size_t ws_bytes, rsr_stream_t stream) {
    int st = check_opts(problem, opts);
    if (st != RSR_OK) return st;
    if ((st = validate_system(system, problem->K)) != RSR_OK) return st;
    if (!ref_L_buf || !ref_U_buf || !result) return RSR_ERR_INVALID_ARG;
    const S1Layout Lw = s1_layout(problem, opts);
    if (Lw.total == 0) return RSR_ERR_INVALID_ARG;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < Lw.total) return RSR_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(ws);
    const int n = problem->n, K = problem->K, wb = words_bucket(n, K);
    const int64_t N = opts->N;
    void *ws_cls = base;
    void *ws_search = base + Lw.off_search;
    uint8_t *labels = reinterpret_cast<uint8_t *>(base + Lw.off_labels);
    int64_t *counts = reinterpret_cast<int64_t *>(base + Lw.off_counts);
    int64_t *starts = reinterpret_cast<int64_t *>(base + Lw.off_starts);
    uint8_t *side = reinterpret_cast<uint8_t *>(base + Lw.off_side);
    uint8_t *fresh = reinterpret_cast<uint8_t *>(base + Lw.off_new);
    int64_t *sel = reinterpret_cast<int64_t *>(base + Lw.off_sel);
    uint8_t *keep = reinterpret_cast<uint8_t *>(base + Lw.off_keep);
    uint8_t *tmp = reinterpret_cast<uint8_t *>(base + Lw.off_tmp);
    uint32_t *enc = reinterpret_cast<uint32_t *>(base + Lw.off_enc);
    int64_t *selscr = reinterpret_cast<int64_t *>(base + Lw.off_selscr);
    int64_t *scal = reinterpret_cast<int64_t *>(base + Lw.off_scal);   // [0] selected, [1] kept, [2] Phi evals
    const WsHeader *hdr_cls = reinterpret_cast<const WsHeader *>(ws_cls);
    const WsHeader *hdr_search = reinterpret_cast<const WsHeader *>(ws_search);

    S1_CUDA(cudaMemsetAsync(scal, 0, 4 * sizeof(int64_t), s));
    int64_t RL = problem->R_L, RU = problem->R_U, n_u = 0;
    // A side's rows are non-dominated among themselves once it has been reduced (an
    // empty side trivially); from then on only the rows a round appends need testing.
    bool reduced[2] = {RL == 0, RU == 0};
    int32_t stop = 2, rounds = 0;
    auto fetch = [&](const void *dev, void *host, size_t bytes) -> int {
        S1_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s));
        S1_CUDA(cudaStreamSynchronize(s));
        return RSR_OK;
    };
    for (int32_t r = 0; r < opts->max_rounds; ++r) {
        const uint64_t off = (uint64_t)r * (uint64_t)N;
        rounds = r + 1;
        if (RL + RU == 0) {
            S1_CUDA(cudaMemsetAsync(labels, 2, (size_t)N, s));   // no references: every sample unclassified
            n_u = N;
        } else {
            rsr_problem q = *problem;
            q.R_L = RL;
            q.R_U = RU;
            q.ref_L = ref_L_buf;
            q.ref_U = ref_U_buf;
            if ((st = rsr_prepare(&q, ws_cls, Lw.cls_bytes, stream)) != RSR_OK) return st;
            S1_CUDA(cudaMemsetAsync(counts, 0, 3 * sizeof(int64_t), s));
            if ((st = rsr_classify(&q, opts->seed, off, N, nullptr, labels, counts, nullptr, nullptr, ws_cls,
                                   Lw.cls_bytes, stream)) != RSR_OK)
                return st;
            int64_t c3[3];
            int32_t err = 0;
            S1_CUDA(cudaMemcpyAsync(&err, &hdr_cls->error, sizeof(err), cudaMemcpyDeviceToHost, s));
            if ((st = fetch(counts, c3, sizeof(c3))) != RSR_OK) return st;
            if (err < 0) return err;
            if (err > 0) return RSR_ERR_INVALID_ARG;
            n_u = c3[2];
        }
        const int64_t R = RL + RU;
        int64_t S = std::min(std::min(opts->max_starts, n_u), opts->R_max - R);
        const bool converged = (double)n_u < opts->eps_u * (double)N;
        const bool full = R >= opts->R_max;
        if (converged || full) S = 0;
        if (history_or_null) {
            int64_t *h = history_or_null + 4 * (size_t)r;
            h[0] = n_u;
            h[1] = RL;
            h[2] = RU;
            h[3] = S;
        }
        if (converged) {
            stop = 0;
            break;
        }
        if (full) {
            stop = 1;
            break;
        }
        S1_CUDA(launch_select(labels, 2, N, S, starts, &scal[0], selscr, s));
        if ((st = rsr_boundary_search(problem, system, opts->seed, off, starts, S, fresh, side, &scal[2],
                                      opts->search_order, ws_search, Lw.search_bytes, stream)) != RSR_OK)
            return st;
        for (int v = 0; v < 2; ++v) {
            int64_t c = 0;
            S1_CUDA(launch_select(side, (uint8_t)v, S, S, sel, &scal[0], selscr, s));
            if ((st = fetch(&scal[0], &c, sizeof(c))) != RSR_OK) return st;
            if (c == 0) continue;
            uint8_t *buf = v ? ref_U_buf : ref_L_buf;
            int64_t &Rs = v ? RU : RL;
            S1_CUDA(launch_gather_rows(fresh, sel, c, n, buf + (size_t)Rs * n, s));
            const int64_t total = Rs + c;
            S1_CUDA(launch_encode_popc(buf, total, n, K - 1, wb, false, enc, s));
            S1_CUDA(cudaMemsetAsync(&scal[1], 0, sizeof(int64_t), s));
            if (reduced[v])
                S1_CUDA(launch_nondominated_appended(enc, Rs, total, wb, v == 1, keep,
                                                     reinterpret_cast<unsigned long long *>(&scal[1]), s));
            else
                S1_CUDA(launch_nondominated(enc, total, wb, v == 1, keep,
                                            reinterpret_cast<unsigned long long *>(&scal[1]), s));
            reduced[v] = true;
            int64_t kept = 0;
            S1_CUDA(launch_select(keep, 1, total, total, sel, &scal[0], selscr, s));
            if ((st = fetch(&scal[0], &kept, sizeof(kept))) != RSR_OK) return st;
            S1_CUDA(launch_gather_rows(buf, sel, kept, n, tmp, s));
            S1_CUDA(cudaMemcpyAsync(buf, tmp, (size_t)kept * n, cudaMemcpyDeviceToDevice, s));
            Rs = kept;
        }
        int32_t err = 0;
        if ((st = fetch(&hdr_search->error, &err, sizeof(err))) != RSR_OK) return st;
        if (err != 0) return RSR_ERR_INVALID_ARG;
    }
    int64_t evals = 0;
    if ((st = fetch(&scal[2], &evals, sizeof(evals))) != RSR_OK) return st;
    result->rounds = rounds;
    result->stop = stop;
    result->R_L = RL;
    result->R_U = RU;
    result->n_u_last = n_u;
    result->phi_evals = evals;
    return RSR_OK;
}

}  // extern "C"
