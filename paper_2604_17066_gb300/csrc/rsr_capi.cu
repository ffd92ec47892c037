// rsr_capi.cu -- the extern "C" entry points of librsr (declared in include/rsr.h).
//
// Host responsibilities: argument checks, the sampler thresholds (fp64 -> integer,
// computed here on the CPU), workspace layout, a registry of prepared
// workspaces, kernel dispatch, and the fp64 estimators (Sec. 3.3 count
// estimators and c.o.v.; Sec. 3.5 Stage 2) and gradient arithmetic.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "rsr.h"
#include "rsr_internal.cuh"
#include "rsr_launch.h"

namespace rsr {

namespace {

thread_local std::string g_last_cuda_error;

int cuda_fail(cudaError_t e, const char *where) {
    char buf[256];
    snprintf(buf, sizeof(buf), "%s: %s (%d)", where, cudaGetErrorString(e), (int)e);
    g_last_cuda_error = buf;
    return RSR_ERR_CUDA;
}

#define RSR_CUDA(call)                                             \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);        \
    } while (0)

uint64_t fnv1a(const void *data, size_t bytes, uint64_t h = 1469598103934665603ull) {
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < bytes; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct Prepared {
    int32_t n, K;
    int64_t R_L, R_U;
    const void *ref_L, *ref_U;
    uint64_t pmf_hash;
    int device;
};

std::mutex g_mu;
std::unordered_map<const void *, Prepared> g_prepared;

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}

int validate(const rsr_problem *p) {
    if (!p) return RSR_ERR_INVALID_ARG;
    if (p->n < 1 || p->K < 2 || p->R_L < 0 || p->R_U < 0 || p->R_L + p->R_U < 1) return RSR_ERR_INVALID_ARG;
    if (p->K > kMaxK || (int64_t)p->n * (p->K - 1) > kMaxKenc) return RSR_ERR_UNSUPPORTED;
    if (p->R_L >= (int64_t(1) << 31) || p->R_U >= (int64_t(1) << 31)) return RSR_ERR_UNSUPPORTED;
    if (!p->pmf) return RSR_ERR_INVALID_ARG;
    if ((p->R_L > 0 && !p->ref_L) || (p->R_U > 0 && !p->ref_U)) return RSR_ERR_INVALID_ARG;
    if (p->path < RSR_PATH_AUTO || p->path > RSR_PATH_TC) return RSR_ERR_INVALID_ARG;
    for (int i = 0; i < p->n; ++i) {
        double s = 0.0;
        for (int k = 0; k < p->K; ++k) {
            const double q = p->pmf[(size_t)i * p->K + k];
            if (!(q >= 0.0 && q <= 1.0)) return RSR_ERR_INVALID_ARG;
            s += q;
        }
        if (std::fabs(s - 1.0) > 1e-9) return RSR_ERR_INVALID_ARG;
    }
    return RSR_OK;
}

int check_ws(const WsLayout &L, const void *ws, size_t ws_bytes) {
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < L.total) return RSR_ERR_WORKSPACE;
    return RSR_OK;
}

WsLayout layout_of(const rsr_problem *p) {
    const int words = (p->n * (p->K - 1) + 31) / 32;
    return make_layout(p->n, p->K, p->R_L, p->R_U, popc_word_bucket(words));
}

// Sampler thresholds T_{i,k} = min(2^32, floor(2^32 * c_{i,k})), c_{i,k} the
// fp64 left-to-right sum of q_{i,0..k-1}.
void host_thresholds(const rsr_problem *p, std::vector<unsigned long long> &T) {
    const int km1 = p->K - 1;
    T.assign((size_t)p->n * km1, 0ull);
    for (int i = 0; i < p->n; ++i) {
        double c = 0.0;
        for (int k = 1; k <= km1; ++k) {
            c += p->pmf[(size_t)i * p->K + (k - 1)];
            const double v = std::floor(std::ldexp(c, 32));
            unsigned long long t;
            if (v <= 0.0) t = 0ull;
            else if (v >= 4294967296.0) t = 4294967296ull;
            else t = (unsigned long long)v;
            T[(size_t)i * km1 + (k - 1)] = t;
        }
    }
}

uint64_t pmf_hash(const rsr_problem *p) { return fnv1a(p->pmf, sizeof(double) * (size_t)p->n * p->K); }

int upload_thresholds(const rsr_problem *p, const WsLayout &L, void *ws, cudaStream_t s) {
    std::vector<unsigned long long> T;
    host_thresholds(p, T);
    // pageable source: the call returns once the data is staged, so T may go out of scope
    RSR_CUDA(cudaMemcpyAsync(static_cast<char *>(ws) + L.off_thr, T.data(), T.size() * sizeof(T[0]),
                             cudaMemcpyHostToDevice, s));
    return RSR_OK;
}

int check_prepared(const rsr_problem *p, const void *ws) {
    std::lock_guard<std::mutex> g(g_mu);
    auto it = g_prepared.find(ws);
    if (it == g_prepared.end()) return RSR_ERR_NOT_PREPARED;
    const Prepared &q = it->second;
    if (q.n != p->n || q.K != p->K || q.R_L != p->R_L || q.R_U != p->R_U || q.ref_L != p->ref_L ||
        q.ref_U != p->ref_U || q.device != current_device() || q.pmf_hash != pmf_hash(p))
        return RSR_ERR_NOT_PREPARED;
    return RSR_OK;
}

ClassifyParams make_params(const rsr_problem *p, const WsLayout &L, void *ws) {
    char *base = static_cast<char *>(ws);
    ClassifyParams c{};
    c.n = p->n;
    c.K = p->K;
    c.km1 = p->K - 1;
    c.kenc = L.kenc;
    c.words = L.words;
    c.thr = reinterpret_cast<const unsigned long long *>(base + L.off_thr);
    c.popc_L = reinterpret_cast<const uint32_t *>(base + L.off_popc_L);
    c.popc_U = reinterpret_cast<const uint32_t *>(base + L.off_popc_U);
    c.tc_L = reinterpret_cast<const uint8_t *>(base + L.off_tc_L);
    c.tc_U = reinterpret_cast<const uint8_t *>(base + L.off_tc_U);
    c.R_L = p->R_L;
    c.R_U = p->R_U;
    c.tc_kpad = L.tc_kpad;
    c.hdr = reinterpret_cast<WsHeader *>(base);
    c.dense = (p->flags & RSR_FLAG_DENSE) ? 1 : 0;
    return c;
}

// Path for RSR_PATH_AUTO: the tensor-core contraction pays once the reference
// sets are large enough to keep 128x128 MMA tiles busy.
int choose_path(const rsr_problem *p) {
    if (p->path != RSR_PATH_AUTO) return p->path;
    const WsLayout L = layout_of(p);
    if (tc_supported() && L.tc_kpad <= tc_max_kpad() && (p->R_L + p->R_U) >= 8192 && (p->flags & RSR_FLAG_DENSE))
        return RSR_PATH_TC;
    return RSR_PATH_POPC;
}

}  // namespace

int device_sm_count() {
    static int cached[64] = {0};
    const int d = current_device();
    if (d >= 0 && d < 64 && cached[d]) return cached[d];
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
    if (v <= 0) v = 1;
    if (d >= 0 && d < 64) cached[d] = v;
    return v;
}

}  // namespace rsr

using namespace rsr;

extern "C" {

size_t rsr_workspace_size(const rsr_problem *problem, int64_t N) {
    (void)N;
    if (validate(problem) != RSR_OK) return 0;
    return layout_of(problem).total;
}

int rsr_prepare(const rsr_problem *problem, void *ws, size_t ws_bytes, rsr_stream_t stream) {
    int st = validate(problem);
    if (st != RSR_OK) return st;
    const WsLayout L = layout_of(problem);
    if ((st = check_ws(L, ws, ws_bytes)) != RSR_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(ws);
    const int path = choose_path(problem);
    if (path == RSR_PATH_TC && (!tc_supported() || L.tc_kpad > tc_max_kpad())) return RSR_ERR_UNSUPPORTED;
    RSR_CUDA(cudaMemsetAsync(base, 0, sizeof(WsHeader), s));
    if ((st = upload_thresholds(problem, L, ws, s)) != RSR_OK) return st;
    const int km1 = problem->K - 1;
    uint32_t *pL = reinterpret_cast<uint32_t *>(base + L.off_popc_L);
    uint32_t *pU = reinterpret_cast<uint32_t *>(base + L.off_popc_U);
    RSR_CUDA(launch_encode_popc(problem->ref_L, problem->R_L, problem->n, km1, L.words, true, pL, s));
    RSR_CUDA(launch_encode_popc(problem->ref_U, problem->R_U, problem->n, km1, L.words, false, pU, s));
    RSR_CUDA(launch_overlap(pL, problem->R_L, pU, problem->R_U, L.words, reinterpret_cast<WsHeader *>(base), s));
    if (tc_supported() && L.tc_kpad <= tc_max_kpad()) {
        RSR_CUDA(launch_encode_tc(problem->ref_L, problem->R_L, L.tc_rows_L, problem->n, km1, L.tc_kpad, false,
                                  reinterpret_cast<uint8_t *>(base + L.off_tc_L), s));
        RSR_CUDA(launch_encode_tc(problem->ref_U, problem->R_U, L.tc_rows_U, problem->n, km1, L.tc_kpad, true,
                                  reinterpret_cast<uint8_t *>(base + L.off_tc_U), s));
    }
    std::lock_guard<std::mutex> g(g_mu);
    g_prepared[ws] = Prepared{problem->n, problem->K, problem->R_L, problem->R_U, problem->ref_L, problem->ref_U,
                              pmf_hash(problem), current_device()};
    return RSR_OK;
}

int rsr_update_pmf(const rsr_problem *problem, void *ws, size_t ws_bytes, rsr_stream_t stream) {
    int st = validate(problem);
    if (st != RSR_OK) return st;
    const WsLayout L = layout_of(problem);
    if ((st = check_ws(L, ws, ws_bytes)) != RSR_OK) return st;
    {
        std::lock_guard<std::mutex> g(g_mu);
        auto it = g_prepared.find(ws);
        if (it == g_prepared.end()) return RSR_ERR_NOT_PREPARED;
        const Prepared &q = it->second;
        if (q.n != problem->n || q.K != problem->K || q.R_L != problem->R_L || q.R_U != problem->R_U ||
            q.ref_L != problem->ref_L || q.ref_U != problem->ref_U || q.device != current_device())
            return RSR_ERR_NOT_PREPARED;
    }
    if ((st = upload_thresholds(problem, L, ws, reinterpret_cast<cudaStream_t>(stream))) != RSR_OK) return st;
    std::lock_guard<std::mutex> g(g_mu);
    g_prepared[ws].pmf_hash = pmf_hash(problem);
    return RSR_OK;
}

int rsr_classify(const rsr_problem *problem, uint64_t seed, uint64_t offset, int64_t N,
                 const uint8_t *samples_or_null, uint8_t *labels_or_null, int64_t *counts3,
                 int64_t *grad_counts_or_null, int64_t *exec_tests_or_null, void *ws, size_t ws_bytes,
                 rsr_stream_t stream) {
    int st = validate(problem);
    if (st != RSR_OK) return st;
    if (N < 0 || !counts3) return RSR_ERR_INVALID_ARG;
    const WsLayout L = layout_of(problem);
    if ((st = check_ws(L, ws, ws_bytes)) != RSR_OK) return st;
    if ((st = check_prepared(problem, ws)) != RSR_OK) return st;
    if (N == 0) return RSR_OK;
    ClassifyParams c = make_params(problem, L, ws);
    c.N = N;
    c.seed = seed;
    c.offset = offset;
    c.samples = samples_or_null;
    c.labels = labels_or_null;
    c.counts3 = reinterpret_cast<unsigned long long *>(counts3);
    c.grad_counts = reinterpret_cast<unsigned long long *>(grad_counts_or_null);
    c.exec_tests = reinterpret_cast<unsigned long long *>(exec_tests_or_null);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int path = choose_path(problem);
    if (path == RSR_PATH_TC) {
        if (!tc_supported() || L.tc_kpad > tc_max_kpad()) return RSR_ERR_UNSUPPORTED;
        RSR_CUDA(launch_classify_tc(c, s));
    } else {
        RSR_CUDA(launch_classify_popc(c, s));
    }
    return RSR_OK;
}

int rsr_estimate(const int64_t counts3[3], int64_t N, int64_t n_u_lower, rsr_estimate_out *out) {
    if (!counts3 || !out || N <= 0 || n_u_lower < 0 || n_u_lower > counts3[2] || counts3[0] < 0 ||
        counts3[1] < 0 || counts3[2] < 0 || counts3[0] + counts3[1] + counts3[2] != N)
        return RSR_ERR_INVALID_ARG;
    const double H = (double)N;
    auto cov = [H](double p) { return std::sqrt((1.0 - p) / (H * p)); };
    out->pL = (double)counts3[0] / H;
    out->pU = (double)counts3[1] / H;
    out->pu = (double)counts3[2] / H;
    out->P_lower = (double)(counts3[0] + n_u_lower) / H;
    out->P_upper = (double)(counts3[1] + (counts3[2] - n_u_lower)) / H;
    out->cov_pL = cov(out->pL);
    out->cov_pU = cov(out->pU);
    out->cov_pu = cov(out->pu);
    out->cov_lower = cov(out->P_lower);
    out->cov_upper = cov(out->P_upper);
    return RSR_OK;
}

int rsr_grad(const rsr_problem *problem, uint64_t seed, uint64_t offset, int64_t N, int64_t *grad_counts,
             const int64_t *u_lower_idx, int64_t n_u_lower, double *grad_out, double *se_out, void *ws,
             size_t ws_bytes, rsr_stream_t stream) {
    int st = validate(problem);
    if (st != RSR_OK) return st;
    if (N <= 0 || !grad_counts || !grad_out || !se_out || n_u_lower < 0 || (n_u_lower > 0 && !u_lower_idx))
        return RSR_ERR_INVALID_ARG;
    const WsLayout L = layout_of(problem);
    if ((st = check_ws(L, ws, ws_bytes)) != RSR_OK) return st;
    if ((st = check_prepared(problem, ws)) != RSR_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ClassifyParams c = make_params(problem, L, ws);
    c.N = N;
    c.seed = seed;
    c.offset = offset;
    c.grad_counts = reinterpret_cast<unsigned long long *>(grad_counts);
    RSR_CUDA(launch_grad_correction(c, u_lower_idx, n_u_lower, s));
    const size_t nk = (size_t)problem->n * problem->K;
    std::vector<int64_t> C(nk);
    int32_t err = 0;
    RSR_CUDA(cudaMemcpyAsync(C.data(), grad_counts, nk * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    RSR_CUDA(cudaMemcpyAsync(&err, &reinterpret_cast<WsHeader *>(ws)->error, sizeof(int32_t),
                             cudaMemcpyDeviceToHost, s));
    RSR_CUDA(cudaStreamSynchronize(s));
    if (err != 0) return RSR_ERR_INVALID_ARG;
    const double H = (double)N;
    for (size_t j = 0; j < nk; ++j) {
        const double p = (double)C[j] / H;
        const double q = problem->pmf[j];
        grad_out[j] = p / q;
        se_out[j] = std::sqrt(p * (1.0 - p) / H) / q;
    }
    return RSR_OK;
}

int rsr_sample(const rsr_problem *problem, uint64_t seed, uint64_t offset, int64_t N, uint8_t *states, void *ws,
               size_t ws_bytes, rsr_stream_t stream) {
    int st = validate(problem);
    if (st != RSR_OK) return st;
    if (N < 0 || (N > 0 && !states)) return RSR_ERR_INVALID_ARG;
    const WsLayout L = layout_of(problem);
    if ((st = check_ws(L, ws, ws_bytes)) != RSR_OK) return st;
    if ((st = check_prepared(problem, ws)) != RSR_OK) return st;
    ClassifyParams c = make_params(problem, L, ws);
    c.N = N;
    c.seed = seed;
    c.offset = offset;
    RSR_CUDA(launch_sample(c, states, reinterpret_cast<cudaStream_t>(stream)));
    return RSR_OK;
}

int rsr_workspace_status(const void *ws, int32_t out[2], rsr_stream_t stream) {
    if (!ws || !out) return RSR_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    RSR_CUDA(cudaMemcpyAsync(out, ws, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    RSR_CUDA(cudaStreamSynchronize(s));
    return RSR_OK;
}

const char *rsr_status_string(int status) {
    switch (status) {
        case RSR_OK: return "ok";
        case RSR_ERR_INVALID_ARG: return "invalid argument";
        case RSR_ERR_CUDA: return "CUDA runtime error";
        case RSR_ERR_WORKSPACE: return "workspace too small or misaligned";
        case RSR_ERR_TIMEOUT: return "bounded device wait timed out";
        case RSR_ERR_UNSUPPORTED: return "unsupported size or device";
        case RSR_ERR_NOT_PREPARED: return "workspace not prepared for this problem/pmf";
        default: return "unknown status";
    }
}

const char *rsr_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

}  // extern "C"
