// noalloc.cu -- classification without any caller-provided or allocated
// device memory beyond the inputs and outputs.
//
// Why: some callers cannot call cudaMalloc at all, or not at the moment they
// need a result -- for example a plugin inside a host application that owns
// every byte of device memory through its own pool and forbids libraries to
// allocate, a real-time loop whose allocation budget is fixed at start-up, or
// a foreign-language caller that reaches this library only through its C ABI
// and has no device allocator of its own.  They still own their inputs and
// outputs; everything else lives here.
//
// What: rsr_classify_static() runs the same preparation and the same
// bit-packed classifier as rsr_prepare() + rsr_classify() on RSR_PATH_POPC,
// but its workspace is the file-scope device array below (kStaticScratchBytes
// = 4 MiB).  Every GPU that loads librsr holds that array until the process
// exits.  Problems whose encoded workspace would exceed it are rejected with
// RSR_ERR_WORKSPACE before any GPU work.
//
// Set-up: host code cannot use the array's name as a device address (on the
// host it names a stand-in object, not GPU memory), so the device address is
// looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call that runs on it; that first call should
// therefore come before any stream capture.
//
// Ordering: the call is asynchronous on its stream.  The sampler thresholds
// reach the array as a kernel argument (copied when the kernel is launched),
// not through a copy from host memory, so no step waits for the stream.
//
// Sharing: all calls on a device share the one array, which keeps whatever
// the previous call left; each call re-clears the header that must start at
// zero (the precedence flag and the error word) and rewrites thresholds and
// encodings.  Calls whose GPU work overlaps (different streams, or another
// host thread) race on the array: serialise them.
#include <mutex>

#include <cuda_runtime.h>

#include "rsr.h"
#include "rsr_internal.cuh"
#include "rsr_launch.h"

namespace rsr {

namespace {

constexpr size_t kStaticScratchBytes = size_t(4) << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void *g_static_addr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
cudaError_t static_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_static_mu);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return cudaSuccess;
}

// A failed CUDA call: consume the runtime's last-error state so that it does
// not resurface in a later, unrelated call, and report RSR_ERR_CUDA.
int fail() {
    (void)cudaGetLastError();
    return RSR_ERR_CUDA;
}

// Every check of the caller-workspace entry points (sizes, reference counts
// below 2^31, pmf rows), with problem->path ignored as documented.
int check_problem(const rsr_problem *p) {
    if (!p) return RSR_ERR_INVALID_ARG;
    rsr_problem q = *p;
    q.path = RSR_PATH_POPC;
    return validate_problem(&q);
}

// The thresholds travel inside the kernel's argument block (8 KB; launches
// accept up to 32 KB of arguments), so no host buffer has to outlive the call.
struct ThresholdArg {
    unsigned long long v[kMaxKenc];
};

__global__ void store_thresholds_kernel(const ThresholdArg a, int count, unsigned long long *dst) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) dst[i] = a.v[i];
}

}  // namespace

}  // namespace rsr

using namespace rsr;

extern "C" int rsr_classify_static(const rsr_problem *problem, uint64_t seed, uint64_t offset, int64_t N,
                                   const uint8_t *samples_or_null, uint8_t *labels_or_null, int64_t *counts3,
                                   int64_t *grad_counts_or_null, rsr_stream_t stream) {
    int st = check_problem(problem);
    if (st != RSR_OK) return st;
    if (N < 0 || !counts3) return RSR_ERR_INVALID_ARG;
    const int km1 = problem->K - 1;
    const int words_b = popc_word_bucket((problem->n * km1 + 31) / 32);
    const WsLayout L = make_layout(problem->n, problem->K, problem->R_L, problem->R_U, words_b);
    // only the header, the thresholds and the bit-packed references live in the array
    if (L.off_tc_L > kStaticScratchBytes) return RSR_ERR_WORKSPACE;
    void *scratch = nullptr;
    if (static_scratch(&scratch) != cudaSuccess) return fail();
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(scratch);

    // thresholds on the host, in a fixed-size argument block (no host allocation either)
    ThresholdArg T;
    const int nthr = problem->n * km1;
    host_thresholds(problem->n, problem->K, problem->pmf, T.v);
    if (cudaMemsetAsync(base, 0, sizeof(WsHeader), s) != cudaSuccess) return fail();
    store_thresholds_kernel<<<1, 256, 0, s>>>(T, nthr, reinterpret_cast<unsigned long long *>(base + L.off_thr));
    if (cudaGetLastError() != cudaSuccess) return fail();
    uint32_t *pL = reinterpret_cast<uint32_t *>(base + L.off_popc_L);
    uint32_t *pU = reinterpret_cast<uint32_t *>(base + L.off_popc_U);
    if (launch_encode_popc(problem->ref_L, problem->R_L, problem->n, km1, words_b, true, pL, s) != cudaSuccess ||
        launch_encode_popc(problem->ref_U, problem->R_U, problem->n, km1, words_b, false, pU, s) != cudaSuccess ||
        launch_overlap(pL, problem->R_L, pU, problem->R_U, words_b, reinterpret_cast<WsHeader *>(base), s) !=
            cudaSuccess)
        return fail();
    if (N == 0) return RSR_OK;
    ClassifyParams c{};
    c.n = problem->n;
    c.K = problem->K;
    c.km1 = km1;
    c.kenc = L.kenc;
    c.words = words_b;
    c.N = N;
    c.seed = seed;
    c.offset = offset;
    c.samples = samples_or_null;
    c.thr = reinterpret_cast<const unsigned long long *>(base + L.off_thr);
    c.popc_L = pL;
    c.popc_U = pU;
    c.R_L = problem->R_L;
    c.R_U = problem->R_U;
    c.labels = labels_or_null;
    c.counts3 = reinterpret_cast<unsigned long long *>(counts3);
    c.grad_counts = reinterpret_cast<unsigned long long *>(grad_counts_or_null);
    c.exec_tests = nullptr;
    c.hdr = reinterpret_cast<WsHeader *>(base);
    c.dense = (problem->flags & RSR_FLAG_DENSE) ? 1 : 0;
    if (launch_classify_popc(c, s) != cudaSuccess) return fail();
    return RSR_OK;
}
