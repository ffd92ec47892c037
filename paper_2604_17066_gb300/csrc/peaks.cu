// peaks.cu -- measured throughput of this GPU, the denominators of the
// classifiers' rooflines.
//
// Integer: the bit-packed classifiers' tests are LOP3 and-or-accumulates and
// their sampler is Philox4x32-10, whose rounds are 32x32->64 multiplies.
//
// Two kernels, each with eight independent dependency chains per thread so
// that issue, not latency, bounds them: one of three-input logic ops (LOP3,
// the ALU pipe), one of wide multiply-adds (IMAD.WIDE, the Philox product).
// A full grid (8 blocks of 256 threads per SM) runs a fixed number of
// iterations; the rate is ops / CUDA-event time of the second of two launches.
// The results feed a never-taken store into a file-scope device word, so
// nothing is allocated and nothing is eliminated.
//
// Tensor (FP8): the classifiers issue tcgen05.mma kind::f8f6f4 with E4M3
// operands from shared memory and FP32 accumulators in tensor memory.  The
// roofline denominator is the same instruction run back to back, one CTA per
// SM, either alone (cta_group::1, M = 128) or on CTA pairs (cta_group::2,
// M = 256, as the dense classifier): operands resident in shared memory
// (pseudo-random E4M3 bytes, never NaN or infinite), no copies and no
// epilogue, alternating between two accumulators so that consecutive MMAs are
// independent.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rsr.h"
#include "rsr_internal.cuh"
#include "rsr_launch.h"
#include "tc_ptx.cuh"

namespace rsr {

namespace {

__device__ uint32_t g_peak_sink;

constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSM = 8;
constexpr int kPeakIters = 1 << 16;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kPeakThreads) lop3_peak_kernel(uint32_t seed) {
    uint32_t a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = seed * (2u * k + 1u) ^ threadIdx.x ^ (blockIdx.x << 10);
    const uint32_t b = seed ^ 0x9E3779B9u, c = ~seed;
    for (int i = 0; i < kPeakIters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k)
            asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[k]) : "r"(b), "r"(c));
    }
    uint32_t x = 0u;
#pragma unroll
    for (int k = 0; k < kChains; ++k) x ^= a[k];
    if (x == 0x5EED5EEDu) g_peak_sink = x;
}

__global__ void __launch_bounds__(kPeakThreads) imad_peak_kernel(uint32_t seed) {
    uint64_t a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (uint64_t)(seed * (2u * k + 1u) ^ threadIdx.x ^ (blockIdx.x << 10));
    const uint32_t m = 0xD2511F53u;
    for (int i = 0; i < kPeakIters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            uint32_t lo = (uint32_t)a[k], hi = (uint32_t)(a[k] >> 32);
            asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(a[k]) : "r"(lo), "r"(m), "l"((uint64_t)hi));
        }
    }
    uint64_t x = 0u;
#pragma unroll
    for (int k = 0; k < kChains; ++k) x ^= a[k];
    if ((uint32_t)x == 0x5EED5EEDu) g_peak_sink = (uint32_t)x;
}

// Philox4x32-10 blocks (the samplers' generator, rsr_internal.cuh) with eight
// independent counters per thread: the generator's own rate, which issue
// slots, not the multiplier alone, bound (each round is two wide products, two
// three-input XORs and two key additions).
constexpr int kPhiloxIters = 1 << 10;

__global__ void __launch_bounds__(kPeakThreads) philox_rate_kernel(uint32_t seed) {
    const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0u;
    for (int i = 0; i < kPhiloxIters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            const U32x4 r = philox4x32_10(gid, (uint32_t)i, (uint32_t)k, 0u, seed, ~seed);
            acc ^= r.x ^ r.y ^ r.z ^ r.w;
        }
    }
    if (acc == 0x5EED5EEDu) g_peak_sink = acc;
}

constexpr int kMmaM = 128, kMmaN = 256;
constexpr int kMmaKBytes = 128;           // four K steps of 32 E4M3 values per iteration
constexpr int kFp8Threads = 128;
constexpr long long kFp8Iters = 1 << 16;  // about 16 ms per launch at the full rate
constexpr size_t kFp8Smem = 120 * 1024;   // more than half an SM: one CTA per SM (512 TMEM columns each)

__device__ int32_t g_fp8_peak_err;

__global__ void __launch_bounds__(kFp8Threads, 1) fp8_mma_peak_kernel(long long iters) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char *sA = smem;                        // 128 rows x 128 bytes
    unsigned char *sB = smem + kMmaM * kMmaKBytes;   // 256 rows x 128 bytes
    for (int i = tid; i < (kMmaM + kMmaN) * kMmaKBytes / 4; i += blockDim.x) {
        uint32_t h = (uint32_t)i * 0x9E3779B1u ^ ((uint32_t)blockIdx.x * 0x85EBCA77u);
        h ^= h >> 15;
        h *= 0x2C1B3C6Du;
        h ^= h >> 12;
        reinterpret_cast<uint32_t *>(smem)[i] = h & 0xBFBFBFBFu;   // exponent top bit clear: |v| < 2
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base, 2 * kMmaN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
        constexpr uint32_t idesc = idesc_f8<kMmaM, kMmaN>();
        const uint32_t sbo = kMmaKBytes * 8, a0 = smem_u32(sA), b0 = smem_u32(sB);
        for (long long it = 0; it < iters; ++it) {
            const uint32_t d = tmem + (uint32_t)((it & 1) * kMmaN);
#pragma unroll
            for (int kk = 0; kk < kMmaKBytes / 32; ++kk)
                mma_f8(d, smem_desc(a0 + kk * 256, 128, sbo), smem_desc(b0 + kk * 256, 128, sbo), idesc,
                       kk > 0 ? 1u : 0u);
        }
        mma_commit(&bar);
        if (!mbar_wait(&bar, 0, &abort_flag, &g_fp8_peak_err)) {
            // the MMAs issued above are still running: give them a second bounded
            // wait before the tensor memory is released
            abort_flag = 0;
            (void)mbar_wait(&bar, 0, &abort_flag, &g_fp8_peak_err);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * kMmaN);
    }
}

// The same on CTA pairs (cta_group::2): the even CTA of each cluster issues
// M = 256 x N = 256 x K = 32 MMAs whose A rows and B rows are split between
// the two CTAs' shared memory; its commit reaches both CTAs, which then meet at
// a cluster barrier before the pair's tensor memory is freed.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kFp8Threads, 1) fp8_mma_pair_peak_kernel(long long iters) {
    using namespace tc;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    const bool leader = cluster_ctarank() == 0;
    unsigned char *sA = smem;                        // this CTA's 128 rows of A
    unsigned char *sB = smem + kMmaM * kMmaKBytes;   // this CTA's 128 rows of B
    for (int i = tid; i < 2 * kMmaM * kMmaKBytes / 4; i += blockDim.x) {
        uint32_t h = (uint32_t)i * 0x9E3779B1u ^ ((uint32_t)blockIdx.x * 0x85EBCA77u);
        h ^= h >> 15;
        h *= 0x2C1B3C6Du;
        h ^= h >> 12;
        reinterpret_cast<uint32_t *>(smem)[i] = h & 0xBFBFBFBFu;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc_pair(&tmem_base, 2 * kMmaN);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();   // both CTAs' operands and barriers are ready
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    if (tid == 0 && leader) {
        constexpr uint32_t idesc = idesc_f8<2 * kMmaM, kMmaN>();
        const uint32_t sbo = kMmaKBytes * 8, a0 = smem_u32(sA), b0 = smem_u32(sB);
        for (long long it = 0; it < iters; ++it) {
            const uint32_t d = tmem + (uint32_t)((it & 1) * kMmaN);
#pragma unroll
            for (int kk = 0; kk < kMmaKBytes / 32; ++kk)
                mma_f8_pair(d, smem_desc(a0 + kk * 256, 128, sbo), smem_desc(b0 + kk * 256, 128, sbo), idesc,
                            kk > 0 ? 1u : 0u);
        }
        mma_commit_pair(&bar, 0x3);
    }
    if (tid == 0) {
        // every CTA waits for the leader's MMAs, which read its shared memory and write its tensor memory
        if (!mbar_wait(&bar, 0, &abort_flag, &g_fp8_peak_err)) {
            abort_flag = 0;
            (void)mbar_wait(&bar, 0, &abort_flag, &g_fp8_peak_err);
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc_pair(tmem, 2 * kMmaN);
    }
}

}  // namespace

}  // namespace rsr

using namespace rsr;

extern "C" int rsr_measure_fp8_peak(int32_t cta_pair, double seconds, double *burst_flops_per_s,
                                    double *sustained_flops_per_s, rsr_stream_t stream) {
    if ((cta_pair != 0 && cta_pair != 1) || !burst_flops_per_s || !sustained_flops_per_s || !(seconds >= 0.0) ||
        seconds > 60.0)
        return RSR_ERR_INVALID_ARG;
    if (!tc_supported()) return RSR_ERR_UNSUPPORTED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int grid = cta_pair ? 2 * (device_sm_count() / 2) : device_sm_count();
    // per CTA: the MMAs of its own 128 rows of D (a pair MMA covers 256 rows over two CTAs)
    const double flops_per_launch =
        (double)grid * (double)kFp8Iters * (kMmaKBytes / 32) * 2.0 * kMmaM * kMmaN * 32.0;
    cudaError_t e = cta_pair ? cudaFuncSetAttribute(fp8_mma_pair_peak_kernel,
                                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFp8Smem)
                             : cudaFuncSetAttribute(fp8_mma_peak_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    (int)kFp8Smem);
    if (e != cudaSuccess) return cuda_fail(e, "rsr_measure_fp8_peak");
    const int32_t zero = 0;
    e = cudaMemcpyToSymbolAsync(g_fp8_peak_err, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "rsr_measure_fp8_peak");
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "rsr_measure_fp8_peak");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "rsr_measure_fp8_peak");
    }
    int st = RSR_OK;
    auto timed = [&](int launches, float *ms) -> cudaError_t {
        cudaEventRecord(e0, s);
        for (int l = 0; l < launches; ++l) {
            if (cta_pair)
                fp8_mma_pair_peak_kernel<<<grid, kFp8Threads, kFp8Smem, s>>>(kFp8Iters);
            else
                fp8_mma_peak_kernel<<<grid, kFp8Threads, kFp8Smem, s>>>(kFp8Iters);
        }
        cudaEventRecord(e1, s);
        cudaError_t r = cudaEventSynchronize(e1);
        if (r == cudaSuccess) r = cudaGetLastError();
        if (r == cudaSuccess) r = cudaEventElapsedTime(ms, e0, e1);
        return r;
    };
    // burst: the fastest of five single launches after one warm-up launch
    float best = 1e30f, ms = 0.0f;
    for (int rep = 0; rep < 6 && st == RSR_OK; ++rep) {
        if ((e = timed(1, &ms)) != cudaSuccess) st = cuda_fail(e, "rsr_measure_fp8_peak");
        else if (rep > 0 && ms < best) best = ms;
    }
    if (st == RSR_OK) *burst_flops_per_s = flops_per_launch / (best / 1000.0);
    // sustained: back-to-back launches for about `seconds`
    *sustained_flops_per_s = 0.0;
    if (st == RSR_OK && seconds > 0.0) {
        const int launches = (int)(seconds / (best / 1000.0)) + 1;
        if ((e = timed(launches, &ms)) != cudaSuccess) st = cuda_fail(e, "rsr_measure_fp8_peak");
        else *sustained_flops_per_s = flops_per_launch * launches / (ms / 1000.0);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == RSR_OK) {
        int32_t err = 0;
        e = cudaMemcpyFromSymbol(&err, g_fp8_peak_err, sizeof(err));
        if (e != cudaSuccess) return cuda_fail(e, "rsr_measure_fp8_peak");
        if (err != 0) return RSR_ERR_TIMEOUT;
    }
    return st;
}

extern "C" int rsr_measure_philox_rate(double *blocks_per_s, rsr_stream_t stream) {
    if (!blocks_per_s) return RSR_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int grid = device_sm_count() * kPeakBlocksPerSM;
    const double blocks = (double)grid * kPeakThreads * (double)kPhiloxIters * kChains;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "rsr_measure_philox_rate");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "rsr_measure_philox_rate");
    }
    int st = RSR_OK;
    float ms = 0.0f;
    for (int rep = 0; rep < 2 && st == RSR_OK; ++rep) {
        cudaEventRecord(e0, s);
        philox_rate_kernel<<<grid, kPeakThreads, 0, s>>>(0x1234u + rep);
        cudaEventRecord(e1, s);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) st = cuda_fail(e, "rsr_measure_philox_rate");
    }
    if (st == RSR_OK) *blocks_per_s = blocks / (ms / 1000.0);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

extern "C" int rsr_measure_int_peak(double *lop3_ops_per_s, double *imad_ops_per_s, rsr_stream_t stream) {
    if (!lop3_ops_per_s || !imad_ops_per_s) return RSR_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int grid = device_sm_count() * kPeakBlocksPerSM;
    const double ops = (double)grid * kPeakThreads * (double)kPeakIters * kChains;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "rsr_measure_int_peak");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "rsr_measure_int_peak");
    }
    int st = RSR_OK;
    for (int which = 0; which < 2 && st == RSR_OK; ++which) {
        float ms = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, s);
            if (which == 0)
                lop3_peak_kernel<<<grid, kPeakThreads, 0, s>>>(0x1234u + rep);
            else
                imad_peak_kernel<<<grid, kPeakThreads, 0, s>>>(0x1234u + rep);
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "rsr_measure_int_peak");
                break;
            }
        }
        if (st == RSR_OK) (which == 0 ? *lop3_ops_per_s : *imad_ops_per_s) = ops / (ms / 1000.0);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}
