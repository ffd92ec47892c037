// peaks.cu -- measured integer throughput of this GPU, the denominator of the
// bit-packed classifiers' roofline (their tests are LOP3 and-or-accumulates,
// their sampler is Philox4x32-10, whose rounds are 32x32->64 multiplies).
//
// Two kernels, each with eight independent dependency chains per thread so
// that issue, not latency, bounds them: one of three-input logic ops (LOP3,
// the ALU pipe), one of wide multiply-adds (IMAD.WIDE, the Philox product).
// A full grid (8 blocks of 256 threads per SM) runs a fixed number of
// iterations; the rate is ops / CUDA-event time of the second of two launches.
// The results feed a never-taken store into a file-scope device word, so
// nothing is allocated and nothing is eliminated.
#include <cuda_runtime.h>
#include <stdint.h>

#include "rsr.h"
#include "rsr_internal.cuh"
#include "rsr_launch.h"

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

}  // namespace

}  // namespace rsr

using namespace rsr;

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
