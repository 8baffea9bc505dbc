// pa_peaks.cu -- measured arithmetic peaks of the GPU for the rooflines of the FP64
// and exact (NTT64) modes: the rate of independent FP64 fused multiply-adds, and
// the rate of products modulo p = 2^64 - 2^32 + 1 computed by the same zp_mul
// (64 x 64 -> 128-bit product and reduction) that the exact transform uses.
// Measurement support; the paper has no counterpart.
#include <cstdint>

#include "pa.h"
#include "pa_internal.h"
#include "pa_kernels.cuh"

namespace pa {
namespace {

constexpr int kChains = 8;  // independent dependency chains per thread

// Each thread runs kChains chains of `iters` dependent FMAs; the result is stored only
// when it equals an impossible value, so nothing is optimised away.
__global__ void __launch_bounds__(256) k_fp64_fma(double *out, int iters, double b, double c) {
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (double)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.0) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_zp_mul(uint64_t *out, int iters, uint64_t y) {
    uint64_t x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = 0x123456789ull * (threadIdx.x + 1) + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = zp_mul(x[k], y);
    }
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s ^= x[k];
    if (s == 1ull) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace pa

extern "C" int pa_alu_peaks(double *fp64_gflops, double *zp_gmul_s, pa_stream_t stream) {
    using namespace pa;
    if (!fp64_gflops || !zp_gmul_s) return PA_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return pa_internal_cuda_fail(e, "pa_alu_peaks: device query");
    const int blocks = sms * 8, threads = 256;  // 2048 resident threads per SM
    void *out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaMalloc(&out, (size_t)blocks * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float ms_fp = 0.f, ms_zp = 0.f;
    const int it_fp = 4096, it_zp = 1024;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first round warms up
        k_fp64_fma<<<blocks, threads, 0, st>>>(static_cast<double *>(out), it_fp, 0.999999999, 1e-9);
        e = cudaEventRecord(a, st);
        if (e == cudaSuccess) k_fp64_fma<<<blocks, threads, 0, st>>>(static_cast<double *>(out), it_fp, 0.999999999, 1e-9);
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_fp, a, b);
        if (e == cudaSuccess) k_zp_mul<<<blocks, threads, 0, st>>>(static_cast<uint64_t *>(out), it_zp, 0xFEDCBA9876543ull);
        if (e == cudaSuccess) e = cudaEventRecord(a, st);
        if (e == cudaSuccess) k_zp_mul<<<blocks, threads, 0, st>>>(static_cast<uint64_t *>(out), it_zp, 0xFEDCBA9876543ull);
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_zp, a, b);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFree(out);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return pa_internal_cuda_fail(e, "pa_alu_peaks");
    const double n = (double)blocks * threads * kChains;
    *fp64_gflops = 2.0 * n * it_fp / (ms_fp * 1e-3) / 1e9;
    *zp_gmul_s = n * it_zp / (ms_zp * 1e-3) / 1e9;
    return PA_OK;
}
