// Measured FP32 FMA issue ceiling of the current GPU: the denominator of the projectors'
// roofline.  Both projectors do two FMAs per (pixel, angle) sample on data staged on chip,
// far right of the HBM ridge, so their bound is the rate at which the SMs retire FP32 FMAs.
// This kernel retires nothing but independent FMA chains (8 per thread, in registers), as
// scalar FFMA and as paired .f32x2 FMA, on a grid of 8 CTAs of 256 threads per SM, and
// reports the faster form in FMA/s.  No allocation: the results land in a static sink.
#include <cmath>

#include "ctr_internal.cuh"

namespace ctr {
namespace {

static __device__ float g_fma_sink[8];

constexpr int FMA_CHAINS = 8;
constexpr int FMA_THREADS = 256;

__global__ void __launch_bounds__(FMA_THREADS) k_fma_scalar(int iters, float a, float b)
{
    float x[FMA_CHAINS];
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < FMA_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < FMA_CHAINS; ++c) s += x[c];
    if (s == 1234.5f) g_fma_sink[threadIdx.x & 7] = s;   // keeps the chains alive, never true in practice
}

__device__ __forceinline__ unsigned long long fma2_u64(unsigned long long x, unsigned long long a,
                                                       unsigned long long b)
{
    unsigned long long d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(x), "l"(a), "l"(b));
    return d;
}

__global__ void __launch_bounds__(FMA_THREADS) k_fma_paired(int iters, float a, float b)
{
    unsigned long long x[FMA_CHAINS / 2];
    const unsigned long long aa = ((unsigned long long)__float_as_uint(a) << 32) | __float_as_uint(a);
    const unsigned long long bb = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
#pragma unroll
    for (int c = 0; c < FMA_CHAINS / 2; ++c) {
        const float lo = (float)(threadIdx.x + 2 * c) * 1e-3f, hi = (float)(threadIdx.x + 2 * c + 1) * 1e-3f;
        x[c] = ((unsigned long long)__float_as_uint(hi) << 32) | __float_as_uint(lo);
    }
    for (int k = 0; k < iters; ++k) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < FMA_CHAINS / 2; ++c) x[c] = fma2_u64(x[c], aa, bb);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < FMA_CHAINS / 2; ++c)
        s += __uint_as_float((unsigned)(x[c] & 0xffffffffu)) + __uint_as_float((unsigned)(x[c] >> 32));
    if (s == 1234.5f) g_fma_sink[threadIdx.x & 7] = s;
}

}  // namespace
}  // namespace ctr

using namespace ctr;

extern "C" ctr_status ctr_fp32_fma_rate(double *fma_per_s, void *stream)
{
    if (!fma_per_s) return fail(CTR_EINVAL, "fma_per_s is NULL");
    int dev = 0, sms = 0;
    CTR_CUDA(cudaGetDevice(&dev));
    CTR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = (cudaStream_t)stream;
    const int blocks = sms * 8, iters = 2048;
    // FMAs per launch: threads x iterations x 16 unrolled rounds x 8 chains
    const double fmas = (double)blocks * FMA_THREADS * iters * 16.0 * FMA_CHAINS;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CTR_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(CTR_ECUDA, "cudaEventCreate");
    }
    double best = 0.0;
    ctr_status st = CTR_OK;
    for (int form = 0; form < 2 && st == CTR_OK; ++form) {
        for (int rep = 0; rep < 4; ++rep) {   // the first run of each form warms the clocks up
            cudaEventRecord(e0, s);
            if (form == 0) k_fma_scalar<<<blocks, FMA_THREADS, 0, s>>>(iters, 0.999f, 1e-4f);
            else k_fma_paired<<<blocks, FMA_THREADS, 0, s>>>(iters, 0.999f, 1e-4f);
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e != cudaSuccess) {
                st = cuda_fail(e, "FMA ceiling kernel");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms > 0.f) best = std::fmax(best, fmas / (ms * 1e-3));
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != CTR_OK) return st;
    *fma_per_s = best;
    return CTR_OK;
}
