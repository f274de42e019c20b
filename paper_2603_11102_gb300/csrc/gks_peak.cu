// gks_peak.cu -- gks_alu_peak_probe: a fused multiply-add loop that measures
// the FP32 or FP64 arithmetic peak of the device the stencil kernels run on,
// the denominator of their ALU roofline. It is a measurement aid, not a step
// of the method.
//
// Every thread runs kChains independent FMA chains x <- x * a + b, unrolled
// kUnroll times per iteration, so the FMA pipes never wait on a dependency
// (kind 2: the same lanes as kChains / 2 chains of packed FP32 pairs, one
// FFMA2 instruction per two FMAs, the form the packed stencil code uses);
// the grid is a whole number of blocks per SM. With a = 1 - 2^-20 and
// b = 2^-20 the chains converge to 1 and stay finite and normal. The result
// is stored only when it equals an impossible value, which the compiler
// cannot know, so the loop is not removed and almost nothing is written.
#include <cuda_runtime.h>

#include <string>

#include "gks_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_loop_kernel(long iters, T a, T b, T *sink)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (long i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-12345.0) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) fma2_loop_kernel(long iters, float a, float b, float *sink)
{
    float2 x[kChains / 2];
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c)
        x[c] = make_float2((float)(threadIdx.x + 2 * c) * 1e-3f, (float)(threadIdx.x + 2 * c + 1) * 1e-3f);
    const float2 A = make_float2(a, a), B = make_float2(b, b);
    for (long i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains / 2; ++c) x[c] = __ffma2_rn(x[c], A, B);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains / 2; ++c) s += x[c].x + x[c].y;
    if (s == -12345.0f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" int gks_alu_peak_probe(int kind, long iters, void *d_sink, void *stream, double *flops)
{
    if (!flops || !d_sink || iters < 1 || kind < 0 || kind > 2) {
        gks::record_error("gks_alu_peak_probe: null pointer, iters < 1 or kind not 0, 1 or 2");
        return GKS_ERR_ARG;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        gks::record_error((std::string("gks_alu_peak_probe: ") + cudaGetErrorString(e)).c_str());
        return GKS_ERR_CUDA;
    }
    const int blocks = sms * kBlocksPerSM;
    cudaStream_t s = (cudaStream_t)stream;
    if (kind == 1)
        fma_loop_kernel<double><<<blocks, kThreads, 0, s>>>(iters, 1.0 - 0x1p-20, 0x1p-20, (double *)d_sink);
    else if (kind == 2)
        fma2_loop_kernel<<<blocks, kThreads, 0, s>>>(iters, 1.0f - 0x1p-20f, 0x1p-20f, (float *)d_sink);
    else
        fma_loop_kernel<float><<<blocks, kThreads, 0, s>>>(iters, 1.0f - 0x1p-20f, 0x1p-20f, (float *)d_sink);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        gks::record_error((std::string("gks_alu_peak_probe: ") + cudaGetErrorString(e)).c_str());
        return GKS_ERR_CUDA;
    }
    *flops = 2.0 * (double)blocks * kThreads * (double)iters * kUnroll * kChains;
    return GKS_OK;
}
