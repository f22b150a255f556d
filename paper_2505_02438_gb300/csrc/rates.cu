// Pipe-rate diagnostic: the FP32 and FP64 fused multiply-add throughput of the
// device, and of f32 -> f64 conversions.  GB300 runs FP64 at a small fraction
// of its FP32 rate; that ratio decides whether FP64-accurate element
// arithmetic runs on the FP64 pipe or in float pairs on the FP32 pipes.
#include <cstdint>

#include "internal.h"

namespace soptx {
namespace {

constexpr int kChains = 8;   // independent FMA chains per thread

__global__ void k_rate_ffma(int iters, float a, float b, float *out)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = threadIdx.x * 1e-3f + c;
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int c = 0; c < kChains; c++) x[c] = __fmaf_rn(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_rate_dfma(int iters, double a, double b, double *out)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int c = 0; c < kChains; c++) x[c] = __fma_rn(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Every iteration converts each chain's float to double and folds the bits
// into an integer (so no conversion can be hoisted or dropped).
__global__ void k_rate_cvt(int iters, float a, float b, double *out)
{
    float x[kChains];
    unsigned long long acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        x[c] = threadIdx.x * 1e-3f + c;
        acc[c] = 0ull;
    }
    for (int it = 0; it < iters; it++)
#pragma unroll
        for (int c = 0; c < kChains; c++) {
            x[c] = __fmaf_rn(x[c], a, b);
            acc[c] ^= (unsigned long long)__double_as_longlong((double)x[c]);
        }
    unsigned long long s = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s ^= acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = __longlong_as_double((long long)s);
}

}  // namespace
}  // namespace soptx

using namespace soptx;

extern "C" soptx_status soptx_measure_pipe_rates(soptx_pipe_rates *out)
{
    if (!out) SOPTX_FAIL(SOPTX_EINVAL, "out is NULL");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        SOPTX_FAIL(SOPTX_ECUDA, "device query failed");
    }
    const int blocks = sms * 8, threads = 256;
    const size_t n = (size_t)blocks * threads;
    void *buf = nullptr;
    if (dev_alloc(&buf, n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        SOPTX_FAIL(SOPTX_ENOMEM, "rate probe buffer");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    const int fi = 1 << 14, di = 1 << 9, ci = 1 << 12;
    double best[3] = {1e30, 1e30, 1e30};
    for (int k = 0; k < 3 && err == cudaSuccess; k++)
        for (int rep = 0; rep < 6 && err == cudaSuccess; rep++) {
            err = cudaEventRecord(e0, 0);
            if (k == 0) k_rate_ffma<<<blocks, threads>>>(fi, 0.999f, 1e-3f, (float *)buf);
            if (k == 1) k_rate_dfma<<<blocks, threads>>>(di, 0.999, 1e-3, (double *)buf);
            if (k == 2) k_rate_cvt<<<blocks, threads>>>(ci, 0.999f, 1e-3f, (double *)buf);
            if (err == cudaSuccess) err = cudaGetLastError();
            if (err == cudaSuccess) err = cudaEventRecord(e1, 0);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
            if (err == cudaSuccess && rep > 0 && ms < best[k]) best[k] = ms;   // the first launch warms up
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (err != cudaSuccess) SOPTX_FAIL(SOPTX_ECUDA, std::string("rate probe: ") + cudaGetErrorString(err));
    const double lanes = (double)n * kChains;
    out->ffma_per_s = lanes * fi / (best[0] * 1e-3);
    out->dfma_per_s = lanes * di / (best[1] * 1e-3);
    out->f2f64_per_s = lanes * ci / (best[2] * 1e-3);
    out->sms = sms;
    return SOPTX_OK;
}
