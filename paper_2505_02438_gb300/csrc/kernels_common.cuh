// Small device helpers shared by the kernels: SIMP interpolation and warp sums.
#pragma once

#include <cuda_runtime.h>

namespace soptx {

// Modified SIMP, Sec. 2.1:  E(rho) = Emin + rho^p (E0 - Emin),
// E'(rho) = p rho^(p-1) (E0 - Emin).  Integer p uses repeated products.
struct SimpParams {
    double Emin, dE, p;
    int p_int;
};

__device__ __forceinline__ double simp_pow(const SimpParams &sp, double r, int minus)
{
    if (sp.p_int > 0) {
        double v = 1.0;
        for (int i = 0; i < sp.p_int - minus; i++) v *= r;
        return v;
    }
    return pow(r, sp.p - minus);
}

__device__ __forceinline__ double simp_E(const SimpParams &sp, double r)
{
    return sp.Emin + simp_pow(sp, r, 0) * sp.dE;
}

__device__ __forceinline__ double simp_dE(const SimpParams &sp, double r)
{
    return sp.p * simp_pow(sp, r, 1) * sp.dE;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct Material;
SimpParams simp_params(const Material &m);

// Element-matrix entries: float pairs (FP64 element matrices, value h + l) or
// plain floats (FP32 element matrices).
template <typename KT> struct KLoad;
template <> struct KLoad<float2> {
    static __device__ __forceinline__ float2 raw(const float2 *p) { return __ldcs(p); }
    static __device__ __forceinline__ double get64(const float2 *p)
    {
        const float2 v = *p;
        return (double)v.x + (double)v.y;
    }
};
template <> struct KLoad<float> {
    static __device__ __forceinline__ float2 raw(const float *p) { return make_float2(__ldcs(p), 0.f); }
    static __device__ __forceinline__ double get64(const float *p) { return (double)*p; }
};

}  // namespace soptx
