// Small device helpers shared by the kernels: SIMP interpolation and warp sums.
#pragma once

#include <cuda_runtime.h>

#include "df64.cuh"

namespace soptx {

// Modified SIMP, Sec. 2.1:  E(rho) = Emin + rho^p (E0 - Emin),
// E'(rho) = p rho^(p-1) (E0 - Emin).  Integer p uses repeated products.
struct SimpParams {
    double Emin, dE, p;
    int p_int;
    // float-pair copies of dE and Emin; pair_ok when p is an integer in 1..4
    // and both are zero or normal floats in [2^-100, 2^100]
    float dEh, dEl, Eminh, Eminl;
    int pair_ok;
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

// E(rho) as the float pair the assembly kernels read; a NaN low word flags a
// modulus outside [2^-60, 2^60] (those nodes are redone in FP64).  For
// integer p and rho in [2^-16, 2^16] the SIMP law is evaluated in float-pair
// arithmetic on the FP32 pipes (relative error below 2^-42); otherwise in FP64.
__device__ __forceinline__ float2 simp_E_pair(const SimpParams &sp, double r)
{
    if (sp.pair_ok && r >= 0x1p-16 && r <= 0x1p16) {
        const df x = df_split(r);
        df v = x;
        for (int i = 1; i < sp.p_int; i++) v = df_mul(v, x);
        const df E = df_add(df_mul(v, df{sp.dEh, sp.dEl}), df{sp.Eminh, sp.Eminl});
        const float a = fabsf(E.h);
        if (a >= 0x1p-60f && a <= 0x1p60f) return make_float2(E.h, E.l);
    }
    const double E = simp_E(sp, r);
    const double a = fabs(E);
    if (E == 0.0) return make_float2(0.f, 0.f);
    if (!(a >= 0x1p-60 && a <= 0x1p60)) return make_float2((float)E, __int_as_float(0x7fc00000));
    const df v = df_from_double(E);
    return make_float2(v.h, v.l);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Programmatic dependent launch (PTX griddepcontrol, sm_90 and later).  A
// kernel launched with the programmatic-serialization attribute may be
// scheduled while the kernel before it in the stream is still running, once
// every block of that kernel has executed launch_dependents; its wait blocks
// until that kernel has completed and its writes are visible.  In a kernel
// launched without the attribute both are no-ops.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with the programmatic-serialization attribute (see grid_dep_wait).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kern)(KArgs...), int grid, int block, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

struct Material;
SimpParams simp_params(const Material &m);

// Walsh-sector blocks B_c[i][j] of a box element's K^0 as float pairs, passed
// to a kernel by value: kernel parameters live in the constant bank, which the
// FP32 instructions read as operands without a shared-memory load.
template <int D> struct SectorTable {
    float2 b[(1 << D) * D * D];
};

// Entries of the sector blocks that vanish on every box: a row or column
// whose Walsh mode is the rigid translation (c xor e_i = 0), and the coupling
// of components i != j whose axes lie on different sides of the sector
// (bit i of c != bit j of c), which the box's reflection symmetry cancels.
// The kernels skip them; the host stores them as exact zeros.
__host__ __device__ constexpr bool sector_zero(int c, int i, int j)
{
    return (c ^ (1 << i)) == 0 || (c ^ (1 << j)) == 0 || (i != j && ((c >> i) & 1) != ((c >> j) & 1));
}

// Sum of `mine` over blocks 0 .. nblk - 1 (the grid, or the blocks one request
// has in a grouped launch) into *c, deterministically: each block writes its
// partial (a fixed-order butterfly per warp, then the warps in order), the last block to finish (an
// atomic ticket on *counter) adds all partials in index order and resets the
// ticket for the next call.  blockDim.x must be a power of two <= 256, and
// calls that share `partial` / `counter` must not overlap on the device.
__device__ __forceinline__ void grid_sum_last_block_n(double mine, double *__restrict__ partial,
                                                      unsigned *__restrict__ counter, double *__restrict__ c,
                                                      unsigned bid, unsigned nblk)
{
    __shared__ double red[256];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if (lane == 0) red[warp] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; w++) t += red[w];
        partial[bid] = t;
        __threadfence();
        last = atomicAdd(counter, 1u) == nblk - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)nblk; i += blockDim.x) t += __ldcg(partial + i);
    red[threadIdx.x] = t;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *c = red[0];
        *counter = 0u;
    }
}

// The same over the launch's own grid.
__device__ __forceinline__ void grid_sum_last_block(double mine, double *__restrict__ partial,
                                                    unsigned *__restrict__ counter, double *__restrict__ c)
{
    grid_sum_last_block_n(mine, partial, counter, c, blockIdx.x, gridDim.x);
}

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
