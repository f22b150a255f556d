// The step after assembly (include/soptx_solve.h): y = K x on the mesh's CSR
// values, and Jacobi-preconditioned conjugate gradients for K u = f under
// Dirichlet constraints.
//
//  k_spmv      : four nodes per warp, eight lanes per node; each lane takes
//                the columns c, c+8, ... of the node's column list (shared by
//                its d rows) and accumulates the first d-1 row sums in
//                float-pair arithmetic (FP32 pipes) and the last row's with
//                FP64 fused multiply-adds (FP64 pipe); the node's lanes then
//                add their sums by a fixed butterfly.
//                Optionally zeroes constrained rows and sums p . y over the grid.
//  k_cg_*      : the element-wise CG updates with their dot products; every
//                grid sum is a fixed-order block partial plus a last-block
//                total, so the iterates are bitwise reproducible.
// One FP64 fused multiply-add per stored value would bind the product to this
// GPU's FP64 pipe (measured: 76% busy, 177 us on the hex Q1 120x40x40 matrix)
// and float pairs for all of them to the issue rate (114 us), so the rows are
// split between the two.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "df64.cuh"
#include "internal.h"
#include "kernels_common.cuh"
#include "../../include/soptx_solve.h"

namespace soptx {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSpWarps = 8;
constexpr int kCgThreads = 256;

// Sums of NV values over the grid into out[0..NV), deterministic (a fixed
// tree per block, the last block to finish adds the block partials in index
// order).  partial: [NV][gridDim.x]; *counter is zero between calls.
template <int NV>
__device__ __forceinline__ void grid_sums(const double (&mine)[NV], double *__restrict__ partial,
                                          unsigned *__restrict__ counter, double *__restrict__ out)
{
    __shared__ double red[NV][kCgThreads / 32];
    __shared__ double fin[NV][kCgThreads];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        double v = mine[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < NV; k++) {
            double t = 0.0;
            for (int w = 0; w < nw; w++) t += red[k][w];
            partial[(size_t)k * gridDim.x + blockIdx.x] = t;
        }
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int k = 0; k < NV; k++) {
        double t = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += __ldcg(partial + (size_t)k * gridDim.x + b);
        fin[k][threadIdx.x] = t;
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < NV; k++) fin[k][threadIdx.x] += fin[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < NV; k++) out[k] = fin[k][0];
        *counter = 0u;
    }
}

template <int D>
__global__ void __launch_bounds__(kSpWarps * 32)
k_spmv(int64_t nn, const int64_t *__restrict__ node_off, const int32_t *__restrict__ indices,
       const double *__restrict__ vals, const double *__restrict__ x, double *__restrict__ y,
       const uint8_t *__restrict__ fixed, const double *__restrict__ dotv, double *__restrict__ partial,
       unsigned *__restrict__ counter, double *__restrict__ dot_out)
{
    // inside the CG loop this kernel is a dependent launch: nothing is read before the wait
    grid_dep_wait();
    grid_dep_launch();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 3, c = lane & 7;       // 4 nodes per warp, 8 lanes per node
    double mine = 0.0;
    const int64_t step = (int64_t)gridDim.x * kSpWarps * 4;
    for (int64_t n0 = ((int64_t)blockIdx.x * kSpWarps + warp) * 4; n0 < nn; n0 += step) {
        const int64_t n = n0 + g;
        const bool has = n < nn;
        // float-pair sums of the node's d rows over this lane's columns c, c+8, ...
        // rows 0 .. d-2 in float pairs on the FP32 pipes, row d-1 in FP64
        // (DFMA) on the FP64 pipe, so that both pipes share the products
        float S[D], C[D];
        double Sd = 0.0;
#pragma unroll
        for (int i = 0; i < D; i++) S[i] = C[i] = 0.f;
        int len = 0;
        if (has) {
            const int64_t off = node_off[n];
            len = D * (int)(node_off[n + 1] - off);
            const int64_t base = (int64_t)D * D * off;
            const int32_t *cols = indices + base;                 // the node's rows share row 0's columns
            const double *v = vals + base;
            // four column rounds per pass: every load of the pass is issued
            // before the arithmetic (a round past the row reads nothing and adds 0)
            constexpr int U = 4;
            for (int t0 = c; t0 < len; t0 += 8 * U) {
                int cj[U];
                double xr[U], vr[U][D];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int t = t0 + 8 * u;
                    cj[u] = t < len ? cols[t] : -1;
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int t = t0 + 8 * u;
                    xr[u] = cj[u] >= 0 ? x[cj[u]] : 0.0;
#pragma unroll
                    for (int i = 0; i < D; i++) vr[u][i] = t < len ? __ldcs(v + (int64_t)i * len + t) : 0.0;
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const df xv = df_split_z(xr[u]);
#pragma unroll
                    for (int i = 0; i < D - 1; i++) {
                        const df pr = df_mul_raw(df_split_z(vr[u][i]), xv);
                        float s2, err;
                        two_sum(S[i], pr.h, s2, err);
                        S[i] = s2;
                        C[i] = __fadd_rn(C[i], __fadd_rn(pr.l, err));
                    }
                    Sd = fma(vr[u][D - 1], xr[u], Sd);
                }
            }
        }
        // fixed-order butterfly over the node's 8 lanes; every lane ends with the same bits
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            const double So = __shfl_xor_sync(kFull, Sd, o);
            Sd = (c & o) == 0 ? Sd + So : So + Sd;
        }
#pragma unroll
        for (int i = 0; i < D - 1; i++)
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const float So = __shfl_xor_sync(kFull, S[i], o), Co = __shfl_xor_sync(kFull, C[i], o);
                // order the pair by lane so both partners add the same operands in the same order
                const bool lo = (c & o) == 0;
                const float Sa = lo ? S[i] : So, Ca = lo ? C[i] : Co, Sb = lo ? So : S[i], Cb = lo ? Co : C[i];
                float s2, err;
                two_sum(Sa, Sb, s2, err);
                S[i] = s2;
                C[i] = __fadd_rn(__fadd_rn(Ca, Cb), err);
            }
        if (has && c < D) {
            float h = 0.f, l = 0.f;
#pragma unroll
            for (int i = 0; i < D - 1; i++)
                if (i == c) two_sum(S[i], C[i], h, l);
            const int64_t row = (int64_t)D * n + c;
            const double sv = c == D - 1 ? Sd : df_to_double(h, l);
            const double yv = (fixed && fixed[row]) ? 0.0 : sv;
            y[row] = yv;
            if (dotv) mine = fma(dotv[row], yv, mine);
        }
    }
    if (dot_out) {
        const double m1[1] = {mine};
        grid_sums<1>(m1, partial, counter, dot_out);
    }
}

// diag[row] = 1 / K[row][row] (1 on constrained rows): the diagonal sits in the node's own column block;
// a binary search over row 0's sorted columns finds it.  A free row with a
// non-positive diagonal raises *bad.
template <int D>
__global__ void k_diag(int64_t nn, const int64_t *__restrict__ node_off, const int32_t *__restrict__ indices,
                       const double *__restrict__ vals, const uint8_t *__restrict__ fixed, double *__restrict__ diag,
                       int *__restrict__ bad)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < D * nn; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t n = r / D;
        const int i = (int)(r - n * D);
        const int64_t off = node_off[n];
        const int len = D * (int)(node_off[n + 1] - off);
        const int64_t base = (int64_t)D * D * off;
        const int32_t *cols = indices + base;
        int lo = 0, hi = len;
        const int32_t want = (int32_t)(D * n);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cols[mid] < want) lo = mid + 1;
            else hi = mid;
        }
        double dv = 0.0;
        if (lo < len && cols[lo] == want) dv = vals[base + (int64_t)i * len + lo + i];
        const bool fx = fixed[r] != 0;
        // the Jacobi preconditioner is applied as a product with the reciprocal: an
        // FP64 division per dof per iteration costs more than the rest of the update
        diag[r] = fx ? 1.0 : (dv > 0.0 ? 1.0 / dv : 0.0);
        if (!fx && !(dv > 0.0)) atomicExch(bad, 1);
    }
}

// u = 0 on the free dofs (the prescribed values stay on the constrained ones)
__global__ void k_cg_zero_free(int64_t ndof, const uint8_t *__restrict__ fixed, double *__restrict__ u)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < ndof; r += (int64_t)gridDim.x * blockDim.x)
        if (!fixed[r]) u[r] = 0.0;
}

// r = f - K u_D on the free rows (q holds K u_D with constrained rows zeroed),
// z = r / diag (as r times the stored reciprocal), p = z; sums r.z and r.r
__global__ void __launch_bounds__(kCgThreads)
k_cg_start(int64_t ndof, const uint8_t *__restrict__ fixed, const double *__restrict__ f,
           const double *__restrict__ q, const double *__restrict__ dinv, double *__restrict__ r,
           double *__restrict__ z, double *__restrict__ p, double *__restrict__ partial,
           unsigned *__restrict__ counter, double *__restrict__ out)
{
    double m[2] = {0.0, 0.0};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ndof; k += (int64_t)gridDim.x * blockDim.x) {
        const double rv = fixed[k] ? 0.0 : f[k] - q[k];
        const double zv = rv * dinv[k];
        r[k] = rv;
        z[k] = zv;
        p[k] = zv;
        m[0] = fma(rv, zv, m[0]);
        m[1] = fma(rv, rv, m[1]);
    }
    grid_sums<2>(m, partial, counter, out);
}

// alpha = (r.z) / (p.q); u += alpha p; r -= alpha q; z = r / diag (times the reciprocal); sums r.z, r.r
__global__ void __launch_bounds__(kCgThreads)
k_cg_step(int64_t ndof, const uint8_t *__restrict__ fixed, const double *__restrict__ dinv,
          const double *__restrict__ p, const double *__restrict__ q, double *__restrict__ u,
          double *__restrict__ r, double *__restrict__ z, const double *__restrict__ rz_old,
          const double *__restrict__ pq, double *__restrict__ partial, unsigned *__restrict__ counter,
          double *__restrict__ out)
{
    grid_dep_wait();
    grid_dep_launch();
    // one FP64 division per block (a division per thread would cost more than the pass)
    __shared__ double alpha_s;
    if (threadIdx.x == 0) {
        const double den = *pq;
        alpha_s = den != 0.0 ? *rz_old / den : 0.0;
    }
    __syncthreads();
    const double alpha = alpha_s;
    double m[2] = {0.0, 0.0};
    // four dofs per thread and pass, their loads issued together
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k0 < ndof; k0 += 4 * stride) {
        double pv[4], qv[4], uv[4], rv[4], dv[4];
        bool on[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const int64_t k = k0 + t * stride;
            on[t] = k < ndof && !fixed[k];
            pv[t] = on[t] ? p[k] : 0.0;
            qv[t] = on[t] ? q[k] : 0.0;
            uv[t] = on[t] ? u[k] : 0.0;
            rv[t] = on[t] ? r[k] : 0.0;
            dv[t] = on[t] ? dinv[k] : 0.0;
        }
#pragma unroll
        for (int t = 0; t < 4; t++) {
            if (!on[t]) continue;
            const int64_t k = k0 + t * stride;
            u[k] = fma(alpha, pv[t], uv[t]);
            const double rn = fma(-alpha, qv[t], rv[t]);
            const double zv = rn * dv[t];
            r[k] = rn;
            z[k] = zv;
            m[0] = fma(rn, zv, m[0]);
            m[1] = fma(rn, rn, m[1]);
        }
    }
    grid_sums<2>(m, partial, counter, out);
}

// beta = (r.z)_new / (r.z)_old; p = z + beta p (zero on constrained dofs)
__global__ void k_cg_direction(int64_t ndof, const uint8_t *__restrict__ fixed, const double *__restrict__ z,
                               double *__restrict__ p, const double *__restrict__ rz_new,
                               const double *__restrict__ rz_old)
{
    grid_dep_wait();
    grid_dep_launch();
    __shared__ double beta_s;
    if (threadIdx.x == 0) {
        const double den = *rz_old;
        beta_s = den != 0.0 ? *rz_new / den : 0.0;
    }
    __syncthreads();
    const double beta = beta_s;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ndof; k += (int64_t)gridDim.x * blockDim.x)
        p[k] = fixed[k] ? 0.0 : fma(beta, p[k], z[k]);
}

int spmv_grid(int64_t nn) { return (int)std::max<int64_t>(1, std::min<int64_t>((nn + 2 * kSpWarps - 1) / (2 * kSpWarps), 152 * 8)); }
// Passes with a grid sum: two blocks per SM, each thread taking several dofs (the
// FP64 butterfly of the sum is paid once per thread).  Plain passes: one dof per
// thread up to 152 x 32 blocks, so that all their loads are in flight at once.
#ifndef SOPTX_CG_BLOCKS_PER_SM
#define SOPTX_CG_BLOCKS_PER_SM 2
#endif
int cg_grid(int64_t ndof) { return (int)std::max<int64_t>(1, std::min<int64_t>((ndof + kCgThreads - 1) / kCgThreads, 152 * SOPTX_CG_BLOCKS_PER_SM)); }
static int cg_grid_wide(int64_t ndof)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((ndof + kCgThreads - 1) / kCgThreads, 152 * 32));
}

cudaError_t launch_spmv(const soptx_mesh_s &m, const double *vals, const double *x, double *y, const uint8_t *fixed,
                        const double *dotv, double *partial, unsigned *counter, double *dot_out, cudaStream_t st,
                        bool dependent = false)
{
    const auto &h = m.h;
    if (h.nn == 0) return cudaSuccess;
    const int grid = spmv_grid(h.nn);
    if (dependent) {
        if (h.dim == 3)
            return launch_dependent(k_spmv<3>, grid, kSpWarps * 32, st, h.nn, m.d.node_off, m.d.indices, vals, x, y,
                                    fixed, dotv, partial, counter, dot_out);
        return launch_dependent(k_spmv<2>, grid, kSpWarps * 32, st, h.nn, m.d.node_off, m.d.indices, vals, x, y,
                                fixed, dotv, partial, counter, dot_out);
    }
    if (h.dim == 3)
        k_spmv<3><<<grid, kSpWarps * 32, 0, st>>>(h.nn, m.d.node_off, m.d.indices, vals, x, y, fixed, dotv, partial,
                                                  counter, dot_out);
    else
        k_spmv<2><<<grid, kSpWarps * 32, 0, st>>>(h.nn, m.d.node_off, m.d.indices, vals, x, y, fixed, dotv, partial,
                                                  counter, dot_out);
    return cudaGetLastError();
}

soptx_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return SOPTX_OK;
    cudaGetLastError();
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SOPTX_ENOMEM : SOPTX_ECUDA;
}

__global__ void k_scale_by_2g(int64_t n, const double *__restrict__ gout, double *__restrict__ y)
{
    const double f = 2.0 * (*gout);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        y[k] *= f;
}

}  // namespace

// out = 2 g K u from the assembled values (the backward's u-gradient)
cudaError_t launch_scaled_product(const soptx_mesh_s &m, const double *vals, const double *u, const double *gout,
                                  double *out, cudaStream_t st)
{
    const auto &h = m.h;
    if (h.nn == 0) return cudaSuccess;
    cudaError_t e = launch_spmv(m, vals, u, out, nullptr, nullptr, nullptr, nullptr, nullptr, st);
    if (e != cudaSuccess) return e;
    k_scale_by_2g<<<cg_grid_wide(h.ndof), kCgThreads, 0, st>>>(h.ndof, gout, out);
    return cudaGetLastError();
}

}  // namespace soptx

using namespace soptx;

extern "C" {

soptx_status soptx_spmv(soptx_mesh m, const double *d_vals, const double *d_x, double *d_y, void *stream)
{
    if (!m) SOPTX_FAIL(SOPTX_EINVAL, "mesh is NULL");
    if (m->h.nnz > 0 && (!d_vals || !d_x || !d_y)) SOPTX_FAIL(SOPTX_EINVAL, "d_vals / d_x / d_y is NULL");
    return cuda_fail(launch_spmv(*m, d_vals, d_x, d_y, nullptr, nullptr, nullptr, nullptr, nullptr,
                                 (cudaStream_t)stream),
                     "soptx_spmv");
}

soptx_status soptx_solve_cg(soptx_mesh m, const double *d_vals, const uint8_t *d_fixed, const double *d_f,
                            double *d_u, const soptx_cg_opts *o, void *stream, soptx_cg_result *res)
{
    if (!m || !o || !res) SOPTX_FAIL(SOPTX_EINVAL, "mesh / opts / result is NULL");
    *res = soptx_cg_result{0, 0, 0.0};
    if (!(o->rtol > 0.0) || o->max_iter < 1 || o->check_every < 1)
        SOPTX_FAIL(SOPTX_EINVAL, "need rtol > 0, max_iter >= 1, check_every >= 1");
    const auto &h = m->h;
    if (h.ndof == 0) {
        res->converged = 1;
        return SOPTX_OK;
    }
    if (!d_vals || !d_fixed || !d_f || !d_u) SOPTX_FAIL(SOPTX_EINVAL, "d_vals / d_fixed / d_f / d_u is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    auto &d = m->d;
    const int sgrid = spmv_grid(h.nn), cgrid = cg_grid(h.ndof);
    const int pmax = std::max(sgrid, cgrid);
    // workspace: r z p q 1/diag [ndof], scalars [8], partials [2][pmax], counters, flag
    if (!d.cg) {
        const size_t bytes = ((size_t)5 * h.ndof + 8 + 2 * (size_t)pmax) * sizeof(double) + 64;
        void *p = nullptr;
        cudaError_t e = dev_alloc(&p, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "CG workspace");
        e = cudaMemsetAsync(p, 0, bytes, st);
        if (e != cudaSuccess) {
            cudaFree(p);
            return cuda_fail(e, "CG workspace");
        }
        d.cg = (double *)p;
        m->device_bytes += (int64_t)bytes;
    }
    double *r = d.cg, *z = r + h.ndof, *pv = z + h.ndof, *q = pv + h.ndof, *diag = q + h.ndof;
    // scalars: 2: p.q; 4,5 and 6,7: (r.z, r.r) of the even and odd iterates (ping-pong)
    double *S = diag + h.ndof;
    double *partial = S + 8;
    unsigned *counter = (unsigned *)(partial + 2 * (size_t)pmax);
    int *bad = (int *)(counter + 4);

    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        const int dg = cg_grid(h.ndof);
        if (h.dim == 3) k_diag<3><<<dg, kCgThreads, 0, st>>>(h.nn, d.node_off, d.indices, d_vals, d_fixed, diag, bad);
        else k_diag<2><<<dg, kCgThreads, 0, st>>>(h.nn, d.node_off, d.indices, d_vals, d_fixed, diag, bad);
        e = cudaGetLastError();
    }
    int bad_h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "soptx_solve_cg");
    if (bad_h) SOPTX_FAIL(SOPTX_EINVAL, "a free dof has a non-positive diagonal (no element touches it?)");

    // the scale of the residual test: ||f - K u_D|| on the free rows
    double rr0 = 0.0;
    // z = u_D on the constrained dofs, 0 on the free ones
    e = cudaMemcpyAsync(z, d_u, h.ndof * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        k_cg_zero_free<<<cgrid, kCgThreads, 0, st>>>(h.ndof, d_fixed, z);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_spmv(*m, d_vals, z, q, d_fixed, nullptr, nullptr, nullptr, nullptr, st);
    if (e == cudaSuccess) {
        k_cg_start<<<cgrid, kCgThreads, 0, st>>>(h.ndof, d_fixed, d_f, q, diag, r, z, pv, partial, counter, S + 4);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&rr0, S + 5, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "soptx_solve_cg");
    // start: u = u_D and 0 (or the given guess) on the free rows, r = f - K u, z = p = r / diag
    if (!o->warm_start) {
        k_cg_zero_free<<<cgrid, kCgThreads, 0, st>>>(h.ndof, d_fixed, d_u);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_spmv(*m, d_vals, d_u, q, d_fixed, nullptr, nullptr, nullptr, nullptr, st);
    if (e == cudaSuccess) {
        k_cg_start<<<cgrid, kCgThreads, 0, st>>>(h.ndof, d_fixed, d_f, q, diag, r, z, pv, partial, counter, S + 4);
        e = cudaGetLastError();
    }
    double rr = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&rr, S + 5, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "soptx_solve_cg");
    const double r0 = std::sqrt(rr0);
    if (r0 == 0.0 || std::sqrt(rr) <= o->rtol * r0) {
        res->converged = 1;
        res->rel_residual = r0 == 0.0 ? 0.0 : std::sqrt(rr) / r0;
        return SOPTX_OK;
    }
    // One CG iteration: three dependent launches (each is scheduled while the one
    // before it finishes and waits for it before reading anything).
    auto iteration = [&](int it_, cudaStream_t s_) -> cudaError_t {
        const int par = it_ & 1;
        double *old_pair = S + 4 + 2 * par, *new_pair = S + 4 + 2 * (par ^ 1);
        // q = K p (constrained rows zero), p.q -> S[2]
        cudaError_t err = launch_spmv(*m, d_vals, pv, q, d_fixed, pv, partial, counter, S + 2, s_, true);
        // u, r, z; (r.z, r.r) -> the other pair
        if (err == cudaSuccess)
            err = launch_dependent(k_cg_step, cgrid, kCgThreads, s_, h.ndof, d_fixed, diag, pv, q, d_u, r, z,
                                   old_pair, S + 2, partial, counter, new_pair);
        if (err == cudaSuccess)
            err = launch_dependent(k_cg_direction, cg_grid_wide(h.ndof), kCgThreads, s_, h.ndof, d_fixed, z, pv,
                                   new_pair, old_pair);
        return err;
    };
    // Between two convergence checks (an even number of iterations, at most 100) the
    // launches are replayed as one CUDA graph: the same kernels in the same order, so
    // the iterates are bitwise those of the launch-by-launch loop, without the host's
    // launch cost per kernel (the bound of small meshes).  The graph is kept with the
    // mesh and updated in place when the call's vectors change.
    const int G = (o->check_every % 2 == 0 && o->check_every <= 100) ? o->check_every : 0;
    bool graph = G > 0 && o->max_iter >= G;
    if (graph) {
        const void *key[4] = {d_vals, d_fixed, d_u, (const void *)(intptr_t)G};
        bool same = d.cg_exec != nullptr;
        for (int k = 0; k < 4; k++) same = same && d.cg_key[k] == key[k];
        if (!same) {
            cudaError_t ge = d.cg_cap ? cudaSuccess : cudaStreamCreateWithFlags(&d.cg_cap, cudaStreamNonBlocking);
            cudaGraph_t g = nullptr;
            if (ge == cudaSuccess) ge = cudaStreamBeginCapture(d.cg_cap, cudaStreamCaptureModeThreadLocal);
            if (ge == cudaSuccess) {
                cudaError_t ce = cudaSuccess;
                for (int k = 0; k < G && ce == cudaSuccess; k++) ce = iteration(k, d.cg_cap);
                ge = cudaStreamEndCapture(d.cg_cap, &g);
                if (ce != cudaSuccess) ge = ce;
            }
            if (ge == cudaSuccess && d.cg_exec) {
                cudaGraphExecUpdateResultInfo info;
                if (cudaGraphExecUpdate(d.cg_exec, g, &info) != cudaSuccess) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(d.cg_exec);
                    d.cg_exec = nullptr;
                }
            }
            if (ge == cudaSuccess && !d.cg_exec) ge = cudaGraphInstantiate(&d.cg_exec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (ge == cudaSuccess) {
                for (int k = 0; k < 4; k++) d.cg_key[k] = key[k];
            } else {
                cudaGetLastError();
                if (d.cg_exec) cudaGraphExecDestroy(d.cg_exec);
                d.cg_exec = nullptr;
                graph = false;          // fall back to launching the kernels one by one
            }
        }
    }
    int it = 0;
    while (it < o->max_iter) {
        if (graph && it + G <= o->max_iter) {
            e = cudaGraphLaunch(d.cg_exec, st);
            if (e != cudaSuccess) break;
            it += G;
        } else {
            e = iteration(it, st);
            if (e != cudaSuccess) break;
            it++;
        }
        if (it % o->check_every == 0 || it == o->max_iter) {
            double *latest = S + 4 + 2 * (it & 1);
            e = cudaMemcpyAsync(&rr, latest + 1, sizeof(double), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) break;
            if (std::sqrt(rr) <= o->rtol * r0) {
                res->converged = 1;
                break;
            }
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "soptx_solve_cg");
    res->iterations = it;
    res->rel_residual = std::sqrt(rr) / r0;
    return SOPTX_OK;
}

}  // extern "C"
