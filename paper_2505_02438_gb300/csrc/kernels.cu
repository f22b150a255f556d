// Device kernels of the general (unstructured) path, sm_103a.
//
//  k_element_matrices : K_e^0 from the exact reference integrals and each
//                       cell's inverse Jacobian (Sec. 3.2.2 fast assembly).
//  k_assemble_gather  : K(rho) = sum_e E(rho_e) K_e^0 (Sec. 2.2) by a
//                       node-owner gather: one warp owns the d rows of one node,
//                       walks the node's incident cells in ascending order and
//                       accumulates in shared memory; each CSR value is summed
//                       in ascending cell order, no atomics.
//  k_sensitivity      : dc_e = -E'(rho_e) u_e^T K_e^0 u_e (Appendix D) and
//                       per-block partial sums of E_e u_e^T K_e^0 u_e.
//  k_reduce_partials  : c = sum of the block partials in a fixed order.
//  k_Ku               : (K(rho) u) without forming K, for the u-gradient.
#include <cstdint>

#include "internal.h"
#include "kernels_common.cuh"

namespace soptx {
namespace {

constexpr int kWarps = 8;   // warps per CTA for the warp-per-item kernels

template <typename KT>
__global__ void k_element_matrices(int dim, int nb, int64_t n_elems, const double *__restrict__ geo,
                                   const double *__restrict__ M, double lam, double mu,
                                   KT *__restrict__ K)
{
    const int ldof = dim * nb, ng = dim * dim + 1;
    for (int64_t e = blockIdx.x; e < n_elems; e += gridDim.x) {
        KT G[9], det;
        for (int q = 0; q < dim * dim; q++) G[q] = (KT)geo[e * ng + q];
        det = (KT)geo[e * ng + dim * dim];
        KT *Ke = K + (size_t)e * ldof * ldof;
        for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
            const int a = t / nb, b = t % nb;
            KT Mab[9];
            for (int kl = 0; kl < dim * dim; kl++) Mab[kl] = (KT)M[((size_t)kl * nb + a) * nb + b];
            // P[i][j] = |det J| sum_kl G[k][i] G[l][j] M^{kl}_{ab}   (G[k][i] = (J^-1)_{k i})
            KT P[9];
            for (int i = 0; i < dim; i++)
                for (int j = 0; j < dim; j++) {
                    KT s = 0;
                    for (int k = 0; k < dim; k++) {
                        KT w = 0;
                        for (int l = 0; l < dim; l++) w += Mab[k * dim + l] * G[l * dim + j];
                        s += G[k * dim + i] * w;
                    }
                    P[i * dim + j] = det * s;
                }
            KT tr = 0;
            for (int m = 0; m < dim; m++) tr += P[m * dim + m];
            for (int i = 0; i < dim; i++)
                for (int j = 0; j < dim; j++) {
                    KT v = (KT)lam * P[i * dim + j] + (KT)mu * P[j * dim + i];
                    if (i == j) v += (KT)mu * tr;
                    Ke[(size_t)(dim * a + i) * ldof + dim * b + j] = v;
                }
        }
    }
}

template <int D, typename KT>
__global__ void __launch_bounds__(kWarps * 32)
k_assemble_gather(int64_t nn, int nb, int max_deg, const int64_t *__restrict__ node_off,
                  const int32_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc,
                  const uint16_t *__restrict__ pos, const KT *__restrict__ K, int64_t kstride,
                  const double *__restrict__ rho, SimpParams sp, double *__restrict__ vals)
{
    extern __shared__ double smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ldof = D * nb;
    double *acc = smem + (size_t)warp * D * D * max_deg;
    for (int64_t n = (int64_t)blockIdx.x * kWarps + warp; n < nn; n += (int64_t)gridDim.x * kWarps) {
        const int64_t off = node_off[n];
        const int deg = (int)(node_off[n + 1] - off);
        const int blk = D * D * deg;
        for (int t = lane; t < blk; t += 32) acc[t] = 0.0;
        __syncwarp();
        for (int32_t q = inc_ptr[n]; q < inc_ptr[n + 1]; q++) {
            const int32_t ea = inc[q];
            const int64_t e = ea / nb;
            const int a = ea - (int)e * nb;
            const double E = simp_E(sp, rho[e]);
            const KT *Ke = K + e * kstride;
            for (int t = lane; t < nb * D * D; t += 32) {
                const int b = t / (D * D), i = (t / D) % D, j = t % D;
                const double kv = (double)Ke[(D * a + i) * ldof + D * b + j];
                const int p = pos[(int64_t)q * nb + b];
                acc[i * (D * deg) + D * p + j] += E * kv;
            }
            __syncwarp();
        }
        double *out = vals + (int64_t)D * D * off;
        for (int t = lane; t < blk; t += 32) out[t] = acc[t];
        __syncwarp();
    }
}

// One warp per element; u_e staged in shared memory.  `gscale` == nullptr:
// out[e] = -E'(rho_e) s_e (the compliance sensitivity); otherwise
// out[e] = (*gscale) E'(rho_e) s_e (the rho-gradient of u^T K(rho) u).
template <int D, typename KT>
__global__ void __launch_bounds__(kWarps * 32)
k_sensitivity(int64_t nc, int nb, const int32_t *__restrict__ cell_node, const KT *__restrict__ K,
              int64_t kstride, const double *__restrict__ rho, const double *__restrict__ u,
              SimpParams sp, const double *__restrict__ gscale, double *__restrict__ out,
              double *__restrict__ partial)
{
    __shared__ double ue_s[kWarps][kMaxLdof];
    __shared__ double wsum[kWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ldof = D * nb;
    const double g = gscale ? *gscale : -1.0;
    double mine = 0.0;   // this warp's running sum of E_e s_e, in element order
    for (int64_t e = (int64_t)blockIdx.x * kWarps + warp; e < nc; e += (int64_t)gridDim.x * kWarps) {
        for (int r = lane; r < ldof; r += 32) {
            const int b = r / D, j = r % D;
            ue_s[warp][r] = u[(int64_t)D * cell_node[e * nb + b] + j];
        }
        __syncwarp();
        const KT *Ke = K + e * kstride;
        double s = 0.0;
        for (int r = lane; r < ldof; r += 32) {
            double kr = 0.0;
            for (int c = 0; c < ldof; c++) kr += (double)Ke[r * ldof + c] * ue_s[warp][c];
            s += ue_s[warp][r] * kr;
        }
        s = warp_sum(s);
        if (lane == 0) {
            out[e] = g * simp_dE(sp, rho[e]) * s;
            mine += simp_E(sp, rho[e]) * s;
        }
        __syncwarp();
    }
    if (partial) {
        if (lane == 0) wsum[warp] = mine;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kWarps; w++) t += wsum[w];
            partial[blockIdx.x] = t;
        }
    }
}

// (K(rho) u)[d n + i] * factor, factor = 2 * (*gout): warp per node.
template <int D, typename KT>
__global__ void __launch_bounds__(kWarps * 32)
k_Ku(int64_t nn, int nb, const int32_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc,
     const int32_t *__restrict__ cell_node, const KT *__restrict__ K, int64_t kstride,
     const double *__restrict__ rho, const double *__restrict__ u, SimpParams sp,
     const double *__restrict__ gout, double *__restrict__ out)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ldof = D * nb;
    const double f = 2.0 * (*gout);
    for (int64_t n = (int64_t)blockIdx.x * kWarps + warp; n < nn; n += (int64_t)gridDim.x * kWarps) {
        double acc[D];
        for (int i = 0; i < D; i++) acc[i] = 0.0;
        for (int32_t q = inc_ptr[n]; q < inc_ptr[n + 1]; q++) {
            const int32_t ea = inc[q];
            const int64_t e = ea / nb;
            const int a = ea - (int)e * nb;
            const KT *Ke = K + e * kstride;
            double part[D];
            for (int i = 0; i < D; i++) part[i] = 0.0;
            for (int c = lane; c < ldof; c += 32) {
                const int b = c / D, j = c % D;
                const double uc = u[(int64_t)D * cell_node[e * nb + b] + j];
                for (int i = 0; i < D; i++) part[i] += (double)Ke[(D * a + i) * ldof + c] * uc;
            }
            const double E = simp_E(sp, rho[e]);
            for (int i = 0; i < D; i++) acc[i] += E * warp_sum(part[i]);
        }
        if (lane < D) {
            double v = acc[0];
            for (int i = 1; i < D; i++)
                if (lane == i) v = acc[i];
            out[(int64_t)D * n + lane] = f * v;
        }
    }
}

int grid_for(int64_t items, int per_block)
{
    int64_t g = (items + per_block - 1) / per_block;
    const int64_t cap = 152 * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

__global__ void k_reduce_partials(int n, const double *__restrict__ partial, double *__restrict__ c)
{
    // fixed-order tree over a fixed number of block partials
    __shared__ double s[256];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += partial[i];
    s[threadIdx.x] = t;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *c = s[0];
}

SimpParams simp_params(const Material &m)
{
    SimpParams sp;
    sp.Emin = m.Emin;
    sp.dE = m.dE;
    sp.p = m.p;
    sp.p_int = m.p_int;
    return sp;
}

cudaError_t launch_element_matrices(const soptx_mesh_s &m, int64_t n_elems, cudaStream_t st)
{
    const auto &h = m.h;
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(n_elems, 1), 152 * 64);
    const int threads = 128;
    if (n_elems == 0) return cudaSuccess;
    if (m.prec == SOPTX_ELEM_FP32)
        k_element_matrices<float><<<grid, threads, 0, st>>>(h.dim, h.nb, n_elems, m.d.geo, m.d.M,
                                                            m.mat.lam, m.mat.mu, (float *)m.d.K);
    else
        k_element_matrices<double><<<grid, threads, 0, st>>>(h.dim, h.nb, n_elems, m.d.geo, m.d.M,
                                                             m.mat.lam, m.mat.mu, (double *)m.d.K);
    return cudaGetLastError();
}

static int64_t kstride_of(const soptx_mesh_s &m)
{
    return m.path == SOPTX_PATH_CACHED ? (int64_t)m.h.ldof * m.h.ldof : 0;
}

template <int D, typename KT>
static cudaError_t assemble_t(const soptx_mesh_s &m, const double *rho, double *vals, cudaStream_t st)
{
    const auto &h = m.h;
    const size_t sm = (size_t)kWarps * D * D * h.max_deg * sizeof(double);
    auto kern = k_assemble_gather<D, KT>;
    if (sm > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (err != cudaSuccess) return err;
    }
    kern<<<grid_for(h.nn, kWarps), kWarps * 32, sm, st>>>(h.nn, h.nb, h.max_deg, m.d.node_off, m.d.inc_ptr,
                                                          m.d.inc, m.d.pos, (const KT *)m.d.K, kstride_of(m),
                                                          rho, simp_params(m.mat), vals);
    return cudaGetLastError();
}

cudaError_t launch_assemble(const soptx_mesh_s &m, const double *rho, double *vals, cudaStream_t st)
{
    if (m.h.nn == 0 || m.h.nnz == 0) return cudaSuccess;
    if (m.path == SOPTX_PATH_LATTICE) return launch_lattice_assemble(m, rho, vals, st);
    const bool f32 = m.prec == SOPTX_ELEM_FP32;
    if (m.h.dim == 2) return f32 ? assemble_t<2, float>(m, rho, vals, st) : assemble_t<2, double>(m, rho, vals, st);
    return f32 ? assemble_t<3, float>(m, rho, vals, st) : assemble_t<3, double>(m, rho, vals, st);
}

int64_t sensitivity_scratch_len(const soptx_mesh_s &m) { return grid_for(m.h.nc, kWarps); }

template <int D, typename KT>
static cudaError_t sens_t(const soptx_mesh_s &m, const double *rho, const double *u, double *out, double *c,
                          const double *gscale, cudaStream_t st)
{
    const auto &h = m.h;
    const int grid = grid_for(h.nc, kWarps);
    k_sensitivity<D, KT><<<grid, kWarps * 32, 0, st>>>(h.nc, h.nb, m.d.cell_node, (const KT *)m.d.K,
                                                       kstride_of(m), rho, u, simp_params(m.mat), gscale, out,
                                                       c ? m.d.scratch : nullptr);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || !c) return err;
    k_reduce_partials<<<1, 256, 0, st>>>(grid, m.d.scratch, c);
    return cudaGetLastError();
}

cudaError_t launch_sensitivity(const soptx_mesh_s &m, const double *rho, const double *u, double *dc, double *c,
                               double /*scale*/, const double *gscale, cudaStream_t st)
{
    if (m.h.nc == 0) {
        if (c) return cudaMemsetAsync(c, 0, sizeof(double), st);
        return cudaSuccess;
    }
    if (m.path == SOPTX_PATH_LATTICE && m.d.sectors) return launch_lattice_sensitivity(m, rho, u, dc, c, gscale, st);
    const bool f32 = m.prec == SOPTX_ELEM_FP32;
    if (m.h.dim == 2)
        return f32 ? sens_t<2, float>(m, rho, u, dc, c, gscale, st) : sens_t<2, double>(m, rho, u, dc, c, gscale, st);
    return f32 ? sens_t<3, float>(m, rho, u, dc, c, gscale, st) : sens_t<3, double>(m, rho, u, dc, c, gscale, st);
}

template <int D, typename KT>
static cudaError_t ku_t(const soptx_mesh_s &m, const double *rho, const double *u, const double *gout, double *out,
                        cudaStream_t st)
{
    const auto &h = m.h;
    k_Ku<D, KT><<<grid_for(h.nn, kWarps), kWarps * 32, 0, st>>>(h.nn, h.nb, m.d.inc_ptr, m.d.inc, m.d.cell_node,
                                                                (const KT *)m.d.K, kstride_of(m), rho, u,
                                                                simp_params(m.mat), gout, out);
    return cudaGetLastError();
}

cudaError_t launch_Ku(const soptx_mesh_s &m, const double *rho, const double *u, const double *gout, double *out,
                      cudaStream_t st)
{
    if (m.h.nn == 0) return cudaSuccess;
    const bool f32 = m.prec == SOPTX_ELEM_FP32;
    if (m.h.dim == 2) return f32 ? ku_t<2, float>(m, rho, u, gout, out, st) : ku_t<2, double>(m, rho, u, gout, out, st);
    return f32 ? ku_t<3, float>(m, rho, u, gout, out, st) : ku_t<3, double>(m, rho, u, gout, out, st);
}

}  // namespace soptx
