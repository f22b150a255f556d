// Setup kernels and dispatch, sm_103a.
//
//  k_element_matrices : K_e^0 from the exact reference integrals and each
//                       cell's inverse Jacobian (Sec. 3.2.2 fast assembly).
//  k_reduce_partials  : c = sum of the block partials in a fixed order.
//  k_Ku               : (K(rho) u) without forming K, for the u-gradient.
// The hot kernels live in lattice.cu (box lattices) and gather.cu (any mesh).
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "internal.h"
#include "kernels_common.cuh"

namespace soptx {
namespace {

constexpr int kWarps = 8;   // warps per CTA for the warp-per-item kernels

__device__ __forceinline__ void store_entry(float2 *K, size_t i, double v)
{
    const float h = __double2float_rn(v);
    K[i] = make_float2(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ void store_entry(float *K, size_t i, float v) { K[i] = v; }

// K_e^0 of cells [0, n_elems): computed in CT (double for FP64 element
// matrices, float for FP32 ones) and stored as OT (float pairs / floats).
template <typename CT, typename OT>
__global__ void k_element_matrices(int dim, int nb, int64_t n_elems, const double *__restrict__ geo,
                                   const double *__restrict__ M, double lam, double mu, OT *__restrict__ K)
{
    const int ldof = dim * nb, ng = dim * dim + 1;
    for (int64_t e = blockIdx.x; e < n_elems; e += gridDim.x) {
        CT G[9], det;
        for (int q = 0; q < dim * dim; q++) G[q] = (CT)geo[e * ng + q];
        det = (CT)geo[e * ng + dim * dim];
        OT *Ke = K + (size_t)e * ldof * ldof;
        for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
            const int a = t / nb, b = t % nb;
            CT Mab[9];
            for (int kl = 0; kl < dim * dim; kl++) Mab[kl] = (CT)M[((size_t)kl * nb + a) * nb + b];
            // P[i][j] = |det J| sum_kl G[k][i] G[l][j] M^{kl}_{ab}   (G[k][i] = (J^-1)_{k i})
            CT P[9];
            for (int i = 0; i < dim; i++)
                for (int j = 0; j < dim; j++) {
                    CT s = 0;
                    for (int k = 0; k < dim; k++) {
                        CT w = 0;
                        for (int l = 0; l < dim; l++) w += Mab[k * dim + l] * G[l * dim + j];
                        s += G[k * dim + i] * w;
                    }
                    P[i * dim + j] = det * s;
                }
            CT tr = 0;
            for (int m = 0; m < dim; m++) tr += P[m * dim + m];
            for (int i = 0; i < dim; i++)
                for (int j = 0; j < dim; j++) {
                    CT v = (CT)lam * P[i * dim + j] + (CT)mu * P[j * dim + i];
                    if (i == j) v += (CT)mu * tr;
                    store_entry(Ke, (size_t)(dim * a + i) * ldof + dim * b + j, v);
                }
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
        // each lane sums E_e K_e[(a,i), c] u_c over its columns c of every incident
        // cell (ascending), then one fixed-order warp sum per row
        double acc[D];
        for (int i = 0; i < D; i++) acc[i] = 0.0;
        for (int32_t q = inc_ptr[n]; q < inc_ptr[n + 1]; q++) {
            const int32_t ea = inc[q];
            const int64_t e = ea / nb;
            const int a = ea - (int)e * nb;
            const KT *Ke = K + e * kstride;
            const double E = simp_E(sp, rho[e]);
            for (int c = lane; c < ldof; c += 32) {
                const int b = c / D, j = c % D;
                const double Eu = E * u[(int64_t)D * cell_node[e * nb + b] + j];
                for (int i = 0; i < D; i++) acc[i] = fma(KLoad<KT>::get64(Ke + (D * a + i) * ldof + c), Eu, acc[i]);
            }
        }
        for (int i = 0; i < D; i++) acc[i] = warp_sum(acc[i]);
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

// K_e^0 of general (non-affine) bilinear / trilinear cells by the reference
// Gauss rule: per point q, J = sum_v x_v (grad N_v)^T, G = J^-1 and
// g_a = G^T grad phi_a; P^{ab}_ij = sum_q w_q |det J_q| (g_a)_i (g_b)_j; then
// the same isotropic combination as the affine kernel.  One block per cell;
// G, w |det J| and the physical gradients of every point are staged in shared
// memory.  Computed in CT, stored as OT.
template <typename CT, typename OT>
__global__ void k_element_matrices_quad(int dim, int nb, int nvc, int nq, int64_t n_elems,
                                        const double *__restrict__ xcell, const double *__restrict__ qw,
                                        const double *__restrict__ dphi, const double *__restrict__ dgeo,
                                        double lam, double mu, OT *__restrict__ K)
{
    extern __shared__ double qsm[];
    double *Gs = qsm;                      // [nq][dim][dim], G[m][i] = (J^-1)_{m i}
    double *wd = Gs + nq * dim * dim;      // [nq]
    double *gx = wd + nq;                  // [nq][nb][dim]
    const int ldof = dim * nb;
    for (int64_t e = blockIdx.x; e < n_elems; e += gridDim.x) {
        const double *xv = xcell + e * nvc * dim;
        for (int q = threadIdx.x; q < nq; q += blockDim.x) {
            double J[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int v = 0; v < nvc; v++)
                for (int i = 0; i < dim; i++)
                    for (int m = 0; m < dim; m++) J[i * dim + m] += xv[v * dim + i] * dgeo[(q * nvc + v) * dim + m];
            double *G = Gs + q * dim * dim;
            double det;
            if (dim == 2) {
                det = J[0] * J[3] - J[1] * J[2];
                G[0] = J[3] / det;
                G[1] = -J[1] / det;
                G[2] = -J[2] / det;
                G[3] = J[0] / det;
            } else {
                const double a00 = J[4] * J[8] - J[5] * J[7], a01 = J[2] * J[7] - J[1] * J[8],
                             a02 = J[1] * J[5] - J[2] * J[4];
                det = J[0] * a00 + J[3] * a01 + J[6] * a02;
                G[0] = a00 / det;
                G[1] = a01 / det;
                G[2] = a02 / det;
                G[3] = (J[5] * J[6] - J[3] * J[8]) / det;
                G[4] = (J[0] * J[8] - J[2] * J[6]) / det;
                G[5] = (J[2] * J[3] - J[0] * J[5]) / det;
                G[6] = (J[3] * J[7] - J[4] * J[6]) / det;
                G[7] = (J[1] * J[6] - J[0] * J[7]) / det;
                G[8] = (J[0] * J[4] - J[1] * J[3]) / det;
            }
            wd[q] = qw[q] * fabs(det);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nq * nb; t += blockDim.x) {
            const int q = t / nb, a = t - q * nb;
            const double *G = Gs + q * dim * dim;
            for (int i = 0; i < dim; i++) {
                double s = 0.0;
                for (int m = 0; m < dim; m++) s += G[m * dim + i] * dphi[(q * nb + a) * dim + m];
                gx[(q * nb + a) * dim + i] = s;
            }
        }
        __syncthreads();
        OT *Ke = K + (size_t)e * ldof * ldof;
        for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
            const int a = t / nb, b = t - a * nb;
            CT P[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            for (int q = 0; q < nq; q++) {
                const double *ga = gx + (q * nb + a) * dim, *gb = gx + (q * nb + b) * dim;
                const CT w = (CT)wd[q];
                for (int i = 0; i < dim; i++)
                    for (int j = 0; j < dim; j++) P[i * dim + j] += w * (CT)ga[i] * (CT)gb[j];
            }
            CT tr = 0;
            for (int m = 0; m < dim; m++) tr += P[m * dim + m];
            for (int i = 0; i < dim; i++)
                for (int j = 0; j < dim; j++) {
                    CT v = (CT)lam * P[i * dim + j] + (CT)mu * P[j * dim + i];
                    if (i == j) v += (CT)mu * tr;
                    store_entry(Ke, (size_t)(dim * a + i) * ldof + dim * b + j, v);
                }
        }
        __syncthreads();
    }
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
    auto split = [](double x, float &h, float &l) {
        h = (float)x;
        l = (float)(x - (double)h);
    };
    split(m.dE, sp.dEh, sp.dEl);
    split(m.Emin, sp.Eminh, sp.Eminl);
    auto normal = [](double x) { return x == 0.0 || (std::fabs(x) >= 0x1p-100 && std::fabs(x) <= 0x1p100); };
    sp.pair_ok = (m.p_int >= 1 && m.p_int <= 4 && normal(m.dE) && normal(m.Emin)) ? 1 : 0;
    return sp;
}

cudaError_t launch_element_matrices(const soptx_mesh_s &m, int64_t n_elems, cudaStream_t st)
{
    const auto &h = m.h;
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(n_elems, 1), 152 * 64);
    const int threads = 128;
    if (n_elems == 0) return cudaSuccess;
    if (h.nonaffine) {
        const size_t smem = (size_t)m.d.nq * (h.dim * h.dim + 1 + h.nb * h.dim) * sizeof(double);
        auto k32 = k_element_matrices_quad<float, float>;
        auto k64 = k_element_matrices_quad<double, float2>;
        cudaError_t err = cudaFuncSetAttribute(m.prec == SOPTX_ELEM_FP32 ? (const void *)k32 : (const void *)k64,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        if (m.prec == SOPTX_ELEM_FP32)
            k32<<<grid, threads, smem, st>>>(h.dim, h.nb, 1 << h.dim, m.d.nq, n_elems, m.d.xcell, m.d.qw, m.d.qdphi,
                                             m.d.qdgeo, m.mat.lam, m.mat.mu, (float *)m.d.K);
        else
            k64<<<grid, threads, smem, st>>>(h.dim, h.nb, 1 << h.dim, m.d.nq, n_elems, m.d.xcell, m.d.qw, m.d.qdphi,
                                             m.d.qdgeo, m.mat.lam, m.mat.mu, (float2 *)m.d.K);
        return cudaGetLastError();
    }
    if (m.prec == SOPTX_ELEM_FP32)
        k_element_matrices<float, float><<<grid, threads, 0, st>>>(h.dim, h.nb, n_elems, m.d.geo, m.d.M, m.mat.lam,
                                                                   m.mat.mu, (float *)m.d.K);
    else
        k_element_matrices<double, float2><<<grid, threads, 0, st>>>(h.dim, h.nb, n_elems, m.d.geo, m.d.M, m.mat.lam,
                                                                     m.mat.mu, (float2 *)m.d.K);
    return cudaGetLastError();
}

static int64_t kstride_of(const soptx_mesh_s &m)
{
    return m.path == SOPTX_PATH_CACHED ? (int64_t)m.h.ldof * m.h.ldof : 0;
}

cudaError_t launch_assemble(const soptx_mesh_s &m, const double *rho, double *vals, cudaStream_t st)
{
    if (m.h.nn == 0 || m.h.nnz == 0) return cudaSuccess;
    if (m.path == SOPTX_PATH_LATTICE) return launch_lattice_assemble(m, rho, vals, st);
    if (m.d.contract || m.d.pcached || m.d.puniform) return launch_contract_assemble(m, rho, vals, st);
    return launch_gather(m, rho, nullptr, vals, nullptr, nullptr, nullptr, st);
}

cudaError_t launch_sensitivity(const soptx_mesh_s &m, const double *rho, const double *u, double *dc, double *c,
                               double /*scale*/, const double *gscale, cudaStream_t st)
{
    if (m.h.nc == 0) {
        if (c) return cudaMemsetAsync(c, 0, sizeof(double), st);
        return cudaSuccess;
    }
    if (m.path == SOPTX_PATH_LATTICE && m.d.sectors) return launch_lattice_sensitivity(m, rho, u, dc, c, gscale, st);
    if (m.d.strain) return launch_strain_sensitivity(m, rho, u, dc, c, gscale, st);
    return launch_gather(m, rho, u, nullptr, dc, c, gscale, st);
}

// gscale: dc = g E' s with g = *gscale (the backward), or the compliance sensitivity when NULL
cudaError_t launch_step(const soptx_mesh_s &m, const double *rho, const double *u, double *vals, double *dc,
                        double *c, cudaStream_t st, const double *gscale)
{
    if (m.path == SOPTX_PATH_LATTICE && m.d.sectors && m.h.nc > 0)
        return launch_lattice_step(m, rho, u, vals, dc, c, st, gscale);
    if (m.d.strain && m.d.side && m.h.nc > 0 && m.h.nnz > 0 &&
        (((m.d.contract || m.d.pcached) && m.h.dim == 2) || m.d.puniform)) {
        // the 2D pair kernel fills every SM with a persistent grid that takes
        // its work from a counter: the sensitivities go first, on the mesh's second
        // stream (highest priority) with one block per SM, and the contraction's
        // CTAs take the rest of the GPU and, as those blocks finish, their slots
        // (in 3D, with one block of 64 threads per SM beside the node-owner
        // contraction, the sensitivities outlasted it: P2 tets 304.5 -> 345.8 us)
        int dev = 0, sms = 0;
        cudaError_t err = cudaGetDevice(&dev);
        if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (err == cudaSuccess) err = cudaEventRecord(m.d.ev[0], st);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(m.d.side, m.d.ev[0], 0);
        if (err == cudaSuccess)
            err = launch_strain_sensitivity(m, rho, u, dc, c, gscale, m.d.side, sms);
        if (err == cudaSuccess) err = cudaEventRecord(m.d.ev[1], m.d.side);
        if (err == cudaSuccess) err = launch_assemble(m, rho, vals, st);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(st, m.d.ev[1], 0);
        return err;
    }
    if (m.d.strain && m.d.side && m.h.nc > 0 && m.h.nnz > 0) {
        // affine cells: the sensitivities need rho and u but not K.  The assembly
        // runs on the mesh's second stream, created at the highest priority and
        // launched first, so the block scheduler gives free SM slots to its blocks
        // and the sensitivities on `stream` fill the slots it leaves
        cudaError_t err = cudaEventRecord(m.d.ev[0], st);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(m.d.side, m.d.ev[0], 0);
        if (err == cudaSuccess) err = launch_assemble(m, rho, vals, m.d.side);
        if (err == cudaSuccess) err = cudaEventRecord(m.d.ev[1], m.d.side);
        if (err == cudaSuccess) err = launch_strain_sensitivity(m, rho, u, dc, c, gscale, st);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(st, m.d.ev[1], 0);
        return err;
    }
    if (m.path == SOPTX_PATH_LATTICE || m.h.nc == 0 || m.d.strain) {
        cudaError_t err = launch_assemble(m, rho, vals, st);
        if (err != cudaSuccess) return err;
        return launch_sensitivity(m, rho, u, dc, c, -1.0, gscale, st);
    }
    return launch_gather(m, rho, u, m.h.nnz > 0 ? vals : nullptr, dc, c, gscale, st);
}

// Block partials of c: enough for every sensitivity grid, the widest being the
// strain-energy kernel with a warp per cell (4 cells per block, at most 152 x 16 blocks).
int64_t sensitivity_scratch_len(const soptx_mesh_s &m)
{
    const int64_t warp_grid = std::min<int64_t>((m.h.nc + 3) / 4, 152 * 16);
    return std::max<int64_t>(std::max<int64_t>(gather_finalize_grid(m.h.nc), warp_grid), 1);
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
    if (m.h.dim == 2) return f32 ? ku_t<2, float>(m, rho, u, gout, out, st) : ku_t<2, float2>(m, rho, u, gout, out, st);
    return f32 ? ku_t<3, float>(m, rho, u, gout, out, st) : ku_t<3, float2>(m, rho, u, gout, out, st);
}

}  // namespace soptx
