// Allocation-free variant of the box-lattice sensitivity kernel.
//
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory pool or allocator hooks, or in a process whose GPU memory
// is fully reserved up front by someone else, may not call cudaMalloc at all.
// They also cannot create a mesh object (soptx_mesh_create allocates).  For
// them, soptx_lattice_sensitivity_noalloc takes the box lattice by its sizes,
// the caller's input and output buffers, and nothing else: the only scratch
// the kernel needs -- one partial sum of c per thread block -- lives in a
// file-scope __device__ array of fixed size, so every GPU that loads this
// library holds those 64 KiB until the process exits.
//
// In host code the array's name is only a host-side handle: its device address
// is looked up with cudaGetSymbolAddress once per device (on the first call
// made on that device, with that device current) and passed to the kernel.
// The address is kept for the life of the process, so this entry point must
// not be called on a device after a cudaDeviceReset of that device (the reset
// unloads the module and the kept address no longer points at the array).
// Because all calls share the one array, calls that overlap on the device
// race on it; each block overwrites its own slot, so nothing needs clearing.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "df64.cuh"
#include "internal.h"
#include "kernels_common.cuh"

namespace soptx {
namespace {

constexpr int kNaThreads = 128;
constexpr int kNaCellsPerThread = 8;
constexpr int kNaCellsPerBlock = kNaThreads * kNaCellsPerThread;     // 1024
constexpr int kNaMaxBlocks = 8192;                                    // 64 KiB of partials
constexpr int64_t kNaMaxCells = (int64_t)kNaMaxBlocks * kNaCellsPerBlock;   // 8,388,608

static __device__ __align__(256) double g_noalloc_partials[kNaMaxBlocks];

constexpr int kNaMaxDevices = 64;
static double *g_partials_ptr[kNaMaxDevices];
static std::mutex g_partials_mu;

// The cell computation of k_lattice_sens: Walsh transform of each displacement
// component over the 2^d corners, then the 2^d sector quadratic forms.
template <int D>
__global__ void __launch_bounds__(kNaThreads)
k_lattice_sens_noalloc(int nx, int ny, int nz, int64_t nc, const double *__restrict__ rho,
                       const double *__restrict__ u, SimpParams sp, SectorTable<D> B, double *__restrict__ out,
                       double *__restrict__ partial)
{
    constexpr int NCR = 1 << D;
    __shared__ double wsum[kNaThreads / 32];
    double mine = 0.0;
    const int64_t first = (int64_t)blockIdx.x * kNaCellsPerBlock;
    for (int k = 0; k < kNaCellsPerThread; k++) {
        const int64_t e = first + (int64_t)k * kNaThreads + threadIdx.x;
        if (e >= nc) break;
        const uint32_t ue = (uint32_t)e;
        const int ex = (int)(ue % (uint32_t)nx);
        const uint32_t r = ue / (uint32_t)nx;
        const int ey = D == 3 ? (int)(r % (uint32_t)ny) : (int)r;
        const int ez = D == 3 ? (int)(r / (uint32_t)ny) : 0;
        df w[NCR][D];
#pragma unroll
        for (int a = 0; a < NCR; a++) {
            const int64_t node = (int64_t)(ex + (a & 1)) +
                                 (int64_t)(nx + 1) * ((ey + ((a >> 1) & 1)) + (int64_t)(ny + 1) * (ez + (a >> 2)));
#pragma unroll
            for (int i = 0; i < D; i++) w[a][i] = df_split(u[D * node + i]);
        }
#pragma unroll
        for (int m = 0; m < D; m++)
#pragma unroll
            for (int a = 0; a < NCR; a++)
                if (!(a & (1 << m)))
#pragma unroll
                    for (int i = 0; i < D; i++) {
                        const df x = w[a][i], y = w[a | (1 << m)][i];
                        w[a][i] = df_add_lazy(x, y);
                        w[a | (1 << m)][i] = df_add_lazy(x, df_neg(y));
                    }
        float S = 0.f, C = 0.f;
#pragma unroll
        for (int c = 0; c < NCR; c++) {
            df x[D];
#pragma unroll
            for (int i = 0; i < D; i++) x[i] = w[c ^ (1 << i)][i];
#pragma unroll
            for (int i = 0; i < D; i++)
#pragma unroll
                for (int j = i; j < D; j++) {
                    if (sector_zero(c, i, j)) continue;
                    const float2 bb = B.b[(c * D + i) * D + j];
                    const df t = df_mul_raw(df_mul_raw(x[i], x[j]), df{bb.x, bb.y});
                    float err;
                    two_sum(S, t.h, S, err);
                    C = __fadd_rn(C, __fadd_rn(t.l, err));
                }
        }
        df s;
        two_sum(S, C, s.h, s.l);
        const double sd = df_to_double(s.h, s.l);
        const double re = rho[e];
        out[e] = -simp_dE(sp, re) * sd;
        mine += simp_E(sp, re) * sd;
    }
    mine = warp_sum(mine);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = mine;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w2 = 0; w2 < kNaThreads / 32; w2++) t += wsum[w2];
        partial[blockIdx.x] = t;
    }
}

// Unit-modulus element matrix of an axis-aligned box with edge lengths h, from
// the exact 1D integrals of the linear Lagrange pair (1 - t, t) on [0, 1]:
// int l_i l_j = [[1/3, 1/6], [1/6, 1/3]], int l_i' l_j = [[-1/2, -1/2], [1/2, 1/2]],
// int l_i' l_j' = [[1, -1], [-1, 1]]; P^{ab}_{ij} = |det J| M^{ij}_{ab} / (h_i h_j)
// and K[(a,i),(b,j)] = lam P_ij + mu P_ji + mu delta_ij sum_m P_mm.  No heap use.
template <int D>
void box_element_matrix(const double *h, double lam, double mu, double *K)
{
    constexpr int NCR = 1 << D, LD = D * NCR;
    const double I0[2][2] = {{1.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 3}};
    const double I1[2][2] = {{-0.5, -0.5}, {0.5, 0.5}};
    const double I2[2][2] = {{1.0, -1.0}, {-1.0, 1.0}};
    double det = 1.0;
    for (int m = 0; m < D; m++) det *= h[m];
    for (int a = 0; a < NCR; a++)
        for (int b = 0; b < NCR; b++) {
            double P[3][3];
            for (int i = 0; i < D; i++)
                for (int j = 0; j < D; j++) {
                    double v = 1.0;
                    for (int m = 0; m < D; m++) {
                        const int ia = (a >> m) & 1, ib = (b >> m) & 1;
                        if (m == i && m == j) v *= I2[ia][ib];
                        else if (m == i) v *= I1[ia][ib];
                        else if (m == j) v *= I1[ib][ia];
                        else v *= I0[ia][ib];
                    }
                    P[i][j] = det * v / (h[i] * h[j]);
                }
            double tr = 0.0;
            for (int m = 0; m < D; m++) tr += P[m][m];
            for (int i = 0; i < D; i++)
                for (int j = 0; j < D; j++)
                    K[(D * a + i) * LD + D * b + j] = lam * P[i][j] + mu * P[j][i] + (i == j ? mu * tr : 0.0);
        }
}

// Sector blocks B_c[i][j] = f_{c^e_i}^T K_ij f_{c^e_j} / 4^d (off-diagonal
// doubled); the entries that vanish on every box (sector_zero) are stored as
// exact zeros, as for a mesh on the lattice path.
template <int D>
void box_sectors(const double *K, SectorTable<D> &B)
{
    constexpr int NCR = 1 << D, LD = D * NCR;
    auto f = [](int t, int a) { return (__builtin_popcount(t & a) & 1) ? -1.0 : 1.0; };
    for (int c = 0; c < NCR; c++)
        for (int i = 0; i < D; i++)
            for (int j = 0; j < D; j++) {
                const int t = c ^ (1 << i), t2 = c ^ (1 << j);
                double s = 0.0;
                for (int a = 0; a < NCR; a++)
                    for (int b = 0; b < NCR; b++) s += f(t, a) * K[(D * a + i) * LD + D * b + j] * f(t2, b);
                const double x = sector_zero(c, i, j) ? 0.0 : (i == j ? 1.0 : 2.0) * s / ((double)NCR * NCR);
                const float hh = (float)x;
                B.b[(c * D + i) * D + j] = make_float2(hh, (float)(x - (double)hh));
            }
}

soptx_status partials_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) SOPTX_FAIL(SOPTX_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kNaMaxDevices) SOPTX_FAIL(SOPTX_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_partials_mu);
    if (!g_partials_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p)
            SOPTX_FAIL(SOPTX_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_partials_ptr[dev] = (double *)p;
    }
    *out = g_partials_ptr[dev];
    return SOPTX_OK;
}

template <int D>
soptx_status run_noalloc(const int32_t *n, const double *h, const soptx_material *mat, const double *rho,
                         const double *u, double *dc, double *c, cudaStream_t st)
{
    const int64_t nc = (int64_t)n[0] * n[1] * (D == 3 ? n[2] : 1);
    if (nc > kNaMaxCells)
        SOPTX_FAIL(SOPTX_EINVAL, "n_cells = " + std::to_string(nc) + " exceeds the allocation-free limit of " +
                                     std::to_string(kNaMaxCells) + " cells");
    double *partials = nullptr;
    soptx_status s = partials_address(&partials);
    if (s != SOPTX_OK) return s;
    const double nu = mat->nu;
    const double mu = 1.0 / (2.0 * (1.0 + nu));
    const double lam = (D == 2 && !mat->plane_strain) ? nu / (1.0 - nu * nu) : nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    double K[(D << D) * (D << D)];
    box_element_matrix<D>(h, lam, mu, K);
    SectorTable<D> B;
    box_sectors<D>(K, B);
    Material m{};
    m.E0 = mat->E0;
    m.Emin = mat->Emin;
    m.nu = mat->nu;
    m.p = mat->p;
    m.dE = mat->E0 - mat->Emin;
    m.lam = lam;
    m.mu = mu;
    m.p_int = (mat->p == std::floor(mat->p) && mat->p <= 16.0) ? (int)mat->p : 0;
    const SimpParams sp = simp_params(m);
    const int grid = (int)((nc + kNaCellsPerBlock - 1) / kNaCellsPerBlock);
    k_lattice_sens_noalloc<D><<<grid, kNaThreads, 0, st>>>(n[0], n[1], D == 3 ? n[2] : 1, nc, rho, u, sp, B, dc,
                                                           partials);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && c) {
        k_reduce_partials<<<1, 256, 0, st>>>(grid, partials, c);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) SOPTX_FAIL(SOPTX_ECUDA, std::string("soptx_lattice_sensitivity_noalloc: ") + cudaGetErrorString(e));
    return SOPTX_OK;
}

}  // namespace
}  // namespace soptx

using namespace soptx;

extern "C" soptx_status soptx_lattice_sensitivity_noalloc(int dim, const int32_t *cells_per_axis,
                                                          const double *cell_size, const soptx_material *mat,
                                                          const double *d_rho, const double *d_u, double *d_dc,
                                                          double *d_c, void *stream)
{
    if (dim != 2 && dim != 3) SOPTX_FAIL(SOPTX_EINVAL, "dim must be 2 or 3");
    if (!cells_per_axis || !cell_size || !mat) SOPTX_FAIL(SOPTX_EINVAL, "cells_per_axis / cell_size / mat is NULL");
    for (int m = 0; m < dim; m++) {
        if (cells_per_axis[m] < 1) SOPTX_FAIL(SOPTX_EINVAL, "every axis needs at least one cell");
        if (!(cell_size[m] > 0.0) || !std::isfinite(cell_size[m])) SOPTX_FAIL(SOPTX_EINVAL, "cell sizes must be positive");
    }
    if (!std::isfinite(mat->E0) || !std::isfinite(mat->Emin) || !std::isfinite(mat->nu) || !std::isfinite(mat->p) ||
        !(mat->Emin >= 0.0) || !(mat->E0 > mat->Emin) || !(mat->nu > -1.0 && mat->nu < 0.5) || !(mat->p >= 1.0))
        SOPTX_FAIL(SOPTX_EINVAL, "need finite E0 > Emin >= 0, -1 < nu < 0.5, p >= 1");
    if (!d_rho || !d_u || !d_dc) SOPTX_FAIL(SOPTX_EINVAL, "d_rho / d_u / d_dc is NULL");
    int64_t nodes = 1;
    for (int m = 0; m < dim; m++) nodes *= (int64_t)cells_per_axis[m] + 1;
    if (dim * nodes >= ((int64_t)1 << 31)) SOPTX_FAIL(SOPTX_EINVAL, "ndof must stay below 2^31");
    cudaStream_t st = (cudaStream_t)stream;
    return dim == 3 ? run_noalloc<3>(cells_per_axis, cell_size, mat, d_rho, d_u, d_dc, d_c, st)
                    : run_noalloc<2>(cells_per_axis, cell_size, mat, d_rho, d_u, d_dc, d_c, st);
}
