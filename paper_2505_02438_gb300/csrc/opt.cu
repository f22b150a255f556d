// The steps of a SIMP iteration after the sensitivities (include/soptx_opt.h):
// filters, Heaviside projection and the optimality-criteria update.
//
//  filter weights : built on the host -- cell centroids bucketed in a uniform
//                   grid of size rmin, each cell's neighbours within rmin in
//                   ascending cell order -- and kept on the device as CSR.
//  k_filter_*     : one thread per cell, its row summed in column order.
//  k_oc_*         : q_e = rho_e (max(0, -dc_e) / dv_e)^eta once, then each
//                   bisection step evaluates rho_e B_e^eta = q_e lambda^-eta
//                   for every cell and sums the volume (fixed-order block
//                   partials, the last block adds them), one thread moves the
//                   bracket in device memory -- a fixed number of launches,
//                   each a no-op once the bracket meets the tolerance, so no
//                   host round trip -- and a last kernel applies the update.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "kernels_common.cuh"
#include "../../include/soptx_opt.h"

struct soptx_filter_s {
    int dim = 0;
    int64_t nc = 0, nnz = 0;
    int64_t *ptr = nullptr;     // [nc+1]
    int32_t *col = nullptr;     // [nnz]
    double *h = nullptr;        // [nnz] H_ij
    double *vol = nullptr;      // [nc]  v_j
    double *hs = nullptr;       // [nc]  sum_j H_ij
    double *hv = nullptr;       // [nc]  sum_j H_ij v_j
    double *w = nullptr;        // [nc]  scratch of the chain rule
};

namespace soptx {
namespace {

constexpr int kOptThreads = 256;
constexpr int kOcMaxSteps = 100;

int opt_grid(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + kOptThreads - 1) / kOptThreads, 152 * 8)); }

__global__ void k_filter_sens(int64_t nc, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                              const double *__restrict__ h, const double *__restrict__ hs,
                              const double *__restrict__ rho, const double *__restrict__ dc, double *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t k = ptr[i]; k < ptr[i + 1]; k++) {
            const int32_t j = col[k];
            s = fma(h[k], rho[j] * dc[j], s);
        }
        out[i] = s / (fmax(1e-3, rho[i]) * hs[i]);
    }
}

// transpose = 0: out_i = sum_j H_ij v_j x_j / hv_i   (the density filter)
// transpose = 1: out_j = v_j sum_i H_ji x_i          (its chain rule, x_i = g_i / hv_i; H symmetric)
__global__ void k_filter_hv(int64_t nc, const int64_t *__restrict__ ptr, const int32_t *__restrict__ col,
                            const double *__restrict__ h, const double *__restrict__ vol,
                            const double *__restrict__ hv, const double *__restrict__ x, double *__restrict__ out,
                            int transpose)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nc; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t k = ptr[i]; k < ptr[i + 1]; k++) {
            const int32_t j = col[k];
            s = transpose ? fma(h[k], x[j], s) : fma(h[k] * vol[j], x[j], s);
        }
        out[i] = transpose ? vol[i] * s : s / hv[i];
    }
}

__global__ void k_div(int64_t n, const double *__restrict__ g, const double *__restrict__ d, double *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = g[i] / d[i];
}

__global__ void k_heaviside(int64_t n, double beta, const double *__restrict__ x, double *__restrict__ out,
                            double *__restrict__ dout)
{
    const double eb = exp(-beta);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double t = exp(-beta * x[i]);
        out[i] = 1.0 - t + x[i] * eb;
        if (dout) dout[i] = beta * t + eb;
    }
}

__device__ __forceinline__ double neg_pow(double l, double eta)
{
    return eta == 0.5 ? 1.0 / sqrt(l) : (eta == 1.0 ? 1.0 / l : pow(l, -eta));
}

// q_e = rho_e (max(0, -dc_e) / dv_e)^eta; the total volume.
__global__ void __launch_bounds__(kOptThreads)
k_oc_prep(int64_t n, double eta, const double *__restrict__ rho, const double *__restrict__ dc,
          const double *__restrict__ dv, const double *__restrict__ vol, double *__restrict__ q,
          double *__restrict__ partial, unsigned *__restrict__ counter, double *__restrict__ vtot)
{
    double mine = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double b = fmax(0.0, -dc[e]) / dv[e];
        q[e] = rho[e] * (eta == 0.5 ? sqrt(b) : (eta == 1.0 ? b : pow(b, eta)));
        mine += vol[e];
    }
    grid_sum_last_block(mine, partial, counter, vtot);
}

__device__ __forceinline__ double oc_candidate(double q, double s, double r, double move)
{
    return fmin(fmin(1.0, r + move), fmax(fmax(0.0, r - move), q * s));
}

// One bisection step's volume.  st: [0] lo, [1] hi, [2] lambda of the last
// step, [3] total volume, [4] the step's volume (k_oc_move then moves the bracket).
__global__ void __launch_bounds__(kOptThreads)
k_oc_step(int64_t n, double eta, double move, double tol, const double *__restrict__ rho,
          const double *__restrict__ q, const double *__restrict__ vol, double *__restrict__ st,
          double *__restrict__ partial, unsigned *__restrict__ counter)
{
    const double lo = st[0], hi = st[1];
    if (!((hi - lo) / (hi + lo) > tol)) return;      // the whole grid agrees: bracket already met
    const double lmid = 0.5 * (hi + lo);
    __shared__ double s_sh;
    if (threadIdx.x == 0) s_sh = neg_pow(lmid, eta);
    __syncthreads();
    const double s = s_sh;
    double mine = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        mine = fma(vol[e], oc_candidate(q[e], s, rho[e], move), mine);
    grid_sum_last_block(mine, partial, counter, st + 4);
}

// the bracket update after a step (one thread; a no-op once the bracket is met)
__global__ void k_oc_move(double volfrac, double tol, double *__restrict__ st)
{
    const double lo = st[0], hi = st[1];
    if (!((hi - lo) / (hi + lo) > tol)) return;
    const double lmid = 0.5 * (hi + lo);
    st[2] = lmid;
    if (st[4] > volfrac * st[3]) st[0] = lmid;
    else st[1] = lmid;
}

// rho_new with the last lambda; the volume and max |rho_new - rho|
__global__ void __launch_bounds__(kOptThreads)
k_oc_apply(int64_t n, double eta, double move, const double *__restrict__ rho, const double *__restrict__ q,
           const double *__restrict__ vol, const double *__restrict__ st, double *__restrict__ out,
           double *__restrict__ partial, unsigned *__restrict__ counter, double *__restrict__ sums,
           unsigned long long *__restrict__ dmax)
{
    const double s = neg_pow(st[2], eta);
    double mine = 0.0, chg = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const double x = oc_candidate(q[e], s, rho[e], move);
        out[e] = x;
        mine = fma(vol[e], x, mine);
        chg = fmax(chg, fabs(x - rho[e]));
    }
    // the maximum of non-negative doubles: their bit patterns order like the values
    for (int o = 16; o > 0; o >>= 1) chg = fmax(chg, __shfl_xor_sync(0xffffffffu, chg, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dmax, (unsigned long long)__double_as_longlong(chg));
    grid_sum_last_block(mine, partial, counter, sums);
}

__global__ void k_oc_stats(const double *__restrict__ st, const double *__restrict__ sums,
                           const unsigned long long *__restrict__ dmax, double *__restrict__ stats)
{
    stats[0] = __longlong_as_double((long long)*dmax);
    stats[1] = st[2];
    stats[2] = sums[0] / st[3];
}

soptx_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return SOPTX_OK;
    cudaGetLastError();
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SOPTX_ENOMEM : SOPTX_ECUDA;
}

void free_filter(soptx_filter_s *f)
{
    void *p[] = {f->ptr, f->col, f->h, f->vol, f->hs, f->hv, f->w};
    for (void *x : p)
        if (x) cudaFree(x);
    delete f;
}

}  // namespace
}  // namespace soptx

using namespace soptx;

extern "C" {

soptx_status soptx_filter_create(int dim, int64_t nc, const double *cen, const double *vol, double rmin, void *stream,
                                 soptx_filter *out)
{
    if (!out) SOPTX_FAIL(SOPTX_EINVAL, "out is NULL");
    *out = nullptr;
    if (dim < 2 || dim > 3 || nc < 0 || (nc > 0 && (!cen || !vol)) || !(rmin > 0.0) || !std::isfinite(rmin))
        SOPTX_FAIL(SOPTX_EINVAL, "need dim 2 or 3, n_cells >= 0, centroids / volumes, finite rmin > 0");
    if (nc >= ((int64_t)1 << 31)) SOPTX_FAIL(SOPTX_EINVAL, "n_cells must stay below 2^31");
    for (int64_t e = 0; e < nc; e++) {
        if (!std::isfinite(vol[e])) SOPTX_FAIL(SOPTX_EINVAL, "non-finite volume");
        for (int m = 0; m < dim; m++)
            if (!std::isfinite(cen[e * dim + m])) SOPTX_FAIL(SOPTX_EINVAL, "non-finite centroid");
    }
    std::vector<int64_t> ptr((size_t)nc + 1, 0);
    std::vector<int32_t> col;
    std::vector<double> h, hs((size_t)nc, 0.0), hv((size_t)nc, 0.0);
    try {
        // buckets of size rmin: the neighbours of a cell lie in its own or the adjacent buckets
        double lo[3] = {0, 0, 0};
        for (int m = 0; m < dim; m++) lo[m] = nc ? cen[m] : 0.0;
        for (int64_t e = 0; e < nc; e++)
            for (int m = 0; m < dim; m++) lo[m] = std::min(lo[m], cen[e * dim + m]);
        auto key = [](int64_t b0, int64_t b1, int64_t b2) { return (b0 * 1000003LL + b1) * 1000003LL + b2; };
        auto bucket = [&](int64_t e, int m) { return (int64_t)std::floor((cen[e * dim + m] - lo[m]) / rmin); };
        std::unordered_map<int64_t, std::vector<int32_t>> grid;
        for (int64_t e = 0; e < nc; e++)
            grid[key(bucket(e, 0), bucket(e, 1), dim == 3 ? bucket(e, 2) : 0)].push_back((int32_t)e);
        std::vector<std::pair<int32_t, double>> row;
        for (int64_t i = 0; i < nc; i++) {
            row.clear();
            const int64_t b[3] = {bucket(i, 0), bucket(i, 1), dim == 3 ? bucket(i, 2) : 0};
            for (int64_t d0 = -1; d0 <= 1; d0++)
                for (int64_t d1 = -1; d1 <= 1; d1++)
                    for (int64_t d2 = (dim == 3 ? -1 : 0); d2 <= (dim == 3 ? 1 : 0); d2++) {
                        auto it = grid.find(key(b[0] + d0, b[1] + d1, b[2] + d2));
                        if (it == grid.end()) continue;
                        for (int32_t j : it->second) {
                            double r2 = 0.0;
                            for (int m = 0; m < dim; m++) {
                                const double t = cen[i * dim + m] - cen[(int64_t)j * dim + m];
                                r2 += t * t;
                            }
                            const double w = rmin - std::sqrt(r2);
                            if (w > 0.0) row.emplace_back(j, w);
                        }
                    }
            std::sort(row.begin(), row.end());
            for (auto &x : row) {
                col.push_back(x.first);
                h.push_back(x.second);
                hs[i] += x.second;
                hv[i] += x.second * vol[x.first];
            }
            ptr[i + 1] = (int64_t)col.size();
        }
    } catch (const std::bad_alloc &) {
        SOPTX_FAIL(SOPTX_ENOMEM, "host allocation failed building the filter");
    }
    soptx_filter_s *f = new (std::nothrow) soptx_filter_s();
    if (!f) SOPTX_FAIL(SOPTX_ENOMEM, "host allocation failed");
    f->dim = dim;
    f->nc = nc;
    f->nnz = (int64_t)col.size();
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    auto up = [&](auto **dst, const auto *src, size_t count) {
        using T = std::remove_reference_t<decltype(**dst)>;
        if (e != cudaSuccess) return;
        e = dev_alloc((void **)dst, std::max<size_t>(count, 1) * sizeof(T));
        if (e == cudaSuccess && count) e = cudaMemcpyAsync(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice, st);
    };
    up(&f->ptr, ptr.data(), ptr.size());
    up(&f->col, col.data(), col.size());
    up(&f->h, h.data(), h.size());
    up(&f->vol, vol, (size_t)nc);
    up(&f->hs, hs.data(), hs.size());
    up(&f->hv, hv.data(), hv.size());
    if (e == cudaSuccess) e = dev_alloc((void **)&f->w, std::max<size_t>((size_t)nc, 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_filter(f);
        return cuda_fail(e, "soptx_filter_create");
    }
    *out = f;
    return SOPTX_OK;
}

soptx_status soptx_filter_info(soptx_filter f, int64_t *n_cells, int64_t *nnz)
{
    if (!f) SOPTX_FAIL(SOPTX_EINVAL, "filter is NULL");
    if (n_cells) *n_cells = f->nc;
    if (nnz) *nnz = f->nnz;
    return SOPTX_OK;
}

soptx_status soptx_filter_sensitivity(soptx_filter f, const double *rho, const double *dc, double *out, void *stream)
{
    if (!f) SOPTX_FAIL(SOPTX_EINVAL, "filter is NULL");
    if (f->nc == 0) return SOPTX_OK;
    if (!rho || !dc || !out) SOPTX_FAIL(SOPTX_EINVAL, "d_rho / d_dc / d_out is NULL");
    k_filter_sens<<<opt_grid(f->nc), kOptThreads, 0, (cudaStream_t)stream>>>(f->nc, f->ptr, f->col, f->h, f->hs, rho,
                                                                             dc, out);
    return cuda_fail(cudaGetLastError(), "soptx_filter_sensitivity");
}

soptx_status soptx_filter_density(soptx_filter f, const double *x, double *out, void *stream)
{
    if (!f) SOPTX_FAIL(SOPTX_EINVAL, "filter is NULL");
    if (f->nc == 0) return SOPTX_OK;
    if (!x || !out) SOPTX_FAIL(SOPTX_EINVAL, "d_x / d_out is NULL");
    k_filter_hv<<<opt_grid(f->nc), kOptThreads, 0, (cudaStream_t)stream>>>(f->nc, f->ptr, f->col, f->h, f->vol, f->hv,
                                                                           x, out, 0);
    return cuda_fail(cudaGetLastError(), "soptx_filter_density");
}

soptx_status soptx_filter_density_grad(soptx_filter f, const double *g, double *out, void *stream)
{
    if (!f) SOPTX_FAIL(SOPTX_EINVAL, "filter is NULL");
    if (f->nc == 0) return SOPTX_OK;
    if (!g || !out) SOPTX_FAIL(SOPTX_EINVAL, "d_g / d_out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    k_div<<<opt_grid(f->nc), kOptThreads, 0, st>>>(f->nc, g, f->hv, f->w);
    k_filter_hv<<<opt_grid(f->nc), kOptThreads, 0, st>>>(f->nc, f->ptr, f->col, f->h, f->vol, f->hv, f->w, out, 1);
    return cuda_fail(cudaGetLastError(), "soptx_filter_density_grad");
}

soptx_status soptx_filter_destroy(soptx_filter f)
{
    if (!f) return SOPTX_OK;
    cudaDeviceSynchronize();
    free_filter(f);
    return SOPTX_OK;
}

soptx_status soptx_heaviside(int64_t n, double beta, const double *x, double *out, double *dout, void *stream)
{
    if (n < 0 || !std::isfinite(beta)) SOPTX_FAIL(SOPTX_EINVAL, "need n >= 0 and a finite beta");
    if (n == 0) return SOPTX_OK;
    if (!x || !out) SOPTX_FAIL(SOPTX_EINVAL, "d_x / d_out is NULL");
    k_heaviside<<<opt_grid(n), kOptThreads, 0, (cudaStream_t)stream>>>(n, beta, x, out, dout);
    return cuda_fail(cudaGetLastError(), "soptx_heaviside");
}

soptx_status soptx_oc_update(int64_t n, const double *rho, const double *dc, const double *dv, const double *vol,
                             const soptx_oc_opts *o, double *out, double *stats, void *stream)
{
    if (!o || n < 0) SOPTX_FAIL(SOPTX_EINVAL, "opts is NULL or n < 0");
    if (!(o->volfrac > 0.0) || !(o->move > 0.0) || !(o->eta > 0.0 && o->eta <= 1.0) || !(o->l_lo >= 0.0) ||
        !(o->l_hi > o->l_lo) || !(o->tol > 0.0))
        SOPTX_FAIL(SOPTX_EINVAL, "need volfrac > 0, move > 0, 0 < eta <= 1, 0 <= l_lo < l_hi, tol > 0");
    if (n == 0) return SOPTX_OK;
    if (!rho || !dc || !dv || !vol || !out) SOPTX_FAIL(SOPTX_EINVAL, "d_rho / d_dc / d_dv / d_vol / d_out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = opt_grid(n);
    // workspace: q [n], bracket state [8], sums [4], partials [grid], then the counter and the maximum
    const size_t bytes = ((size_t)n + 8 + 4 + (size_t)grid) * sizeof(double) + 64;
    void *ws = nullptr;
    cudaError_t e = dev_alloc(&ws, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "OC workspace");
    double *q = (double *)ws, *stt = q + n, *sums = stt + 8, *partial = sums + 4;
    unsigned *counter = (unsigned *)(partial + grid);
    unsigned long long *dmax = (unsigned long long *)(partial + grid + 1);
    const double init[8] = {o->l_lo, o->l_hi, 0.5 * (o->l_lo + o->l_hi), 0, 0, 0, 0, 0};
    e = cudaMemsetAsync(ws, 0, bytes, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stt, init, sizeof(init), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        k_oc_prep<<<grid, kOptThreads, 0, st>>>(n, o->eta, rho, dc, dv, vol, q, partial, counter, stt + 3);
        e = cudaGetLastError();
    }
    for (int k = 0; k < kOcMaxSteps && e == cudaSuccess; k++) {
        k_oc_step<<<grid, kOptThreads, 0, st>>>(n, o->eta, o->move, o->tol, rho, q, vol, stt, partial, counter);
        k_oc_move<<<1, 1, 0, st>>>(o->volfrac, o->tol, stt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_oc_apply<<<grid, kOptThreads, 0, st>>>(n, o->eta, o->move, rho, q, vol, stt, out, partial, counter, sums,
                                                 dmax);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && stats) {
        k_oc_stats<<<1, 1, 0, st>>>(stt, sums, dmax, stats);
        e = cudaGetLastError();
    }
    // the workspace is released once the stream has passed it
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(ws);
    return cuda_fail(e, "soptx_oc_update");
}

}  // extern "C"
