// General path (any mesh, per-cell K_e^0 cached on the device, or one shared
// K^0 when every cell has the same Jacobian), FP64-accurate on the FP32 pipes.
//
//  k_prep          : E(rho_e) per cell and, when u is given, u per dof, as
//                    float pairs (FP64 math once per item).
//  k_gather_fused  : one warp owns the d rows of one node; it walks the node's
//                    incident cells in ascending order and for each reads the
//                    node's row block of K_e^0 once, adding E_e K_e^0 into the
//                    rows' CSR values (float-pair accumulators in shared
//                    memory, so every value is summed in ascending cell
//                    order, no atomics) and, when u is given, forming the
//                    cell's partial  sum_i u_(a,i) sum_(b,j) K_e[(a,i),(b,j)] u_(b,j)
//                    for this node a.  The rows leave through coalesced
//                    streaming stores.
//  k_sens_finalize : s_e = sum of the cell's node partials (fixed order),
//                    dc_e = -E'(rho_e) s_e and block partials of E_e s_e.
// Nodes touching a modulus outside [2^-60, 2^60] are redone in plain FP64.
#include <algorithm>
#include <cstdint>

#include "df64.cuh"
#include "internal.h"
#include "kernels_common.cuh"

namespace soptx {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kGW = 8;   // warps per CTA
constexpr int kMaxRounds = (kMaxNb * 9 + 31) / 32;   // 32-entry rounds of a node's row block

__global__ void k_prep(int64_t nc, const double *__restrict__ rho, SimpParams sp, float2 *__restrict__ Edf,
                       int64_t ndof, const double *__restrict__ u, float2 *__restrict__ udf)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc; e += stride) {
        const double E = simp_E(sp, rho[e]);
        const double a = fabs(E);
        float2 out;
        if (E == 0.0) out = make_float2(0.f, 0.f);
        else if (!(a >= 0x1p-60 && a <= 0x1p60)) out = make_float2((float)E, __int_as_float(0x7fc00000));
        else {
            const df v = df_from_double(E);
            out = make_float2(v.h, v.l);
        }
        Edf[e] = out;
    }
    if (u)
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < ndof; r += stride) {
            const df v = df_split(u[r]);
            udf[r] = make_float2(v.h, v.l);
        }
}

// Plain-FP64 rows of one node (a modulus outside the float-pair range).
template <int D, typename KT>
__device__ __noinline__ void gather_node_fp64(int lane, int nb, int ldof, int deg, int32_t q0, int32_t q1,
                                              const int32_t *__restrict__ inc, const uint16_t *__restrict__ pos,
                                              const KT *__restrict__ K, int64_t kstride,
                                              const double *__restrict__ rho, SimpParams sp, double *out)
{
    for (int t = lane; t < D * D * deg; t += 32) out[t] = 0.0;
    __syncwarp();
    for (int32_t q = q0; q < q1; q++) {
        const int32_t ea = inc[q];
        const int64_t e = ea / nb;
        const int a = ea - (int)e * nb;
        const double E = simp_E(sp, rho[e]);
        const KT *Ke = K + e * kstride;
        for (int t = lane; t < nb * D * D; t += 32) {
            const int b = t / (D * D), i = (t / D) % D, j = t % D;
            out[i * (D * deg) + D * pos[(int64_t)q * nb + b] + j] += E * KLoad<KT>::get64(Ke + (D * a + i) * ldof + D * b + j);
        }
        __syncwarp();
    }
}

template <int D, typename KT, bool SENS>
__global__ void __launch_bounds__(kGW * 32)
k_gather_fused(int64_t nn, int nb, int max_deg, const int64_t *__restrict__ node_off,
               const int32_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc,
               const int32_t *__restrict__ inc_e, const uint8_t *__restrict__ inc_a,
               const uint16_t *__restrict__ pos, const int32_t *__restrict__ cell_node,
               const KT *__restrict__ K, int64_t kstride, const float2 *__restrict__ Edf,
               const float2 *__restrict__ udf, const double *__restrict__ rho, SimpParams sp,
               double *__restrict__ vals, double *__restrict__ part)
{
    extern __shared__ float smem_f[];
    __shared__ int tab_koff[kMaxRounds * 32], tab_bij[kMaxRounds * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ldof = D * nb;
    const int per = nb * D * D;
    const int rounds = (per + 31) / 32;
    // entry t of a node's row block: (b, i, j) = (t / d^2, (t / d) % d, t % d)
    for (int t = threadIdx.x; t < rounds * 32; t += blockDim.x) {
        const int tt = t < per ? t : 0;
        const int b = tt / (D * D), i = (tt / D) % D, j = tt % D;
        tab_koff[t] = i * ldof + D * b + j;
        tab_bij[t] = b | (i << 8) | (j << 16);
    }
    __syncthreads();
    float *acc_h = smem_f + (size_t)warp * 2 * D * D * max_deg;
    float *acc_l = acc_h + D * D * max_deg;
    double *acc_d = reinterpret_cast<double *>(acc_h);   // FP64 route reuses the same space
    for (int64_t n = (int64_t)blockIdx.x * kGW + warp; n < nn; n += (int64_t)gridDim.x * kGW) {
        const int64_t off = node_off[n];
        const int deg = (int)(node_off[n + 1] - off);
        const int blk = D * D * deg;
        const int32_t q0 = inc_ptr[n], q1 = inc_ptr[n + 1];
        double *out = vals + (int64_t)D * D * off;
        // any incident modulus outside the float-pair range?
        bool bad = false;
        for (int32_t q = q0 + lane; q < q1; q += 32) bad |= isnan(Edf[inc[q] / nb].y);
        if (__any_sync(kFull, bad)) {
            if (vals) {
                gather_node_fp64<D, KT>(lane, nb, ldof, deg, q0, q1, inc, pos, K, kstride, rho, sp, acc_d);
                __syncwarp();
                for (int t = lane; t < blk; t += 32) __stcs(out + t, acc_d[t]);
                __syncwarp();
            }
            if (SENS) {
                for (int32_t q = q0; q < q1; q++) {
                    const int32_t ea = inc[q];
                    const int64_t e = ea / nb;
                    const int a = ea - (int)e * nb;
                    const KT *Ke = K + e * kstride;
                    double s = 0.0;
                    for (int t = lane; t < nb * D * D; t += 32) {
                        const int b = t / (D * D), i = (t / D) % D, j = t % D;
                        const float2 ua = udf[(int64_t)D * n + i], ub = udf[(int64_t)D * cell_node[e * nb + b] + j];
                        s += ((double)ua.x + ua.y) * KLoad<KT>::get64(Ke + (D * a + i) * ldof + D * b + j) *
                             ((double)ub.x + ub.y);
                    }
                    s = warp_sum(s);
                    if (lane == 0) part[ea] = s;
                }
            }
            continue;
        }
        if (vals) {
            for (int t = lane; t < blk; t += 32) {
                acc_h[t] = 0.f;
                acc_l[t] = 0.f;
            }
        }
        __syncwarp();
        // Flattened (incidence, round) items: round r of incidence q covers the
        // entries t = 32 r + lane of the node's row block of K_e (offsets from
        // the per-block table).  The next item's loads are issued before the
        // current item is accumulated.
        const int n_items = (q1 - q0) * rounds;
        struct Inc {
            const KT *kb;
            const int32_t *cn;
            const uint16_t *ps;
            float2 E;
            int32_t ea;
        };
        auto fetch_inc = [&](int32_t q) {
            Inc c;
            const int32_t e = inc_e[q];
            const int a = inc_a[q];
            c.ea = e * nb + a;
            c.kb = K + (int64_t)e * kstride + (int64_t)(D * a) * ldof;
            c.cn = cell_node + (int64_t)e * nb;
            c.ps = pos + (int64_t)q * nb;
            c.E = Edf[e];
            return c;
        };
        struct Item {
            float2 k, ub, ua;
            int slot;
        };
        auto fetch = [&](const Inc &c, int r) {
            Item it;
            const int t = 32 * r + lane;
            const int koff = tab_koff[t], bij = tab_bij[t];
            const int bb = bij & 0xff, ii = (bij >> 8) & 0xff, jj = bij >> 16;
            const bool live = t < per;
            it.k = live ? KLoad<KT>::raw(c.kb + koff) : make_float2(0.f, 0.f);
            it.slot = (vals && live) ? ii * (D * deg) + D * c.ps[bb] + jj : 0;
            it.ub = (SENS && live) ? udf[(int64_t)D * c.cn[bb] + jj] : make_float2(0.f, 0.f);
            it.ua = (SENS && live) ? udf[(int64_t)D * n + ii] : make_float2(0.f, 0.f);
            return it;
        };
        float S = 0.f, C = 0.f;     // this lane's share of the current cell's node partial
        int32_t q = q0;
        int r = 0;
        Inc ccur = n_items > 0 ? fetch_inc(q0) : Inc{};
        Item cur = n_items > 0 ? fetch(ccur, 0) : Item{};
        Inc cnxt = ccur;
        for (int item = 0; item < n_items; item++) {
            int32_t qn = q;
            int rn = r + 1;
            if (rn == rounds) {
                rn = 0;
                qn++;
                if (qn < q1) cnxt = fetch_inc(qn);
            }
            Item nxt;
            if (item + 1 < n_items) nxt = fetch(cnxt, rn);
            if (32 * r + lane < per) {
                const df kv = df{cur.k.x, cur.k.y};
                if (vals) {
                    const df pr = df_mul_raw(df{ccur.E.x, ccur.E.y}, kv);
                    float s, err;
                    two_sum(acc_h[cur.slot], pr.h, s, err);
                    acc_h[cur.slot] = s;
                    acc_l[cur.slot] = __fadd_rn(acc_l[cur.slot], __fadd_rn(pr.l, err));
                }
                if (SENS) {
                    const df t1 = df_mul_raw(df_mul_raw(kv, df{cur.ub.x, cur.ub.y}), df{cur.ua.x, cur.ua.y});
                    float s, err;
                    two_sum(S, t1.h, s, err);
                    S = s;
                    C = __fadd_rn(C, __fadd_rn(t1.l, err));
                }
            }
            if (rn == 0) {   // last round of this cell
                __syncwarp();
                if (SENS) {
                    // fixed-order butterfly of the lanes' (S, C) pairs
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const float So = __shfl_xor_sync(kFull, S, o), Co = __shfl_xor_sync(kFull, C, o);
                        float s, err;
                        two_sum(S, So, s, err);
                        S = s;
                        C = __fadd_rn(__fadd_rn(C, Co), err);
                    }
                    if (lane == 0) {
                        float h, l;
                        two_sum(S, C, h, l);
                        part[ccur.ea] = df_to_double(h, l);
                    }
                    S = 0.f;
                    C = 0.f;
                }
                ccur = cnxt;
            }
            q = qn;
            r = rn;
            cur = nxt;
        }
        if (vals) {
            for (int t = lane; t < blk; t += 32) {
                float h, l;
                two_sum(acc_h[t], acc_l[t], h, l);
                __stcs(out + t, df_to_double(h, l));
            }
        }
        __syncwarp();
    }
}

// Same computation with the R rounds of a node's row block unrolled: each
// lane's entry offsets live in registers and the next incidence's entries are
// loaded into register arrays while the current one is accumulated.
template <int D, typename KT, bool SENS, int R>
__global__ void __launch_bounds__(kGW * 32)
k_gather_unrolled(int64_t nn, int nb, int max_deg, const int64_t *__restrict__ node_off,
                  const int32_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc,
                  const int32_t *__restrict__ inc_e, const uint8_t *__restrict__ inc_a,
                  const uint16_t *__restrict__ pos, const int32_t *__restrict__ cell_node,
                  const KT *__restrict__ K, int64_t kstride, const float2 *__restrict__ Edf,
                  const float2 *__restrict__ udf, const double *__restrict__ rho, SimpParams sp,
                  double *__restrict__ vals, double *__restrict__ part)
{
    extern __shared__ float smem_f[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ldof = D * nb;
    const int per = nb * D * D;
    int koff[R], bq[R], iq[R], jq[R];
    bool live[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int t = 32 * r + lane;
        live[r] = t < per;
        const int tt = live[r] ? t : 0;
        bq[r] = tt / (D * D);
        iq[r] = (tt / D) % D;
        jq[r] = tt % D;
        koff[r] = iq[r] * ldof + D * bq[r] + jq[r];
    }
    float *acc_h = smem_f + (size_t)warp * 2 * D * D * max_deg;
    float *acc_l = acc_h + D * D * max_deg;
    double *acc_d = reinterpret_cast<double *>(acc_h);
    for (int64_t n = (int64_t)blockIdx.x * kGW + warp; n < nn; n += (int64_t)gridDim.x * kGW) {
        const int64_t off = node_off[n];
        const int deg = (int)(node_off[n + 1] - off);
        const int blk = D * D * deg;
        const int32_t q0 = inc_ptr[n], q1 = inc_ptr[n + 1];
        double *out = vals + (int64_t)D * D * off;
        bool bad = false;
        for (int32_t q = q0 + lane; q < q1; q += 32) bad |= isnan(Edf[inc_e[q]].y);
        if (__any_sync(kFull, bad)) {
            if (vals) {
                gather_node_fp64<D, KT>(lane, nb, ldof, deg, q0, q1, inc, pos, K, kstride, rho, sp, acc_d);
                __syncwarp();
                for (int t = lane; t < blk; t += 32) __stcs(out + t, acc_d[t]);
                __syncwarp();
            }
            if (SENS) {
                for (int32_t q = q0; q < q1; q++) {
                    const int64_t e = inc_e[q];
                    const int a = inc_a[q];
                    const KT *Ke = K + e * kstride;
                    double s = 0.0;
                    for (int t = lane; t < per; t += 32) {
                        const int b = t / (D * D), i = (t / D) % D, j = t % D;
                        const float2 ua = udf[(int64_t)D * n + i], ub = udf[(int64_t)D * cell_node[e * nb + b] + j];
                        s += ((double)ua.x + ua.y) * KLoad<KT>::get64(Ke + (D * a + i) * ldof + D * b + j) *
                             ((double)ub.x + ub.y);
                    }
                    s = warp_sum(s);
                    if (lane == 0) part[e * nb + a] = s;
                }
            }
            continue;
        }
        if (vals)
            for (int t = lane; t < blk; t += 32) {
                acc_h[t] = 0.f;
                acc_l[t] = 0.f;
            }
        float2 ua[R];
        if (SENS)
#pragma unroll
            for (int r = 0; r < R; r++) ua[r] = udf[(int64_t)D * n + iq[r]];
        __syncwarp();
        // prefetched next incidence
        float2 kN[R], ubN[R], EN = make_float2(0.f, 0.f);
        int slotN[R];
        int32_t eaN = 0;
        auto load = [&](int32_t q) {
            const int32_t e = inc_e[q];
            const int a = inc_a[q];
            eaN = e * nb + a;
            EN = Edf[e];
            const KT *kb = K + (int64_t)e * kstride + (int64_t)(D * a) * ldof;
            const int32_t *cn = cell_node + (int64_t)e * nb;
            const uint16_t *ps = pos + (int64_t)q * nb;
#pragma unroll
            for (int r = 0; r < R; r++) {
                kN[r] = live[r] ? KLoad<KT>::raw(kb + koff[r]) : make_float2(0.f, 0.f);
                if (vals) slotN[r] = live[r] ? iq[r] * (D * deg) + D * ps[bq[r]] + jq[r] : 0;
                if (SENS) ubN[r] = live[r] ? udf[(int64_t)D * cn[bq[r]] + jq[r]] : make_float2(0.f, 0.f);
            }
        };
        if (q0 < q1) load(q0);
        for (int32_t q = q0; q < q1; q++) {
            float2 kc[R], ubc[R];
            int slotc[R];
#pragma unroll
            for (int r = 0; r < R; r++) {
                kc[r] = kN[r];
                ubc[r] = ubN[r];
                slotc[r] = slotN[r];
            }
            const float2 Ec = EN;
            const int32_t eac = eaN;
            if (q + 1 < q1) load(q + 1);
            float S = 0.f, C = 0.f;
#pragma unroll
            for (int r = 0; r < R; r++) {
                if (!live[r]) continue;
                const df kv = df{kc[r].x, kc[r].y};
                if (vals) {
                    const df pr = df_mul_raw(df{Ec.x, Ec.y}, kv);
                    float s2, err;
                    two_sum(acc_h[slotc[r]], pr.h, s2, err);
                    acc_h[slotc[r]] = s2;
                    acc_l[slotc[r]] = __fadd_rn(acc_l[slotc[r]], __fadd_rn(pr.l, err));
                }
                if (SENS) {
                    const df t1 = df_mul_raw(df_mul_raw(kv, df{ubc[r].x, ubc[r].y}), df{ua[r].x, ua[r].y});
                    float s2, err;
                    two_sum(S, t1.h, s2, err);
                    S = s2;
                    C = __fadd_rn(C, __fadd_rn(t1.l, err));
                }
            }
            __syncwarp();
            if (SENS) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float So = __shfl_xor_sync(kFull, S, o), Co = __shfl_xor_sync(kFull, C, o);
                    float s2, err;
                    two_sum(S, So, s2, err);
                    S = s2;
                    C = __fadd_rn(__fadd_rn(C, Co), err);
                }
                if (lane == 0) {
                    float h, l;
                    two_sum(S, C, h, l);
                    part[eac] = df_to_double(h, l);
                }
            }
        }
        if (vals) {
            for (int t = lane; t < blk; t += 32) {
                float h, l;
                two_sum(acc_h[t], acc_l[t], h, l);
                __stcs(out + t, df_to_double(h, l));
            }
        }
        __syncwarp();
    }
}

// One thread per cell: s_e = sum_a part[e][a] in node order.  out[e] =
// g E'(rho_e) s_e with g = *gscale, or -1 (the compliance sensitivity).
__global__ void k_sens_finalize(int64_t nc, int nb, const double *__restrict__ part, const double *__restrict__ rho,
                                SimpParams sp, const double *__restrict__ gscale, double *__restrict__ out,
                                double *__restrict__ partial)
{
    __shared__ double wsum[8];
    const double g = gscale ? *gscale : -1.0;
    double mine = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int a = 0; a < nb; a++) s += part[e * nb + a];
        const double r = rho[e];
        if (out) out[e] = g * simp_dE(sp, r) * s;
        mine += simp_E(sp, r) * s;
    }
    if (partial) {
        mine = warp_sum(mine);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = mine;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += wsum[w];
            partial[blockIdx.x] = t;
        }
    }
}

int ggrid(int64_t items, int per) { return (int)std::max<int64_t>(1, std::min<int64_t>((items + per - 1) / per, 152 * 16)); }

template <int D, typename KT>
cudaError_t gather_t(const soptx_mesh_s &m, const double *rho, double *vals, bool sens, cudaStream_t st)
{
    const auto &h = m.h;
    const size_t sm = (size_t)kGW * 2 * D * D * h.max_deg * sizeof(float);
    const int rounds = (h.nb * D * D + 31) / 32;
    auto kern = sens ? k_gather_fused<D, KT, true> : k_gather_fused<D, KT, false>;
#define SOPTX_PICK(RR)                                                                                     \
    if (rounds == RR) kern = sens ? k_gather_unrolled<D, KT, true, RR> : k_gather_unrolled<D, KT, false, RR>;
    SOPTX_PICK(1)
    SOPTX_PICK(2)
    SOPTX_PICK(3)
    SOPTX_PICK(4)
    SOPTX_PICK(5)
    SOPTX_PICK(6)
#undef SOPTX_PICK
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    const KT *K = (const KT *)m.d.K;
    const int64_t kstride = m.path == SOPTX_PATH_CACHED ? (int64_t)h.ldof * h.ldof : 0;
    kern<<<ggrid(h.nn, kGW), kGW * 32, sm, st>>>(h.nn, h.nb, h.max_deg, m.d.node_off, m.d.inc_ptr, m.d.inc,
                                                 m.d.inc_e, m.d.inc_a, m.d.pos,
                                                 m.d.cell_node, K, kstride, m.d.Edf, m.d.udf, rho,
                                                 simp_params(m.mat), vals, m.d.part);
    return cudaGetLastError();
}

}  // namespace

int gather_finalize_grid(int64_t nc) { return ggrid(nc, 256); }

// vals may be nullptr (sensitivity only); u may be nullptr (assembly only).
cudaError_t launch_gather(const soptx_mesh_s &m, const double *rho, const double *u, double *vals, double *dc,
                          double *c, const double *gscale, cudaStream_t st)
{
    const auto &h = m.h;
    k_prep<<<ggrid(std::max(h.nc, u ? h.ndof : 0), 256), 256, 0, st>>>(h.nc, rho, simp_params(m.mat), m.d.Edf,
                                                                       h.ndof, u, m.d.udf);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const bool sens = u != nullptr;
    const bool f32 = m.prec == SOPTX_ELEM_FP32;
    if (h.nn > 0 && (vals || sens)) {
        if (h.dim == 2) err = f32 ? gather_t<2, float>(m, rho, vals, sens, st) : gather_t<2, float2>(m, rho, vals, sens, st);
        else err = f32 ? gather_t<3, float>(m, rho, vals, sens, st) : gather_t<3, float2>(m, rho, vals, sens, st);
        if (err != cudaSuccess) return err;
    }
    if (!sens) return cudaSuccess;
    const int grid = gather_finalize_grid(h.nc);
    k_sens_finalize<<<grid, 256, 0, st>>>(h.nc, h.nb, m.d.part, rho, simp_params(m.mat), gscale, dc,
                                          c ? m.d.scratch : nullptr);
    err = cudaGetLastError();
    if (err != cudaSuccess || !c) return err;
    k_reduce_partials<<<1, 256, 0, st>>>(grid, m.d.scratch, c);
    return cudaGetLastError();
}

}  // namespace soptx
