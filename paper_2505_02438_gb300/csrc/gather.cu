// General path (any mesh, per-cell K_e^0 cached on the device, or one shared
// K^0 when every cell has the same Jacobian), FP64-accurate on the FP32 pipes.
//
//  k_prep          : E(rho_e) per cell and, when u is given, u per dof, as
//                    float pairs (integer operations and float-pair SIMP).
//  k_gather_nodes  : a group of lanes owns the d rows of one node; it walks
//                    the node's incident cells in ascending order and for
//                    each reads the node's row block of K_e^0 once, adding
//                    E_e K_e^0 into the rows' CSR values (float-pair
//                    accumulators in shared memory, so every value is summed
//                    in ascending cell order, no atomics) and, when u is
//                    given, forming the cell's partial
//                    sum_i u_(a,i) sum_(b,j) K_e[(a,i),(b,j)] u_(b,j)  for
//                    this node a.  The rows leave through coalesced streaming
//                    stores.
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

// Resident CTAs per SM the generic gather is compiled for (the row gathers
// take theirs as a template argument): it caps the registers and, through the
// per-warp accumulator buffers, the warps a CTA gets.
constexpr int kGatherMinB = 2;

__global__ void k_prep(int64_t nc, const double *__restrict__ rho, SimpParams sp, float2 *__restrict__ Edf,
                       int64_t ndof, const double *__restrict__ u, float2 *__restrict__ udf)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc; e += stride) Edf[e] = simp_E_pair(sp, rho[e]);
    if (u)
        for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < ndof; r += stride) {
            const df v = df_split(u[r]);
            udf[r] = make_float2(v.h, v.l);
        }
}

// Arguments of the node-group gather.
template <typename KT>
struct GatherArgs {
    int64_t nn;
    int nb, max_deg, nck;
    const int64_t *__restrict__ node_off;
    const int32_t *__restrict__ inc_ptr;
    const int32_t *__restrict__ inc_e;
    const uint8_t *__restrict__ inc_a;
    const uint16_t *__restrict__ pos;
    const int32_t *__restrict__ cell_node;
    const int32_t *__restrict__ indices;
    const KT *__restrict__ K;
    int64_t kstride;
    const float2 *__restrict__ Edf;
    const float2 *__restrict__ udf;
    const double *__restrict__ rho;
    SimpParams sp;
    double *__restrict__ vals;
    double *__restrict__ part;
};

// E * k as an unnormalised pair: float pairs (FP64 element matrices) or a
// float (FP32 element matrices, one rounding-free TwoProd and one FMA).
__device__ __forceinline__ df mul_k(df E, float2 k) { return df_mul_raw(E, df{k.x, k.y}); }
__device__ __forceinline__ df mul_kf(df E, float k)
{
    const float p = __fmul_rn(E.h, k);
    return df{p, __fmaf_rn(E.l, k, __fmaf_rn(E.h, k, -p))};
}
template <typename KT> struct KEntry;
template <> struct KEntry<float2> {
    using T = float2;
    static __device__ __forceinline__ T load(const float2 *p) { return __ldcs(p); }
    static __device__ __forceinline__ T zero() { return make_float2(0.f, 0.f); }
    static __device__ __forceinline__ df mul(df a, T k) { return mul_k(a, k); }
};
template <> struct KEntry<float> {
    using T = float;
    static __device__ __forceinline__ T load(const float *p) { return __ldcs(p); }
    static __device__ __forceinline__ T zero() { return 0.f; }
    static __device__ __forceinline__ df mul(df a, T k) { return mul_kf(a, k); }
};

// Accumulate x into the unnormalised pair (s, c).
__device__ __forceinline__ void acc_add(float &s, float &c, df x)
{
    float t, err;
    two_sum(s, x.h, t, err);
    s = t;
    c = __fadd_rn(c, __fadd_rn(x.l, err));
}

// Plain-FP64 redo of one node by the whole warp (a modulus outside the
// float-pair range): rows into acc (as doubles), and the node's partials.
template <int D, typename KT>
__device__ __noinline__ void gather_node_fp64_warp(const GatherArgs<KT> &A, bool sens, int lane, int64_t n, int deg,
                                                   int32_t q0, int32_t cnt, double *acc)
{
    const int nb = A.nb, ldof = D * nb, rowlen = D * deg;
    const int per = nb * D * D;
    for (int t = lane; t < D * rowlen; t += 32) acc[t] = 0.0;
    __syncwarp();
    for (int32_t q = q0; q < q0 + cnt; q++) {
        const int64_t e = A.inc_e[q];
        const int a = A.inc_a[q];
        const double E = simp_E(A.sp, A.rho[e]);
        const KT *Ke = A.K + e * A.kstride;
        double s = 0.0;
        for (int t = lane; t < per; t += 32) {
            const int b = t / (D * D), i = (t / D) % D, j = t % D;
            const double k = KLoad<KT>::get64(Ke + (D * a + i) * ldof + D * b + j);
            if (A.vals) acc[i * rowlen + D * A.pos[(int64_t)q * nb + b] + j] += E * k;
            if (sens) {
                const float2 ua = A.udf[(int64_t)D * n + i], ub = A.udf[(int64_t)D * A.cell_node[e * nb + b] + j];
                s += ((double)ua.x + ua.y) * k * ((double)ub.x + ub.y);
            }
        }
        __syncwarp();
        if (sens) {
            s = warp_sum(s);
            if (lane == 0) A.part[e * nb + a] = s;
        }
    }
    __syncwarp();
    if (A.vals) {
        double *out = A.vals + (int64_t)D * D * A.node_off[n];
        for (int t = lane; t < D * rowlen; t += 32) __stcs(out + t, acc[t]);
    }
    __syncwarp();
}

// General path, any mesh.  A warp serves NPW nodes at once, GL = 32 / NPW
// lanes per node.  Lane ll of a group owns row i = ll / LPR of the node's d
// rows and the columns c, c + LPR, c + 2 LPR, ... (c = ll % LPR) of each
// incident cell's row block K_e^0[(a, i), :], so its entries of one cell are
// R rounds apart, and in each round the lanes of a row read consecutive
// entries.  Entry (b, j) of cell e lands in column block pos(e, b) of the
// node's rows, i.e. at offset s = d pos + j of row i; the displacement it
// meets, u_(b,j), is entry s of the node's neighbour displacements, staged
// in shared memory once per node from the CSR column indices.  For every
// incident cell (ascending) a lane adds E_e k into the node's row
// accumulators (float pairs in shared memory; no two lanes of a group hold
// the same slot within one cell, so there is no race and the order is fixed)
// and, with u, sums k u_(b,j) for its row; the group then forms the cell's
// partial  sum_i u_(a,i) (K_e u_e)_(a,i)  by a fixed-order butterfly.  The
// next cell's entries and positions are loaded while the current one is
// accumulated (its index two cells ahead).  Rows longer than R LPR columns
// take nck chunks (CH).
template <int D, typename KT, bool SENS, int NPW, int R, bool CH>
__global__ void __launch_bounds__(kGW * 32, kGatherMinB) k_gather_nodes(const GatherArgs<KT> A)
{
    using KE = KEntry<KT>;
    using KV = typename KE::T;
    constexpr int GL = 32 / NPW;
    constexpr int LPR = GL / D;
    extern __shared__ float2 smem_s[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int g = lane / GL, ll = lane % GL;
    const int irow = ll / LPR, c = ll - irow * LPR;
    const bool act = irow < D;
    const int i = act ? irow : 0;
    const int nb = A.nb, ldof = D * nb, nck = CH ? A.nck : 1;
    const int gslot = warp * NPW + g;
    const int acc_len = D * D * A.max_deg, un_len = SENS ? D * A.max_deg : 0;
    float2 *acc = smem_s + (size_t)gslot * acc_len;
    float2 *un = smem_s + (size_t)wpb * NPW * acc_len + (size_t)gslot * un_len;
    const int64_t step = (int64_t)gridDim.x * wpb * NPW;
    for (int64_t n0 = ((int64_t)blockIdx.x * wpb + warp) * NPW; n0 < A.nn; n0 += step) {
        const int64_t n = n0 + g;
        const bool has = n < A.nn;
        int64_t off = 0;
        int deg = 0;
        int32_t q0 = 0, cnt = 0;
        if (has) {
            off = A.node_off[n];
            deg = (int)(A.node_off[n + 1] - off);
            q0 = A.inc_ptr[n];
            cnt = A.inc_ptr[n + 1] - q0;
        }
        const int rowlen = D * deg, blk = D * rowlen;
        if (A.vals)
            for (int t = ll; t < blk; t += GL) acc[t] = make_float2(0.f, 0.f);
        df uni = df{0.f, 0.f};
        if (SENS) {
            // displacements of the node's neighbour dofs, in CSR column order
            const int32_t *cols = A.indices + (int64_t)D * D * off;
            for (int t = ll; t < rowlen; t += GL) un[t] = A.udf[cols[t]];
            if (has && act) {
                const float2 v = A.udf[(int64_t)D * n + i];
                uni = df{v.x, v.y};
            }
        }
        const int items = cnt * nck;
        int imax = items;
#pragma unroll
        for (int o = GL; o < 32; o <<= 1) imax = max(imax, __shfl_xor_sync(kFull, imax, o));
        __syncwarp();

        // item = (incidence t, chunk kc): the lane's R entries of it
        struct Item {
            KV k[R];
            int p[R];
            float2 E;
            int32_t ea;
        };
        auto fetch = [&](int it, int32_t e, int a, Item &d) {
            const bool on = it < items;
            const int t = !on ? 0 : (CH ? it / nck : it), kc = (!on || !CH) ? 0 : it - t * nck;
            d.E = on ? A.Edf[e] : make_float2(0.f, 0.f);
            d.ea = e * nb + a;
            const KT *kr = A.K + (int64_t)e * A.kstride + (int64_t)(D * a + i) * ldof + c + LPR * R * kc;
            const uint16_t *ps = A.pos + (int64_t)(q0 + t) * nb;
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int col = c + LPR * (R * kc + r);
                const bool lv = on && act && col < ldof;
                const int b = col / D, j = col - D * b;
                d.k[r] = lv ? KE::load(kr + LPR * r) : KE::zero();
                d.p[r] = lv ? D * ps[b] + j : -1;
            }
        };
        auto fetch_ea = [&](int it, int32_t &e, int &a) {
            const int t = CH ? it / nck : it;
            e = it < items ? A.inc_e[q0 + t] : 0;
            a = it < items ? A.inc_a[q0 + t] : 0;
        };
        int32_t e1, e2;
        int a1, a2;
        fetch_ea(0, e1, a1);
        fetch_ea(1, e2, a2);
        Item nxt;
        fetch(0, e1, a1, nxt);
        bool bad = false;
        float S = 0.f, C = 0.f;
        for (int it = 0; it < imax; it++) {
            const Item cur = nxt;
            e1 = e2;
            a1 = a2;
            fetch_ea(it + 2, e2, a2);
            fetch(it + 1, e1, a1, nxt);
            if (it < items) {
                bad |= isnan(cur.E.y);
                const df E = df{cur.E.x, cur.E.y};
                float2 *arow = acc + i * rowlen;
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const int s = cur.p[r];
                    if (s < 0) continue;
                    if (A.vals) {
                        float2 v = arow[s];
                        acc_add(v.x, v.y, KE::mul(E, cur.k[r]));
                        arow[s] = v;
                    }
                    if (SENS) {
                        const float2 ub = un[s];
                        acc_add(S, C, KE::mul(df{ub.x, ub.y}, cur.k[r]));
                    }
                }
            }
            __syncwarp();
            if (SENS && (!CH || it % nck == nck - 1)) {
                // the group's fixed-order butterfly of  u_(a,i) * (lane's share of (K_e u_e)_(a,i))
                float Sp, Cp;
                {
                    float h, l;
                    two_sum(S, C, h, l);
                    const df v = df_mul_raw(uni, df{h, l});
                    Sp = v.h;
                    Cp = v.l;
                }
#pragma unroll
                for (int o = GL / 2; o > 0; o >>= 1) {
                    const float So = __shfl_xor_sync(kFull, Sp, o), Co = __shfl_xor_sync(kFull, Cp, o);
                    float s, err;
                    two_sum(Sp, So, s, err);
                    Sp = s;
                    Cp = __fadd_rn(__fadd_rn(Cp, Co), err);
                }
                if (ll == 0 && it < items) {
                    float h, l;
                    two_sum(Sp, Cp, h, l);
                    A.part[cur.ea] = df_to_double(h, l);
                }
                S = 0.f;
                C = 0.f;
            }
        }
        // a group whose node met an out-of-range modulus is redone in FP64 by the whole warp
        const unsigned badm = __ballot_sync(kFull, bad);
        constexpr unsigned kGroup = GL == 32 ? kFull : ((1u << GL) - 1u);
        if (badm) {
#pragma unroll 1
            for (int gg = 0; gg < NPW; gg++) {
                if (!(badm & (kGroup << (gg * GL)))) continue;
                const int src = gg * GL;
                const int64_t ng = __shfl_sync(kFull, n, src);
                const int dg = __shfl_sync(kFull, deg, src);
                const int32_t qg = __shfl_sync(kFull, q0, src), cg = __shfl_sync(kFull, cnt, src);
                gather_node_fp64_warp<D, KT>(A, SENS, lane, ng, dg, qg, cg,
                                             reinterpret_cast<double *>(smem_s + (size_t)(warp * NPW + gg) * acc_len));
            }
        }
        if (A.vals && !(badm & (kGroup << (g * GL)))) {
            double *out = A.vals + (int64_t)D * D * off;
            for (int t = ll; t < blk; t += GL) {
                const float2 v = acc[t];
                __stcs(out + t, pair_to_double(v.x, v.y));
            }
        }
        __syncwarp();
    }
}

// The same gather for the cell types whose row blocks tile exactly into
// the group's lanes (d nb = LPR R): P2 tetrahedra, P3 triangles, Q1 hexahedra
// and Q1 quadrilaterals.  Every
// lane-round constant is fixed at compile time or per lane; the positions of
// a cell's nodes arrive once per cell (lane b of the group loads pos(e, b))
// and reach the lanes that need them by shuffles; the item loop is unrolled
// by two so the prefetched item never has to be copied.
template <int D, int NB, typename KT, bool SENS, int NPW, int R, int LPR, int MINB>
__global__ void __launch_bounds__(kGW * 32, MINB) k_gather_rows(const GatherArgs<KT> A)
{
    using KE = KEntry<KT>;
    using KV = typename KE::T;
    constexpr int GL = 32 / NPW, LDOF = D * NB, NPOS = (NB + GL - 1) / GL;
    static_assert(LPR * R == LDOF && D * LPR <= GL, "the rounds must tile the row block");
    static_assert(NPOS <= 2, "at most two positions per lane");
    extern __shared__ float2 smem_s[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int g = lane / GL, ll = lane % GL;
    const int irow = ll / LPR, c = ll - irow * LPR;
    const bool act = irow < D;
    const int i = act ? irow : 0;
    int srcl[R], jr[R];
    bool hi[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int col = c + LPR * r, b = col / D;
        jr[r] = col - D * b;
        srcl[r] = g * GL + b % GL;
        hi[r] = b >= GL;
    }
    const int gslot = warp * NPW + g;
    const int acc_len = D * D * A.max_deg, un_len = SENS ? D * A.max_deg : 0;
    float2 *acc = smem_s + (size_t)gslot * acc_len;
    float2 *un = smem_s + (size_t)wpb * NPW * acc_len + (size_t)gslot * un_len;
    const int64_t step = (int64_t)gridDim.x * wpb * NPW;
    for (int64_t n0 = ((int64_t)blockIdx.x * wpb + warp) * NPW; n0 < A.nn; n0 += step) {
        const int64_t n = n0 + g;
        const bool has = n < A.nn;
        int64_t off = 0;
        int deg = 0;
        int32_t q0 = 0, cnt = 0;
        if (has) {
            off = A.node_off[n];
            deg = (int)(A.node_off[n + 1] - off);
            q0 = A.inc_ptr[n];
            cnt = A.inc_ptr[n + 1] - q0;
        }
        const int rowlen = D * deg, blk = D * rowlen;
        if (A.vals)
            for (int t = ll; t < blk; t += GL) acc[t] = make_float2(0.f, 0.f);
        df uni = df{0.f, 0.f};
        if (SENS) {
            const int32_t *cols = A.indices + (int64_t)D * D * off;
            for (int t = ll; t < rowlen; t += GL) un[t] = A.udf[cols[t]];
            if (has && act) {
                const float2 v = A.udf[(int64_t)D * n + i];
                uni = df{v.x, v.y};
            }
        }
        int imax = cnt;
#pragma unroll
        for (int o = GL; o < 32; o <<= 1) imax = max(imax, __shfl_xor_sync(kFull, imax, o));
        __syncwarp();

        struct Item {
            KV k[R];
            int pv[NPOS];
            float2 E;
            int32_t ea;
        };
        auto fetch = [&](int it, int32_t e, int a, Item &d) {
            const bool on = it < cnt;
            d.E = on ? A.Edf[e] : make_float2(0.f, 0.f);
            d.ea = e * NB + a;
            const KT *kr = A.K + (int64_t)e * A.kstride + (int64_t)(D * a + i) * LDOF + c;
#pragma unroll
            for (int r = 0; r < R; r++) d.k[r] = (on && act) ? KE::load(kr + LPR * r) : KE::zero();
            const uint16_t *ps = A.pos + (int64_t)(q0 + it) * NB;
#pragma unroll
            for (int q = 0; q < NPOS; q++) d.pv[q] = (on && ll + q * GL < NB) ? (int)ps[ll + q * GL] : 0;
        };
        int32_t e1 = 0, e2 = 0;
        int a1 = 0, a2 = 0;
        auto fetch_ea = [&](int it, int32_t &e, int &a) {
            e = it < cnt ? A.inc_e[q0 + it] : 0;
            a = it < cnt ? A.inc_a[q0 + it] : 0;
        };
        bool bad = false;
        auto body = [&](const Item &cur, Item &nxt, int it) {
            e1 = e2;
            a1 = a2;
            fetch_ea(it + 2, e2, a2);
            fetch(it + 1, e1, a1, nxt);
            int s[R];
#pragma unroll
            for (int r = 0; r < R; r++) {
                int pb = __shfl_sync(kFull, cur.pv[0], srcl[r]);
                if (NPOS == 2) {
                    const int p1 = __shfl_sync(kFull, cur.pv[NPOS - 1], srcl[r]);
                    pb = hi[r] ? p1 : pb;
                }
                s[r] = D * pb + jr[r];
            }
            float S = 0.f, C = 0.f;
            if (it < cnt && act) {
                bad |= isnan(cur.E.y);
                const df E = df{cur.E.x, cur.E.y};
                float2 *arow = acc + i * rowlen;
                // a lane's R slots are distinct (distinct columns of one cell), so all
                // of them are read before any is written back: one shared-memory round
                // trip per cell instead of R dependent ones
                if (A.vals) {
                    float2 v[R];
#pragma unroll
                    for (int r = 0; r < R; r++) v[r] = arow[s[r]];
#pragma unroll
                    for (int r = 0; r < R; r++) acc_add(v[r].x, v[r].y, KE::mul(E, cur.k[r]));
#pragma unroll
                    for (int r = 0; r < R; r++) arow[s[r]] = v[r];
                }
                if (SENS) {
                    float2 ub[R];
#pragma unroll
                    for (int r = 0; r < R; r++) ub[r] = un[s[r]];
#pragma unroll
                    for (int r = 0; r < R; r++) acc_add(S, C, KE::mul(df{ub[r].x, ub[r].y}, cur.k[r]));
                }
            }
            __syncwarp();
            if (SENS) {
                float Sp, Cp;
                {
                    float h, l;
                    two_sum(S, C, h, l);
                    const df v = df_mul_raw(uni, df{h, l});
                    Sp = v.h;
                    Cp = v.l;
                }
#pragma unroll
                for (int o = GL / 2; o > 0; o >>= 1) {
                    const float So = __shfl_xor_sync(kFull, Sp, o), Co = __shfl_xor_sync(kFull, Cp, o);
                    float s2, err;
                    two_sum(Sp, So, s2, err);
                    Sp = s2;
                    Cp = __fadd_rn(__fadd_rn(Cp, Co), err);
                }
                if (ll == 0 && it < cnt) {
                    float h, l;
                    two_sum(Sp, Cp, h, l);
                    A.part[cur.ea] = df_to_double(h, l);
                }
            }
        };
        fetch_ea(0, e1, a1);
        fetch_ea(1, e2, a2);
        Item I0, I1;
        fetch(0, e1, a1, I0);
        for (int it = 0; it < imax; it += 2) {
            body(I0, I1, it);
            if (it + 1 < imax) body(I1, I0, it + 1);
        }
        const unsigned badm = __ballot_sync(kFull, bad);
        constexpr unsigned kGroup = GL == 32 ? kFull : ((1u << GL) - 1u);
        if (badm) {
#pragma unroll 1
            for (int gg = 0; gg < NPW; gg++) {
                if (!(badm & (kGroup << (gg * GL)))) continue;
                const int src = gg * GL;
                const int64_t ng = __shfl_sync(kFull, n, src);
                const int dg = __shfl_sync(kFull, deg, src);
                const int32_t qg = __shfl_sync(kFull, q0, src), cg = __shfl_sync(kFull, cnt, src);
                gather_node_fp64_warp<D, KT>(A, SENS, lane, ng, dg, qg, cg,
                                             reinterpret_cast<double *>(smem_s + (size_t)(warp * NPW + gg) * acc_len));
            }
        }
        if (A.vals && !(badm & (kGroup << (g * GL)))) {
            double *out = A.vals + (int64_t)D * D * off;
            for (int t = ll; t < blk; t += GL) {
                const float2 v = acc[t];
                __stcs(out + t, pair_to_double(v.x, v.y));
            }
        }
        __syncwarp();
    }
}

// One thread per cell: s_e = sum_a part[e][a] in node order.  out[e] =
// g E'(rho_e) s_e with g = *gscale, or -1 (the compliance sensitivity).  With
// c, also c = sum_e E_e s_e over the grid (fixed order, last block).
__global__ void __launch_bounds__(256) k_sens_finalize(int64_t nc, int nb, const double *__restrict__ part,
                                                       const double *__restrict__ rho, SimpParams sp,
                                                       const double *__restrict__ gscale, double *__restrict__ out,
                                                       double *__restrict__ partial, unsigned *__restrict__ counter,
                                                       double *__restrict__ c)
{
    const double g = gscale ? *gscale : -1.0;
    double mine = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int a = 0; a < nb; a++) s += part[e * nb + a];
        const double r = rho[e];
        if (out) out[e] = g * simp_dE(sp, r) * s;
        mine += simp_E(sp, r) * s;
    }
    if (c) grid_sum_last_block(mine, partial, counter, c);
}

int ggrid(int64_t items, int per) { return (int)std::max<int64_t>(1, std::min<int64_t>((items + per - 1) / per, 152 * 16)); }

// Launch of one gather: NPW nodes per warp, lpr lanes per row, R rounds per
// chunk, and as many warps per CTA as let minb CTAs share an SM's shared
// memory (the layouts per cell type are chosen in gather_t).
template <int D, typename KT, int NPW, typename Kern>
cudaError_t gather_launch(const soptx_mesh_s &m, const double *rho, double *vals, bool sens, int R, int lpr,
                          int minb, Kern kern, cudaStream_t st)
{
    const auto &h = m.h;
    GatherArgs<KT> A;
    A.nn = h.nn;
    A.nb = h.nb;
    A.max_deg = h.max_deg;
    const int rounds = (h.ldof + lpr - 1) / lpr;
    A.nck = (rounds + R - 1) / R;
    A.node_off = m.d.node_off;
    A.inc_ptr = m.d.inc_ptr;
    A.inc_e = m.d.inc_e;
    A.inc_a = m.d.inc_a;
    A.pos = m.d.pos;
    A.cell_node = m.d.cell_node;
    A.indices = m.d.indices;
    A.K = (const KT *)m.d.K;
    A.kstride = m.path == SOPTX_PATH_CACHED ? (int64_t)h.ldof * h.ldof : 0;
    A.Edf = m.d.Edf;
    A.udf = m.d.udf;
    A.rho = rho;
    A.sp = simp_params(m.mat);
    A.vals = vals;
    A.part = sens ? m.d.part : nullptr;
    const size_t per_warp = (size_t)NPW * (D * D + (sens ? D : 0)) * h.max_deg * sizeof(float2);
    // minb CTAs must fit in the SM's 228 KiB of shared memory (1 KiB of it reserved per CTA)
    const size_t cta_smem = std::min<size_t>(200 * 1024, (228 * 1024) / minb - 1024);
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(kGW, cta_smem / per_warp));
    const size_t smem = per_warp * wpb;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int64_t groups = (h.nn + NPW - 1) / NPW;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((groups + wpb - 1) / wpb, 152 * 16));
    kern<<<grid, wpb * 32, smem, st>>>(A);
    return cudaGetLastError();
}

template <int D, typename KT>
cudaError_t gather_t(const soptx_mesh_s &m, const double *rho, double *vals, bool sens, cudaStream_t st)
{
    const int nb = m.h.nb;
#define SOPTX_ROWS(NB, SENS, NPW, R, LPR, MINB)                                                                \
    return gather_launch<D, KT, NPW>(m, rho, vals, sens, R, LPR, MINB,                                        \
                                     k_gather_rows<D, NB, KT, SENS, NPW, R, LPR, MINB>, st)
    // Per cell type the lane layout and the CTAs per SM, measured: with the
    // sensitivity the kernels hold more registers and run at 3 CTAs per SM
    // (80 registers); the assembly alone fits in 64 registers at 4 CTAs per SM.
    if constexpr (D == 3) {
        if (nb == 10) {   // P2 tetrahedra
            if (sens) SOPTX_ROWS(10, true, 2, 6, 5, 3);   // 2 nodes x 3 rows x 5 lanes, 6 rounds
            SOPTX_ROWS(10, false, 1, 3, 10, 4);           // 1 node x 3 rows x 10 lanes, 3 rounds
        }
        if (nb == 8) {    // Q1 hexahedra
            if (sens) SOPTX_ROWS(8, true, 2, 6, 4, 3);    // 2 nodes x 3 rows x 4 lanes, 6 rounds
            SOPTX_ROWS(8, false, 1, 3, 8, 4);             // 1 node x 3 rows x 8 lanes, 3 rounds
        }
    } else {
        if (nb == 10) {   // P3 triangles: 4 nodes x 2 rows x 4 lanes, 5 rounds
            if (sens) SOPTX_ROWS(10, true, 4, 5, 4, 3);
            SOPTX_ROWS(10, false, 4, 5, 4, 4);
        }
        if (nb == 4) {    // Q1 quadrilaterals: 4 nodes x 2 rows x 4 lanes, 2 rounds
            if (sens) SOPTX_ROWS(4, true, 4, 2, 4, 3);
            SOPTX_ROWS(4, false, 4, 2, 4, 4);
        }
    }
#undef SOPTX_ROWS
    return gather_launch<D, KT, 1>(m, rho, vals, sens, 4, 32 / D, kGatherMinB,
                                   sens ? k_gather_nodes<D, KT, true, 1, 4, true> : k_gather_nodes<D, KT, false, 1, 4, true>, st);
}

}  // namespace

int gather_finalize_grid(int64_t nc) { return ggrid(nc, 256); }

// E(rho_e) per cell (and, with u, u per dof) as float pairs into the mesh's buffers.
cudaError_t launch_prep(const soptx_mesh_s &m, const double *rho, const double *u, cudaStream_t st)
{
    const auto &h = m.h;
    k_prep<<<ggrid(std::max(h.nc, u ? h.ndof : 0), 256), 256, 0, st>>>(h.nc, rho, simp_params(m.mat), m.d.Edf,
                                                                       h.ndof, u, m.d.udf);
    return cudaGetLastError();
}

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
    k_sens_finalize<<<grid, 256, 0, st>>>(h.nc, h.nb, m.d.part, rho, simp_params(m.mat), gscale, dc, m.d.scratch,
                                          m.d.counter, c);
    return cudaGetLastError();
}

}  // namespace soptx
