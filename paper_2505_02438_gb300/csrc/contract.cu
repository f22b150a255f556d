// General (non-lattice) meshes of affine cells: the element matrices formed in
// registers from the reference integrals and each cell's Jacobian, and the
// sensitivities from the strain energy at quadrature points.
//
//  k_contract_rows : FP32 element matrices, never stored.  A group of NB lanes
//                    (NB = basis functions per cell) owns the d rows of one
//                    node and walks the node's incident cells as a chain
//                    fixed at mesh creation (each next cell shares as many
//                    of the lanes' current column nodes as possible); for
//                    each cell, a lane takes one local node b and forms the
//                    d x d block K_e^0[(a,.),(b,.)] of the node's local
//                    index a by the
//                    fast assembly of Sec. 3.2.2: the reference integrals
//                    M^{kl}_{ab} = int d_k phi_a d_l phi_b (shared memory,
//                    FP32) contracted with the cell's G = J^-1 and |det J|,
//                        P_ij = |det J| sum_kl G_ki G_lj M^{kl}_{ab},
//                        K_ij = lam P_ij + mu P_ji + mu delta_ij tr P,
//                    and adds E_e K_ij into the rows' float-pair accumulators
//                    in shared memory (FP64-accurate sums in the chain's
//                    fixed order, no atomics); a lane whose column block
//                    continues into the next cell keeps its sums in
//                    registers meanwhile.  The rows leave as FP64 values.
//  k_strain_energy : s_e = u_e^T K_e^0 u_e = int_e lam (div u)^2 + 2 mu eps:eps
//                    by a quadrature rule exact for the energy density of the
//                    cell's order, one thread per cell: the reference
//                    displacement gradient U^_q = sum_b u_b (grad^ phi_b(xi_q))^T,
//                    grad u = U^_q G, the density lam (tr grad u)^2 +
//                    mu sum_ij g_ij (g_ij + g_ji); in float pairs for FP64
//                    element matrices (FP64-accurate) or in FP32 for FP32 ones.
//                    dc_e = -E'(rho_e) s_e, c = sum_e E(rho_e) s_e in FP64
//                    (fixed-order block partials, last block adds them).
#include <algorithm>
#include <cstdint>

#include "df64.cuh"
#include "internal.h"
#include "kernels_common.cuh"

namespace soptx {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Per-cell record of the contraction (FP32): G row-major (G[m][i] = (J^-1)_{mi})
// then |det J|, padded to whole float4s.
template <int D> struct CGeo {
    static constexpr int n4 = D == 3 ? 3 : 2;
};
// Reference integrals of one (a, b) pair in shared memory: M[k][l] padded to
// whole float4s.
template <int D> struct MPad {
    static constexpr int n = D == 3 ? 12 : 4;
};

struct ContractArgs {
    int64_t nn;
    int max_deg;
    const int4 *__restrict__ nrec;       // per processing position: row block offset, q0, cnt << 16 | deg
    unsigned *__restrict__ ticket;       // [0] rounds handed out, [1] warps done (both zero between calls)
    const int32_t *__restrict__ inc_e;   // each node's cells in chain order
    const uint8_t *__restrict__ inc_a;   // the node's local index in each
    const uint16_t *__restrict__ rec;    // per (incidence, lane): column block p (bits 0-8), local node b
                                         // (9-13), first (14) / last (15) meeting of the block
    const float4 *__restrict__ cgeo;
    const float *__restrict__ Mf;
    const float2 *__restrict__ Edf;
    const double *__restrict__ rho;
    SimpParams sp;
    float lam, mu;
    double *__restrict__ vals;
};

// The d x d block K_e^0[(a,.),(b,.)] in FP32 from the pair's reference
// integrals M (d x d, row-major) and the cell's G and |det J|.
template <int D>
__device__ __forceinline__ void contract_block(const float *M, const float *G, float det, float lam, float mu,
                                               float K[D][D])
{
    float T[D][D];
#pragma unroll
    for (int k = 0; k < D; k++)
#pragma unroll
        for (int j = 0; j < D; j++) {
            float t = M[k * D] * G[j];
#pragma unroll
            for (int l = 1; l < D; l++) t = fmaf(M[k * D + l], G[l * D + j], t);
            T[k][j] = t;
        }
    float P[D][D];
#pragma unroll
    for (int i = 0; i < D; i++)
#pragma unroll
        for (int j = 0; j < D; j++) {
            float p = G[i] * T[0][j];
#pragma unroll
            for (int k = 1; k < D; k++) p = fmaf(G[k * D + i], T[k][j], p);
            P[i][j] = p;
        }
    float tr = P[0][0];
#pragma unroll
    for (int m = 1; m < D; m++) tr += P[m][m];
    const float l2 = det * lam, m2 = det * mu;
#pragma unroll
    for (int i = 0; i < D; i++)
#pragma unroll
        for (int j = 0; j < D; j++) K[i][j] = fmaf(l2, P[i][j], m2 * (i == j ? P[j][i] + tr : P[j][i]));
}

template <int D>
__device__ __forceinline__ void load_cgeo(const float4 *__restrict__ cg, int64_t e, float G[D * D], float &det)
{
    if (D == 3) {
        const float4 g0 = __ldg(cg + 3 * e), g1 = __ldg(cg + 3 * e + 1), g2 = __ldg(cg + 3 * e + 2);
        G[0] = g0.x; G[1] = g0.y; G[2] = g0.z; G[3] = g0.w;
        G[4] = g1.x; G[5] = g1.y; G[6] = g1.z; G[7] = g1.w;
        G[8] = g2.x;
        det = g2.y;
    } else {
        const float4 g0 = __ldg(cg + 2 * e), g1 = __ldg(cg + 2 * e + 1);
        G[0] = g0.x; G[1] = g0.y; G[2] = g0.z; G[3] = g0.w;
        det = g1.x;
    }
}

template <int D>
__device__ __forceinline__ void load_mpair(const float *Ms, int pair, float M[D * D])
{
    const float4 *p = reinterpret_cast<const float4 *>(Ms + pair * MPad<D>::n);
    if (D == 3) {
        const float4 a = p[0], b = p[1], c = p[2];
        M[0] = a.x; M[1] = a.y; M[2] = a.z; M[3] = a.w;
        M[4] = b.x; M[5] = b.y; M[6] = b.z; M[7] = b.w;
        M[8] = c.x;
    } else {
        const float4 a = p[0];
        M[0] = a.x; M[1] = a.y; M[2] = a.z; M[3] = a.w;
    }
}

// Accumulate x into the unnormalised pair (s, c).
__device__ __forceinline__ void acc_add(float &s, float &c, df x)
{
    float t, err;
    two_sum(s, x.h, t, err);
    s = t;
    c = __fadd_rn(c, __fadd_rn(x.l, err));
}

// Plain-FP64 redo of one node by its group (a modulus outside the float-pair
// range): the same FP32 blocks times E(rho_e) in FP64, summed in ascending
// cell order into acc (as doubles), then stored.
template <int D, int NB>
__device__ __noinline__ void contract_node_fp64(const ContractArgs &A, const float *Ms, unsigned gmask, int b,
                                                int64_t off, int deg, int32_t q0, int32_t cnt, double *acc)
{
    const int rowlen = D * deg, blk = D * rowlen;
    for (int t = b; t < blk; t += NB) acc[t] = 0.0;
    __syncwarp(gmask);
    for (int32_t t = 0; t < cnt; t++) {
        const int32_t q = q0 + t;
        const int64_t e = A.inc_e[q];
        const int a = A.inc_a[q];
        const uint32_t r = A.rec[(int64_t)q * NB + b];
        const int p = (int)(r & 511u), lb = (int)((r >> 9) & 31u);
        float G[D * D], det, M[D * D], K[D][D];
        load_cgeo<D>(A.cgeo, e, G, det);
        load_mpair<D>(Ms, a * NB + lb, M);
        contract_block<D>(M, G, det, A.lam, A.mu, K);
        const double E = simp_E(A.sp, A.rho[e]);
#pragma unroll
        for (int i = 0; i < D; i++)
#pragma unroll
            for (int j = 0; j < D; j++) acc[i * rowlen + D * p + j] += E * (double)K[i][j];
        __syncwarp(gmask);
    }
    double *out = A.vals + (int64_t)D * D * off;
    for (int t = b; t < blk; t += NB) __stcs(out + t, acc[t]);
    __syncwarp(gmask);
}

// NPW = 32 / NB nodes per warp, NB lanes each; lanes beyond NPW NB idle.
template <int D, int NB, int MINB>
__global__ void __launch_bounds__(256, MINB) k_contract_rows(const ContractArgs A)
{
    constexpr int NPW = 32 / NB;
    constexpr int MP = MPad<D>::n;
    constexpr int G4 = CGeo<D>::n4;
    extern __shared__ float4 csm4[];
    float *Ms = reinterpret_cast<float *>(csm4);
    float2 *accs = reinterpret_cast<float2 *>(Ms + NB * NB * MP);
    for (int t = threadIdx.x; t < NB * NB * MP; t += blockDim.x) Ms[t] = A.Mf[t];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int g = lane / NB, b = lane - g * NB;
    const bool act = g < NPW;
    const int gg = act ? g : NPW - 1;
    const unsigned gmask = (NB == 32 ? kFull : ((1u << NB) - 1u)) << (gg * NB);
    const int acc_len = D * D * A.max_deg;
    const int gacc = (warp * NPW + gg) * acc_len;   // the group's accumulators: accs[gacc ...]
    // Round r takes positions r NPW .. r NPW + NPW - 1 of the processing order
    // (nodes by incident-cell count, largest first), so a warp's groups walk
    // about as many cells each.  Warps take rounds from a counter, three ahead
    // (the prefetch below reaches two rounds past the current one), so a CTA
    // that starts late, beside another kernel, simply takes fewer.  The last warp
    // to finish sets the counter back to zero.  A node's record is one 16-byte load.
    const int64_t rounds = (A.nn + NPW - 1) / NPW;
    const bool aligned16 = (reinterpret_cast<uintptr_t>(A.vals) & 15u) == 0;
    auto grab = [&]() -> int64_t {
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(A.ticket, 1u);
        return (int64_t)__shfl_sync(kFull, t, 0);
    };
    struct Node {
        int64_t off;
        int32_t q0, cnt, deg;
    };
    auto load_node = [&](int64_t n0, Node &N) {
        N = Node{0, 0, 0, 0};
        if (act && n0 + g < A.nn) {
            const int4 r = __ldg(A.nrec + n0 + g);
            N.off = (int64_t)(uint32_t)r.x | ((int64_t)r.y << 32);
            N.q0 = r.z;
            N.cnt = (int32_t)((uint32_t)r.w >> 16);
            N.deg = r.w & 0xffff;
        }
    };
    auto warp_max = [](int x) { return (int)__reduce_max_sync(kFull, (unsigned)x); };
    struct Cell {
        float4 g[G4];
        float2 E;
        int a, p;
    };
    // The rounds' incidences form one stream: cell, a and the lane record are
    // loaded two items ahead, geometry and modulus one ahead, across the end of
    // a round into the next one (or the one after, when the next has a single
    // item), so a node's first cells are in flight while the previous node's
    // rows are written.  Position s counts from the current round's first item;
    // a group's index past its node's last incidence is clamped to it (the item
    // is not used), so the loads need no predicates.
    // the round after next: only its first incidence and cell count
    auto load_head = [&](int64_t n0, int32_t &q, int32_t &c) {
        q = 0;
        c = 0;
        if (act && n0 + g < A.nn) {
            const int2 r = __ldg(reinterpret_cast<const int2 *>(A.nrec + n0 + g) + 1);
            q = r.x;
            c = (int32_t)((uint32_t)r.y >> 16);
        }
    };
    Node N0, N1;
    int32_t q02, cnt2;
    int64_t r0 = grab(), r1 = grab(), r2 = grab();
    load_node(r0 * NPW, N0);
    load_node(r1 * NPW, N1);
    load_head(r2 * NPW, q02, cnt2);
    int imax0 = warp_max(N0.cnt), imax1 = warp_max(N1.cnt);
    auto fetch_idx = [&](int s, int32_t &e, int &a, int &p) {
        int32_t qs = N0.q0, cs = N0.cnt;
        int k = s;
        if (s >= imax0) {
            k = s - imax0;
            if (k < imax1) {
                qs = N1.q0;
                cs = N1.cnt;
            } else {
                k -= imax1;
                qs = q02;
                cs = cnt2;
            }
        }
        const int32_t q = qs + min(k, max(cs - 1, 0));
        e = __ldg(A.inc_e + q);
        a = __ldg(A.inc_a + q);
        p = __ldg(A.rec + (int64_t)q * NB + b);
    };
    auto fetch_data = [&](int32_t e, int a, int p, Cell &c) {
        const float4 *gp = A.cgeo + (int64_t)G4 * e;
#pragma unroll
        for (int w = 0; w < G4; w++) c.g[w] = __ldg(gp + w);
        c.E = __ldg(A.Edf + e);
        c.a = a;
        c.p = p;
    };
    int32_t e1, e2;
    int a1, p1, a2, p2;
    fetch_idx(0, e1, a1, p1);
    fetch_idx(1, e2, a2, p2);
    Cell c0, c1;
    fetch_data(e1, a1, p1, c0);
    while (r0 < rounds) {
        const int64_t n0 = r0 * NPW;
        const bool has = act && n0 + g < A.nn;
        const int64_t off = N0.off;
        const int deg = N0.deg;
        const int32_t q0 = N0.q0, cnt = N0.cnt;
        // 3D: no zeroing, every block of the rows is met by some cell and its first
        // meeting starts the sums from zero; 2D (few rows, a tight register budget)
        // zeroes the rows first
        constexpr bool kFirst = D == 3;   // (in 2D it spilled at the 80-register cap: P3 236 -> 254 us)
        // 2D: a block's last meeting converts it and stores it straight to the rows
        // (few contributions per value there), so there is no output pass
        constexpr bool kDirect = D == 2;
        double *const out = A.vals + (int64_t)D * D * off;
        const int rowlen = D * deg, blk = D * rowlen;
        if (!kFirst) {
            for (int t = b; t < blk; t += NB) accs[gacc + t] = make_float2(0.f, 0.f);
            __syncwarp();
        }

        const int ro1 = rowlen, ro2 = 2 * rowlen;
        bool bad = false;
        // the lane's row sums of its current column block: read from shared memory
        // when the block starts, written back when the next cell has another one
        float2 v[D][D];
        bool held = false;
        auto body = [&](const Cell &cur, Cell &nxt, int it) {
            fetch_data(e2, a2, p2, nxt);
            fetch_idx(it + 2, e2, a2, p2);
            if (it < cnt) {
                bad |= isnan(cur.E.y);
                float G[D * D], det;
                if (D == 3) {
                    G[0] = cur.g[0].x; G[1] = cur.g[0].y; G[2] = cur.g[0].z; G[3] = cur.g[0].w;
                    G[4] = cur.g[1].x; G[5] = cur.g[1].y; G[6] = cur.g[1].z; G[7] = cur.g[1].w;
                    G[8] = cur.g[2].x;
                    det = cur.g[2].y;
                } else {
                    G[0] = cur.g[0].x; G[1] = cur.g[0].y; G[2] = cur.g[0].z; G[3] = cur.g[0].w;
                    det = cur.g[1].x;
                }
                const int slot = cur.p & 511, lb = (cur.p >> 9) & 31;
                float M[D * D], K[D][D];
                load_mpair<D>(Ms, cur.a * NB + lb, M);
                contract_block<D>(M, G, det, A.lam, A.mu, K);
                // the lane's slots are distinct within a cell, and a block held in
                // registers is no other lane's in the next cell
                const int base = gacc + D * slot;
                const int rbase[3] = {base, base + ro1, base + ro2};
                const bool keep = it + 1 < cnt && (nxt.p & 511) == slot;
                if (!held) {
                    if (kFirst && (cur.p & 0x4000)) {
#pragma unroll
                        for (int i = 0; i < D; i++)
#pragma unroll
                            for (int j = 0; j < D; j++) v[i][j] = make_float2(0.f, 0.f);
                    } else {
#pragma unroll
                        for (int i = 0; i < D; i++)
#pragma unroll
                            for (int j = 0; j < D; j++) v[i][j] = accs[rbase[i] + j];
                    }
                }
#pragma unroll
                for (int i = 0; i < D; i++)
#pragma unroll
                    for (int j = 0; j < D; j++) {
                        // E K as a pair: TwoProd of the head, the tail's product
                        const float k = K[i][j];
                        const float ph = __fmul_rn(cur.E.x, k);
                        const float pl = __fmaf_rn(cur.E.y, k, __fmaf_rn(cur.E.x, k, -ph));
                        acc_add(v[i][j].x, v[i][j].y, df{ph, pl});
                    }
                if (!keep) {
                    if (kDirect && (cur.p & 0x8000)) {
#pragma unroll
                        for (int i = 0; i < D; i++) {
                            double *o = out + (int64_t)i * rowlen + D * slot;
                            // row 0 widens on the FP64 pipe, row 1 with integer operations
                            // only: the two pipes share the conversions
                            double d0, d1;
                            if (i == 0) {
                                d0 = pair_to_double(v[i][0].x, v[i][0].y);
                                d1 = pair_to_double(v[i][1].x, v[i][1].y);
                            } else {
                                float h, l;
                                two_sum(v[i][0].x, v[i][0].y, h, l);
                                d0 = df_to_double(h, l);
                                two_sum(v[i][1].x, v[i][1].y, h, l);
                                d1 = df_to_double(h, l);
                            }
                            if (aligned16) {
                                __stcs(reinterpret_cast<double2 *>(o), make_double2(d0, d1));
                            } else {
                                __stcs(o, d0);
                                __stcs(o + 1, d1);
                            }
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < D; i++)
#pragma unroll
                            for (int j = 0; j < D; j++) accs[rbase[i] + j] = v[i][j];
                    }
                }
                held = keep;
            }
            __syncwarp();
        };
        for (int it = 0; it < imax0; it += 2) {
            body(c0, c1, it);
            if (it + 1 < imax0) body(c1, c0, it + 1);
        }
        if (imax0 & 1) {
            // after an odd count the next round's first cell arrived in c1
            const Cell t = c0;
            c0 = c1;
            c1 = t;
        }
        // a group whose node met an out-of-range modulus redoes it in FP64
        const unsigned badm = __ballot_sync(kFull, bad);
        if (has && (badm & gmask)) {
            contract_node_fp64<D, NB>(A, Ms, gmask, b, off, deg, q0, cnt, reinterpret_cast<double *>(accs + gacc));
        } else if (has && !kDirect) {
            // the rows leave as FP64 values, two per store where the destination is
            // 16-byte aligned (an odd 8-byte head is stored on its own)
            const int head = (int)((reinterpret_cast<uintptr_t>(out) >> 3) & 1u);
            if (head && b == 0) {
                const float2 v = accs[gacc];
                __stcs(out, pair_to_double(v.x, v.y));
            }
            for (int t = head + 2 * b; t < blk; t += 2 * NB) {
                const float2 v0 = accs[gacc + t];
                const double d0 = pair_to_double(v0.x, v0.y);
                if (t + 1 < blk) {
                    const float2 v1 = accs[gacc + t + 1];
                    __stcs(reinterpret_cast<double2 *>(out + t), make_double2(d0, pair_to_double(v1.x, v1.y)));
                } else {
                    __stcs(out + t, d0);
                }
            }
        }
        __syncwarp();
        r0 = r1;
        r1 = r2;
        r2 = grab();
        N0 = N1;
        load_node(r1 * NPW, N1);
        load_head(r2 * NPW, q02, cnt2);
        imax0 = imax1;
        imax1 = warp_max(N1.cnt);
    }
    if (lane == 0) {
        __threadfence();
        if (atomicAdd(A.ticket + 1, 1u) == gridDim.x * (unsigned)wpb - 1u) {
            A.ticket[0] = 0u;
            A.ticket[1] = 0u;
        }
    }
}

// ------------------------------------------------------------------ strain energy

// Arithmetic of the sensitivity: float pairs (FP64 element matrices) or FP32.
template <bool PAIR> struct SArith;
template <> struct SArith<true> {
    using V = df;
    struct Acc {
        float s = 0.f, c = 0.f;
    };
    static __device__ __forceinline__ void fma(Acc &a, V x, V y) { acc_add(a.s, a.c, df_mul_raw(x, y)); }
    static __device__ __forceinline__ V val(const Acc &a)
    {
        df r;
        two_sum(a.s, a.c, r.h, r.l);
        return r;
    }
    static __device__ __forceinline__ V add(V x, V y) { return df_add_lazy(x, y); }
    static __device__ __forceinline__ V sum(V x, V y) { return df_add(x, y); }
    static __device__ __forceinline__ V shfl_xor(V x, int o)
    {
        return df{__shfl_xor_sync(kFull, x.h, o), __shfl_xor_sync(kFull, x.l, o)};
    }
    static __device__ __forceinline__ V mul(V x, V y) { return df_mul(x, y); }
    static __device__ __forceinline__ V from_u(double x) { return df_split_z(x); }
    static __device__ __forceinline__ V from_pair(float2 v) { return df{v.x, v.y}; }
    static __device__ __forceinline__ double to_double(V v)
    {
        df r;
        two_sum(v.h, v.l, r.h, r.l);
        return df_to_double(r.h, r.l);
    }
};
template <> struct SArith<false> {
    using V = float;
    struct Acc {
        float s = 0.f;
    };
    static __device__ __forceinline__ void fma(Acc &a, V x, V y) { a.s = fmaf(x, y, a.s); }
    static __device__ __forceinline__ V val(const Acc &a) { return a.s; }
    static __device__ __forceinline__ V add(V x, V y) { return x + y; }
    static __device__ __forceinline__ V sum(V x, V y) { return x + y; }
    static __device__ __forceinline__ V shfl_xor(V x, int o) { return __shfl_xor_sync(kFull, x, o); }
    static __device__ __forceinline__ V mul(V x, V y) { return x * y; }
    // rounded to FP32 with integer operations (no FP64 conversion)
    static __device__ __forceinline__ V from_u(double x)
    {
        const df t = df_split_z(x);
        return __fadd_rn(t.h, t.l);
    }
    static __device__ __forceinline__ V from_pair(float2 v) { return v.x; }
    static __device__ __forceinline__ double to_double(V v) { return (double)v; }
};

struct StrainArgs {
    int64_t nc;
    int nb, nq;
    const int32_t *__restrict__ cell_node;
    const double *__restrict__ u;
    const double *__restrict__ rho;
    SimpParams sp;
    const float2 *__restrict__ geo;   // [nc or 1][d*d + 1] G row-major, |det J|, as pairs
    int64_t geo_stride;               // d*d + 1, or 0 when every cell has the same Jacobian
    const float2 *__restrict__ qw;    // [nq] weights
    const float2 *__restrict__ qd;    // [nq][nb][d] reference gradients
    float2 lam, mu;                   // Lame constants at E = 1, as pairs
    const double *__restrict__ gscale;
    double *__restrict__ out;
    double *__restrict__ partial;
    unsigned *__restrict__ counter;
    double *__restrict__ c;
};

// One thread per cell; the cell's displacements are staged in shared memory
// ([nb * d][blockDim.x], one column per thread).  blockDim.x is a power of two
// <= 256 (the grid sum of c).
// NBT = the cell's node count, so the staging loads of a cell issue together,
// or 0 for any count (runtime loops).
template <int D, bool PAIR, int NBT>
__global__ void __launch_bounds__(128) k_strain_energy(const StrainArgs A)
{
    using S = SArith<PAIR>;
    using V = typename S::V;
    extern __shared__ float2 ush2[];
    V *us = reinterpret_cast<V *>(ush2);
    const int T = blockDim.x, tid = threadIdx.x;
    const int nb = NBT ? NBT : A.nb, nq = A.nq;
    const double g = A.gscale ? *A.gscale : -1.0;
    const V lam = S::from_pair(A.lam), mu = S::from_pair(A.mu);
    double mine = 0.0;
    for (int64_t e0 = (int64_t)blockIdx.x * T; e0 < A.nc; e0 += (int64_t)gridDim.x * T) {
        const int64_t e = e0 + tid;
        if (e < A.nc) {
            if (NBT) {
                // every node id first, then every displacement: one round trip each
                int32_t nd[NBT ? NBT : 1];
#pragma unroll
                for (int bb = 0; bb < NBT; bb++) nd[bb] = __ldg(A.cell_node + e * NBT + bb);
                double uv[NBT ? NBT : 1][D];
#pragma unroll
                for (int bb = 0; bb < NBT; bb++)
#pragma unroll
                    for (int i = 0; i < D; i++) uv[bb][i] = __ldg(A.u + (int64_t)D * nd[bb] + i);
#pragma unroll
                for (int bb = 0; bb < NBT; bb++)
#pragma unroll
                    for (int i = 0; i < D; i++) us[(bb * D + i) * T + tid] = S::from_u(uv[bb][i]);
            } else {
                for (int bb = 0; bb < nb; bb++) {
                    const int64_t node = A.cell_node[e * nb + bb];
#pragma unroll
                    for (int i = 0; i < D; i++) us[(bb * D + i) * T + tid] = S::from_u(A.u[D * node + i]);
                }
            }
            V G[D * D], det;
            const float2 *gp = A.geo + e * A.geo_stride;
#pragma unroll
            for (int t = 0; t < D * D; t++) G[t] = S::from_pair(gp[t]);
            det = S::from_pair(gp[D * D]);
            typename S::Acc s;
            for (int q = 0; q < nq; q++) {
                typename S::Acc U[D][D];
                const float2 *dq = A.qd + (size_t)q * nb * D;
#pragma unroll 2
                for (int bb = 0; bb < nb; bb++) {
                    V ub[D], dp[D];
#pragma unroll
                    for (int i = 0; i < D; i++) ub[i] = us[(bb * D + i) * T + tid];
#pragma unroll
                    for (int m = 0; m < D; m++) dp[m] = S::from_pair(__ldg(dq + bb * D + m));
#pragma unroll
                    for (int i = 0; i < D; i++)
#pragma unroll
                        for (int m = 0; m < D; m++) S::fma(U[i][m], ub[i], dp[m]);
                }
                V Uv[D][D];
#pragma unroll
                for (int i = 0; i < D; i++)
#pragma unroll
                    for (int m = 0; m < D; m++) Uv[i][m] = S::val(U[i][m]);
                // grad u = U^ G: g_ij = sum_m U^_im G[m][j]
                V gu[D][D];
#pragma unroll
                for (int i = 0; i < D; i++)
#pragma unroll
                    for (int j = 0; j < D; j++) {
                        typename S::Acc a;
#pragma unroll
                        for (int m = 0; m < D; m++) S::fma(a, Uv[i][m], G[m * D + j]);
                        gu[i][j] = S::val(a);
                    }
                // lam (tr g)^2 + mu sum_ij g_ij (g_ij + g_ji)
                V tr = gu[0][0];
#pragma unroll
                for (int m = 1; m < D; m++) tr = S::add(tr, gu[m][m]);
                typename S::Acc sh;
#pragma unroll
                for (int i = 0; i < D; i++)
#pragma unroll
                    for (int j = 0; j < D; j++) S::fma(sh, gu[i][j], S::add(gu[i][j], gu[j][i]));
                typename S::Acc dens;
                S::fma(dens, lam, S::mul(tr, tr));
                S::fma(dens, mu, S::val(sh));
                S::fma(s, S::from_pair(__ldg(A.qw + q)), S::val(dens));
            }
            const double sd = S::to_double(S::mul(S::val(s), det));
            const double r = A.rho[e];
            A.out[e] = g * simp_dE(A.sp, r) * sd;
            mine += simp_E(A.sp, r) * sd;
        }
    }
    if (A.c) grid_sum_last_block(mine, A.partial, A.counter, A.c);
}

// The strain energy density at quadrature point q of a cell whose
// displacements are staged at us[(b d + i) * ustride] (reference gradients at
// the point dq[b][m], G row-major), times the point's weight.
template <int D, bool PAIR>
__device__ __forceinline__ typename SArith<PAIR>::V
point_energy(const StrainArgs &A, const typename SArith<PAIR>::V *us, int ustride, int q,
             const typename SArith<PAIR>::V *G, typename SArith<PAIR>::V lam, typename SArith<PAIR>::V mu)
{
    using S = SArith<PAIR>;
    using V = typename S::V;
    typename S::Acc U[D][D];
    const float2 *dq = A.qd + (size_t)q * A.nb * D;
    for (int bb = 0; bb < A.nb; bb++) {
        V ub[D], dp[D];
#pragma unroll
        for (int i = 0; i < D; i++) ub[i] = us[(bb * D + i) * ustride];
#pragma unroll
        for (int m = 0; m < D; m++) dp[m] = S::from_pair(__ldg(dq + bb * D + m));
#pragma unroll
        for (int i = 0; i < D; i++)
#pragma unroll
            for (int m = 0; m < D; m++) S::fma(U[i][m], ub[i], dp[m]);
    }
    V Uv[D][D];
#pragma unroll
    for (int i = 0; i < D; i++)
#pragma unroll
        for (int m = 0; m < D; m++) Uv[i][m] = S::val(U[i][m]);
    V gu[D][D];
#pragma unroll
    for (int i = 0; i < D; i++)
#pragma unroll
        for (int j = 0; j < D; j++) {
            typename S::Acc a;
#pragma unroll
            for (int m = 0; m < D; m++) S::fma(a, Uv[i][m], G[m * D + j]);
            gu[i][j] = S::val(a);
        }
    V tr = gu[0][0];
#pragma unroll
    for (int m = 1; m < D; m++) tr = S::add(tr, gu[m][m]);
    typename S::Acc sh;
#pragma unroll
    for (int i = 0; i < D; i++)
#pragma unroll
        for (int j = 0; j < D; j++) S::fma(sh, gu[i][j], S::add(gu[i][j], gu[j][i]));
    typename S::Acc dens;
    S::fma(dens, lam, S::mul(tr, tr));
    S::fma(dens, mu, S::val(sh));
    return S::mul(S::from_pair(__ldg(A.qw + q)), S::val(dens));
}

// The same sensitivities with a warp per cell, for cells with many nodes and
// points (nb nq >= 256: Q3 quadrilaterals, Q2/Q3 hexahedra, P3 tetrahedra),
// where one thread per cell leaves most of the GPU idle: the warp stages the
// cell's displacements in shared memory, each lane takes the points q = lane,
// lane + 32, ..., and a fixed-order butterfly sums the lanes' energies (the
// same bits on every lane).
template <int D, bool PAIR>
__global__ void __launch_bounds__(128) k_strain_energy_warp(const StrainArgs A)
{
    using S = SArith<PAIR>;
    using V = typename S::V;
    extern __shared__ float2 ush2[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int nb = A.nb, nv = nb * D;
    V *us = reinterpret_cast<V *>(ush2) + (size_t)warp * nv;
    const double g = A.gscale ? *A.gscale : -1.0;
    const V lam = S::from_pair(A.lam), mu = S::from_pair(A.mu);
    double mine = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * wpb + warp; e < A.nc; e += (int64_t)gridDim.x * wpb) {
        __syncwarp();
        for (int t = lane; t < nv; t += 32) {
            const int bb = t / D, i = t - D * bb;
            us[t] = S::from_u(A.u[(int64_t)D * A.cell_node[e * nb + bb] + i]);
        }
        __syncwarp();
        V G[D * D];
        const float2 *gp = A.geo + e * A.geo_stride;
#pragma unroll
        for (int t = 0; t < D * D; t++) G[t] = S::from_pair(gp[t]);
        const V det = S::from_pair(gp[D * D]);
        V sv = S::from_pair(make_float2(0.f, 0.f));
        for (int q = lane; q < A.nq; q += 32) sv = S::sum(sv, point_energy<D, PAIR>(A, us, 1, q, G, lam, mu));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sv = S::sum(sv, S::shfl_xor(sv, o));
        if (lane == 0) {
            const double sd = S::to_double(S::mul(sv, det));
            const double r = A.rho[e];
            A.out[e] = g * simp_dE(A.sp, r) * sd;
            mine += simp_E(A.sp, r) * sd;
        }
    }
    if (A.c) grid_sum_last_block(mine, A.partial, A.counter, A.c);
}

template <int D, int NB, int MINB>
cudaError_t contract_launch(const soptx_mesh_s &m, const double *rho, double *vals, cudaStream_t st)
{
    const auto &h = m.h;
    ContractArgs A;
    A.nn = h.nn;
    A.max_deg = h.max_deg;
    A.nrec = m.d.cnrec;
    A.ticket = m.d.cticket;
    A.inc_e = m.d.cinc_e;
    A.inc_a = m.d.cinc_a;
    A.rec = m.d.crec;
    A.cgeo = m.d.cgeo;
    A.Mf = m.d.Mf;
    A.Edf = m.d.Edf;
    A.rho = rho;
    A.sp = simp_params(m.mat);
    A.lam = (float)m.mat.lam;
    A.mu = (float)m.mat.mu;
    A.vals = vals;
    constexpr int NPW = 32 / NB;
    const size_t mbytes = (size_t)NB * NB * MPad<D>::n * sizeof(float);
    const size_t per_warp = (size_t)NPW * D * D * h.max_deg * sizeof(float2);
    // MINB CTAs must fit in the SM's 228 KiB of shared memory (1 KiB of it reserved per CTA)
    const size_t cta_smem = std::min<size_t>(200 * 1024, (228 * 1024) / MINB - 1024);
    if (cta_smem < mbytes + per_warp) return cudaErrorInvalidConfiguration;
    const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, (cta_smem - mbytes) / per_warp));
    const size_t smem = mbytes + per_warp * wpb;
    auto kern = k_contract_rows<D, NB, MINB>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    // persistent: the CTAs that fit at once, each warp taking many rounds
    int dev = 0, sms = 0, per_sm = 0;
    err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, wpb * 32, smem);
    if (err != cudaSuccess) return err;
    const int64_t groups = (h.nn + NPW - 1) / NPW;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((groups + wpb - 1) / wpb, (int64_t)sms * std::max(per_sm, 1)));
    // (as a dependent launch of the moduli kernel the separate call was 3% faster,
    // but in the one-call step its CTAs took the SMs the strain-energy kernel
    // beside it had been getting: slower steps)
    kern<<<grid, wpb * 32, smem, st>>>(A);
    return cudaGetLastError();
}

}  // namespace

// CTAs per SM each contraction layout is compiled for (its register cap).
static int contract_minb(int dim, int nb) { return dim == 2 ? 3 : (nb >= 20 ? 1 : 2); }

static bool contract_layout(int dim, int nb)
{
    if (dim == 2) return nb == 3 || nb == 4 || nb == 6 || nb == 9 || nb == 10 || nb == 16;
    return dim == 3 && (nb == 4 || nb == 8 || nb == 10 || nb == 20 || nb == 27);
}

// Whether the contraction serves this cell type: a compiled layout, and the
// reference integrals plus one warp's accumulators (at the largest node
// degree) fit in a CTA's share of shared memory.
bool contract_fits(int dim, int nb, int max_deg)
{
    // a lane record holds the column block in 9 bits and the local node in 5
    if (!contract_layout(dim, nb) || nb > 32 || max_deg > 512) return false;
    const size_t mbytes = (size_t)nb * nb * (dim == 3 ? 12 : 4) * sizeof(float);
    const size_t per_warp = (size_t)(32 / nb) * dim * dim * max_deg * sizeof(float2);
    const int minb = contract_minb(dim, nb);
    const size_t cta_smem = std::min<size_t>(200 * 1024, (228 * 1024) / minb - 1024);
    return mbytes + per_warp <= cta_smem;
}

// Element moduli as float pairs (k_prep of the gather), then the contraction.
cudaError_t launch_contract_assemble(const soptx_mesh_s &m, const double *rho, double *vals, cudaStream_t st)
{
    const auto &h = m.h;
    cudaError_t err = launch_prep(m, rho, nullptr, st);
    if (err != cudaSuccess) return err;
    if (h.nn == 0 || h.nnz == 0) return cudaSuccess;
    const int nb = h.nb;
#define SOPTX_CT(DD, NBB, MINB)                                     \
    if (h.dim == DD && nb == NBB) return contract_launch<DD, NBB, MINB>(m, rho, vals, st);
    SOPTX_CT(2, 3, 3) SOPTX_CT(2, 4, 3) SOPTX_CT(2, 6, 3) SOPTX_CT(2, 9, 3) SOPTX_CT(2, 10, 3) SOPTX_CT(2, 16, 3)
    SOPTX_CT(3, 4, 2) SOPTX_CT(3, 8, 2) SOPTX_CT(3, 10, 2) SOPTX_CT(3, 20, 1) SOPTX_CT(3, 27, 1)
#undef SOPTX_CT
    return cudaErrorInvalidValue;
}

cudaError_t launch_strain_sensitivity(const soptx_mesh_s &m, const double *rho, const double *u, double *out,
                                      double *c, const double *gscale, cudaStream_t st)
{
    const auto &h = m.h;
    if (h.nc == 0) return c ? cudaMemsetAsync(c, 0, sizeof(double), st) : cudaSuccess;
    StrainArgs A;
    A.nc = h.nc;
    A.nb = h.nb;
    A.nq = m.d.snq;
    A.cell_node = m.d.cell_node;
    A.u = u;
    A.rho = rho;
    A.sp = simp_params(m.mat);
    A.geo = m.d.sgeo;
    A.geo_stride = m.path == SOPTX_PATH_UNIFORM ? 0 : h.dim * h.dim + 1;
    A.qw = m.d.sq;
    A.qd = m.d.sq + m.d.snq;
    auto pair = [](double x) {
        const float hh = (float)x;
        return make_float2(hh, (float)(x - (double)hh));
    };
    A.lam = pair(m.mat.lam);
    A.mu = pair(m.mat.mu);
    A.gscale = gscale;
    A.out = out;
    A.partial = m.d.scratch;
    A.counter = m.d.counter;
    A.c = c;
    const bool f32 = m.prec == SOPTX_ELEM_FP32;
    const size_t vb = f32 ? sizeof(float) : sizeof(float2);
    if ((int64_t)h.nb * A.nq >= 256) {
        // a warp per cell: 4 warps per block, each staging one cell's displacements
        const size_t smem = (size_t)4 * h.nb * h.dim * vb;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((h.nc + 3) / 4, m.d.scratch_len));
        auto k = h.dim == 3 ? (f32 ? k_strain_energy_warp<3, false> : k_strain_energy_warp<3, true>)
                            : (f32 ? k_strain_energy_warp<2, false> : k_strain_energy_warp<2, true>);
        cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        k<<<grid, 128, smem, st>>>(A);
        return cudaGetLastError();
    }
    // threads per block: a power of two whose staging fits in 96 KiB
    int T = 128;
    while (T > 32 && (size_t)T * h.nb * h.dim * vb > 96 * 1024) T >>= 1;
    const size_t smem = (size_t)T * h.nb * h.dim * vb;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((h.nc + T - 1) / T, m.d.scratch_len));
    void (*k)(StrainArgs) = nullptr;
#define SOPTX_SE(DD, NBB)                                                                                     \
    if (h.dim == DD && (NBB == 0 || h.nb == NBB) && !k)                                                      \
        k = f32 ? k_strain_energy<DD, false, NBB> : k_strain_energy<DD, true, NBB>;
    SOPTX_SE(2, 3) SOPTX_SE(2, 4) SOPTX_SE(2, 6) SOPTX_SE(2, 9) SOPTX_SE(2, 10) SOPTX_SE(2, 0)
    SOPTX_SE(3, 4) SOPTX_SE(3, 8) SOPTX_SE(3, 10) SOPTX_SE(3, 0)
#undef SOPTX_SE
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k<<<grid, T, smem, st>>>(A);
    return cudaGetLastError();
}

}  // namespace soptx
