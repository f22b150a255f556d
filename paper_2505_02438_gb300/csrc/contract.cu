// General (non-lattice) meshes of affine cells: the element matrices formed in
// registers from the reference integrals and each cell's Jacobian, and the
// sensitivities from the strain energy at quadrature points.
//
//  k_contract_pairs : FP32 element matrices of 2D cells, never stored.  K is
//                    symmetric, so one lane serves a pair of nodes {a, b} (a
//                    first in the processing order, or b = a): it walks the
//                    cells that hold both, in ascending order, and for each
//                    forms the d x d block K_e^0[(a,.),(b,.)] by the fast
//                    assembly of Sec. 3.2.2: the reference integrals
//                    M^{kl}_{ab} = int d_k phi_a d_l phi_b (shared memory,
//                    FP32) contracted with the cell's G = J^-1 and |det J|,
//                        P_ij = |det J| sum_kl G_ki G_lj M^{kl}_{ab},
//                        K_ij = lam P_ij + mu P_ji + mu delta_ij tr P,
//                    and adds E_e K_ij into float-pair sums held in
//                    registers (FP64-accurate, no atomics, a fixed order).
//                    The block leaves as FP64 values into row block (a, b)
//                    and, transposed, into (b, a).  Each lane's pair, its
//                    cells and both destinations come from tables made at
//                    mesh creation; a warp's 32 pairs have about as many
//                    cells each.
//                    The same kernel reads the blocks instead for the cached
//                    FP64 element matrices of 2D affine cells (each record's
//                    block gathered into record order at mesh creation) and
//                    for the one FP64 matrix of a uniform mesh (boxes of order
//                    2 and 3; in 3D each node then assembles all of its own
//                    rows, no transposed writes).
//  k_contract_rows : the same blocks for 3D cells, with the rows of one node
//                    owned by a group of nb lanes (nb = basis functions per
//                    cell) that walks the node's incident cells as a chain
//                    fixed at mesh creation (each next cell shares as many of
//                    the lanes' current column nodes as possible); lane b takes
//                    the cell's local node b and adds E_e K into the rows'
//                    float-pair accumulators in shared memory, keeping them in
//                    registers while its column block continues into the next
//                    cell.  (The pair layout in 3D writes every transposed
//                    block as three scattered 24-byte row pieces; the L2 then
//                    writes partly filled sectors back and fetches them again.)
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

// The pair tables made at mesh creation.  Pairs come in tiles of 32, one per
// lane; tile t's records are toff[t] * 32 ... toff[t + 1] * 32 - 1, record k of
// lane l at toff[t] * 32 + 32 k + l (lanes with fewer cells than the tile's
// longest are padded with cell 0).  The pair arrays are padded to whole chunks
// of 8 tiles and toff by 16 entries past the last chunk.
struct PairArgs {
    int64_t ntiles;
    unsigned *__restrict__ ticket;       // [0] chunks handed out, [1] CTAs done (both zero between calls)
    const uint32_t *__restrict__ toff;   // first record of each tile / 32
    const uint32_t *__restrict__ ia;     // [32 ntiles] value index of block (a, b), divided by d
    const uint32_t *__restrict__ ib;     // value index of block (b, a) / d (equal to ia when b = a)
    const uint32_t *__restrict__ meta;   // cells (bits 0-9), row length of a's rows (10-20), of b's (21-31)
    const int32_t *__restrict__ re;      // per record: the cell
    const uint16_t *__restrict__ rm;     // per record: a_loc nb + b_loc (contraction), a_loc << 8 | b_loc (the others)
    const float4 *__restrict__ cgeo;
    const float *__restrict__ Mf;
    int nmf;                             // floats in Mf
    const float2 *__restrict__ Kc;       // FP64 element matrices as float pairs: the cache [nc][ldof][ldof]
                                         // or a uniform mesh's one matrix [ldof][ldof]
    int ldof;
    const float4 *__restrict__ blk;      // per record: its 2 x 2 block of Kc, two rows of two float pairs
    const float2 *__restrict__ Edf;
    const double *__restrict__ rho;
    SimpParams sp;
    float lam, mu;
    double *__restrict__ vals;
};

// The node-owner contraction of 3D cells (k_contract_rows).
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
    static_assert(D == 3, "the node-owner contraction serves 3D cells");
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
        // no zeroing: every block of the rows is met by some cell, and its first
        // meeting starts the sums from zero
        double *const out = A.vals + (int64_t)D * D * off;
        const int rowlen = D * deg, blk = D * rowlen;

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
                    if (cur.p & 0x4000) {
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
#pragma unroll
                    for (int i = 0; i < D; i++)
#pragma unroll
                        for (int j = 0; j < D; j++) accs[rbase[i] + j] = v[i][j];
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
        } else if (has) {
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

// Row i of a d x d block of FP64 values at o (row stride rl), and the block's
// transpose at ot (row stride rlt): a block row of two values is one 16-byte
// store when the destination is aligned.
template <int D>
__device__ __forceinline__ void store_block(double *o, int rl, double *ot, int rlt, bool both, bool al16,
                                            const double (&d)[D][D])
{
#pragma unroll
    for (int i = 0; i < D; i++) {
        double *r = o + (int64_t)i * rl;
        if (D == 2 && al16) {
            *reinterpret_cast<double2 *>(r) = make_double2(d[i][0], d[i][1]);
        } else {
#pragma unroll
            for (int j = 0; j < D; j++) r[j] = d[i][j];
        }
    }
    if (!both) return;
#pragma unroll
    for (int j = 0; j < D; j++) {
        double *r = ot + (int64_t)j * rlt;
        if (D == 2 && al16) {
            *reinterpret_cast<double2 *>(r) = make_double2(d[0][j], d[1][j]);
        } else {
#pragma unroll
            for (int i = 0; i < D; i++) r[i] = d[i][j];
        }
    }
}

// Plain-FP64 redo of one lane's pair (a modulus outside the float-pair range):
// the same FP32 blocks times E(rho_e) in FP64, summed in the same cell order.
template <int D>
__device__ __noinline__ void pair_fp64(const PairArgs &A, const float *Ms, int64_t rb, int cnt, uint32_t pa,
                                       uint32_t pb, uint32_t meta, bool al16)
{
    double acc[D][D];
#pragma unroll
    for (int i = 0; i < D; i++)
#pragma unroll
        for (int j = 0; j < D; j++) acc[i][j] = 0.0;
    for (int k = 0; k < cnt; k++) {
        const int64_t r = rb + (int64_t)k * 32;
        const int32_t e = A.re[r];
        float G[D * D], det, M[D * D], K[D][D];
        load_cgeo<D>(A.cgeo, e, G, det);
        load_mpair<D>(Ms, A.rm[r], M);
        contract_block<D>(M, G, det, A.lam, A.mu, K);
        const double E = simp_E(A.sp, A.rho[e]);
#pragma unroll
        for (int i = 0; i < D; i++)
#pragma unroll
            for (int j = 0; j < D; j++) acc[i][j] += E * (double)K[i][j];
    }
    store_block<D>(A.vals + (int64_t)D * pa, (int)((meta >> 10) & 2047u), A.vals + (int64_t)D * pb,
                   (int)(meta >> 21), pa != pb, al16, acc);
}

// The same redo over cached FP64 element matrices (float pairs, 2D).
__device__ __noinline__ void pair_fp64_cached(const PairArgs &A, int64_t rb, int cnt, uint32_t pa, uint32_t pb,
                                              uint32_t meta, bool al16)
{
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int k = 0; k < cnt; k++) {
        const int64_t r = rb + (int64_t)k * 32;
        const int32_t e = A.re[r];
        const int m = A.rm[r];
        const double E = simp_E(A.sp, A.rho[e]);
        const float2 *kb = A.Kc + (int64_t)e * A.ldof * A.ldof + (int64_t)(2 * (m >> 8)) * A.ldof + 2 * (m & 255);
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int j = 0; j < 2; j++) {
                const float2 kk = kb[i * A.ldof + j];
                acc[i][j] += E * ((double)kk.x + (double)kk.y);
            }
    }
    store_block<2>(A.vals + (int64_t)2 * pa, (int)((meta >> 10) & 2047u), A.vals + (int64_t)2 * pb,
                   (int)(meta >> 21), pa != pb, al16, acc);
}

// The same redo over the one element matrix of a uniform mesh (float pairs).
template <int D>
__device__ __noinline__ void pair_fp64_unif(const PairArgs &A, int64_t rb, int cnt, uint32_t pa, uint32_t pb,
                                            uint32_t meta, bool al16)
{
    double acc[D][D];
#pragma unroll
    for (int i = 0; i < D; i++)
#pragma unroll
        for (int j = 0; j < D; j++) acc[i][j] = 0.0;
    for (int k = 0; k < cnt; k++) {
        const int64_t r = rb + (int64_t)k * 32;
        const int32_t e = A.re[r];
        const int m = A.rm[r];
        const double E = simp_E(A.sp, A.rho[e]);
        const float2 *kb = A.Kc + (int64_t)(D * (m >> 8)) * A.ldof + D * (m & 255);
#pragma unroll
        for (int i = 0; i < D; i++)
#pragma unroll
            for (int j = 0; j < D; j++) {
                const float2 kk = kb[i * A.ldof + j];
                acc[i][j] += E * ((double)kk.x + (double)kk.y);
            }
    }
    store_block<D>(A.vals + (int64_t)D * pa, (int)((meta >> 10) & 2047u), A.vals + (int64_t)D * pb,
                   (int)(meta >> 21), pa != pb, al16, acc);
}

// Asynchronous 16-byte copies global -> shared (cp.async); the waits are the
// hardware's (cp.async.wait_group), no polling.
__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// A chunk is kChunkTiles consecutive tiles, one per warp of a CTA.  Its tables
// are staged in shared memory: the tiles' record offsets, the lanes' pairs, and
// the chunk's first kChunkRecs records (a tile's records past those are read
// from global memory).
constexpr int kChunkTiles = 8;
constexpr int kChunkRecs = 2048;
struct ChunkBuf {
    uint32_t toff[16];
    uint32_t meta[kChunkTiles * 32], pa[kChunkTiles * 32], pb[kChunkTiles * 32];
    int32_t re[kChunkRecs];
    uint16_t rm[kChunkRecs];
};

// A persistent grid (the CTAs that fit); each CTA takes chunks in increasing
// order from a counter, so at any time the GPU works through a contiguous range
// of tiles and the two destinations of a pair's block meet in L2.  The next
// chunk's tables are copied into the other buffer while this one is worked;
// within a tile the cell one position ahead is loaded while the current one is
// summed.  A record's block is formed by the contraction (FP32 element
// matrices), read from its place in record order (CACHED: the cached FP64
// matrices of 2D cells) or read through L1 from the one matrix of a uniform
// mesh (UNIF).
template <int D, bool CACHED, bool UNIF>
__global__ void __launch_bounds__(256, D == 2 ? 4 : 3) k_contract_pairs(const PairArgs A)
{
    static_assert(D == 2 || !CACHED, "cached blocks are read as whole float4s in 2D only");
    static_assert(!(CACHED && UNIF), "one source of element matrices");
    constexpr int G4 = CGeo<D>::n4;
    extern __shared__ float4 csm4[];
    ChunkBuf *bufs = reinterpret_cast<ChunkBuf *>(csm4);
    float *Ms = reinterpret_cast<float *>(bufs + 2);
    for (int t = threadIdx.x; t < A.nmf; t += blockDim.x) Ms[t] = A.Mf[t];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool al16 = (reinterpret_cast<uintptr_t>(A.vals) & 15u) == 0;
    const int64_t nchunks = (A.ntiles + kChunkTiles - 1) / kChunkTiles;
    // a chunk's first record / 32 and the next chunk's, loaded a chunk ahead of
    // their use
    auto bounds = [&](int64_t c, uint32_t &r0, uint32_t &r1) {
        r0 = r1 = 0u;
        if (c < nchunks) {
            r0 = __ldg(A.toff + c * kChunkTiles);
            r1 = __ldg(A.toff + min((c + 1) * kChunkTiles, A.ntiles));
        }
    };
    auto issue = [&](int64_t c, uint32_t r0, uint32_t r1, ChunkBuf &B) {
        const int64_t t0 = c * kChunkTiles;
        const int nrec = (int)min((r1 - r0) * 32u, (uint32_t)kChunkRecs);
        const int nre = nrec / 4, nrm = nrec / 8;   // 16-byte pieces
        const int64_t rbase = (int64_t)r0 * 32;
        for (int p = threadIdx.x; p < 4 + 3 * 64 + nre + nrm; p += blockDim.x) {
            if (p < 4) {
                cp_async16(B.toff + 4 * p, A.toff + t0 + 4 * p);
            } else if (p < 4 + 3 * 64) {
                const int q = p - 4, w = q >> 6, o = (q & 63) * 4;
                const uint32_t *src = (w == 0 ? A.meta : w == 1 ? A.ia : A.ib) + t0 * 32 + o;
                cp_async16((w == 0 ? B.meta : w == 1 ? B.pa : B.pb) + o, src);
            } else if (p < 4 + 3 * 64 + nre) {
                const int o = (p - 4 - 3 * 64) * 4;
                cp_async16(B.re + o, A.re + rbase + o);
            } else {
                const int o = (p - 4 - 3 * 64 - nre) * 8;
                cp_async16(B.rm + o, A.rm + rbase + o);
            }
        }
    };
    // a record's cell: its geometry (contraction) or its cached block
    // K_e^0[(a,.),(b,.)] (two rows of two float pairs), and its modulus
    struct Cell {
        float4 g[G4];
        float2 E;
    };
    auto fetch_geo = [&](int32_t e, Cell &c) {
        const float4 *gp = A.cgeo + (int64_t)G4 * e;
#pragma unroll
        for (int w = 0; w < G4; w++) c.g[w] = __ldg(gp + w);
        c.E = __ldg(A.Edf + e);
    };
    // the cached block of record r (the lanes of a warp read consecutive records)
    auto fetch_blk = [&](int64_t r, int32_t e, Cell &c) {
        c.g[0] = __ldcs(A.blk + 2 * r);
        c.g[1] = __ldcs(A.blk + 2 * r + 1);
        c.E = __ldg(A.Edf + e);
    };
    // chunks are taken from a counter, so a CTA that starts late beside another
    // kernel simply takes fewer; three ahead: the chunk being worked (c), the one
    // being copied (cn), the one whose bounds are loading (cnn), and the ticket
    // of the next in flight meanwhile
    __shared__ unsigned s_ticket;
    auto grab = [&]() -> int64_t {
        if (threadIdx.x == 0) s_ticket = atomicAdd(A.ticket, 1u);
        __syncthreads();
        const int64_t v = s_ticket;
        __syncthreads();
        return v;
    };
    int64_t c = grab(), cn = grab(), cnn = grab();
    int cur = 0;
    uint32_t a0, a1, b0, b1;
    bounds(c, a0, a1);
    bounds(cn, b0, b1);
    if (c < nchunks) issue(c, a0, a1, bufs[0]);
    cp_async_commit();
    while (c < nchunks) {
        if (cn < nchunks) issue(cn, b0, b1, bufs[cur ^ 1]);
        cp_async_commit();
        bounds(cnn, b0, b1);
        unsigned tk = 0u;
        if (threadIdx.x == 0) tk = atomicAdd(A.ticket, 1u);
        cp_async_wait_1();
        __syncthreads();
        const ChunkBuf &B = bufs[cur];
        const int64_t t = c * kChunkTiles + warp;
        if (t < A.ntiles) {
            const int ct = (int)(B.toff[warp + 1] - B.toff[warp]);
            const int rel = (int)(B.toff[warp] - B.toff[0]) * 32 + lane;
            const uint32_t meta = B.meta[warp * 32 + lane], pa = B.pa[warp * 32 + lane], pb = B.pb[warp * 32 + lane];
            const int cnt = (int)(meta & 1023u);
            const int64_t gbase = (int64_t)B.toff[0] * 32;
            auto rec = [&](int k, int32_t &e, int &m) {
                const int r = rel + min(k, ct - 1) * 32;
                if (r < kChunkRecs) {
                    e = B.re[r];
                    m = B.rm[r];
                } else {
                    e = __ldg(A.re + gbase + r);
                    m = __ldg(A.rm + gbase + r);
                }
            };
            int32_t e0, e1;
            int m0, m1;
            rec(0, e0, m0);
            rec(1, e1, m1);
            Cell c0;
            const int64_t rabs = gbase + rel;   // the lane's first record
            if constexpr (CACHED) {
                fetch_blk(rabs, e0, c0);
            } else if constexpr (UNIF) {
                c0.E = __ldg(A.Edf + e0);
            } else {
                fetch_geo(e0, c0);
            }
            float2 v[D][D];
            bool bad = false;
            // cell k in cur, cell k + 1 loaded into nxt meanwhile (the two swap roles,
            // so the loop copies no cell)
            Cell c1;
            auto step = [&](const Cell &cur, Cell &nxt, int k) {
                if constexpr (CACHED)
                    fetch_blk(rabs + (int64_t)min(k + 1, ct - 1) * 32, e1, nxt);
                else if constexpr (UNIF)
                    nxt.E = __ldg(A.Edf + e1);
                else
                    fetch_geo(e1, nxt);
                if constexpr (UNIF) {
                  if (k < cnt) {
                    bad |= isnan(cur.E.y);
                    // E K^0 (the mesh's one element matrix, read through L1) as an
                    // unnormalised pair product, entry by entry
                    const df E{cur.E.x, cur.E.y};
                    const float2 *kb = A.Kc + (int64_t)(D * (m0 >> 8)) * A.ldof + D * (m0 & 255);
#pragma unroll
                    for (int i = 0; i < D; i++)
#pragma unroll
                        for (int j = 0; j < D; j++) {
                            const float2 kk = __ldg(kb + i * A.ldof + j);
                            const df x = df_mul_raw(E, df{kk.x, kk.y});
                            if (k == 0) {
                                v[i][j] = make_float2(x.h, x.l);
                            } else {
                                acc_add(v[i][j].x, v[i][j].y, x);
                            }
                        }
                  }
                } else if constexpr (CACHED) {
                  if (k < cnt) {
                    bad |= isnan(cur.E.y);
                    // E K_e^0 as an unnormalised pair product, entry by entry
                    const df E{cur.E.x, cur.E.y};
                    const df Kb[2][2] = {{df{cur.g[0].x, cur.g[0].y}, df{cur.g[0].z, cur.g[0].w}},
                                         {df{cur.g[1].x, cur.g[1].y}, df{cur.g[1].z, cur.g[1].w}}};
#pragma unroll
                    for (int i = 0; i < D; i++)
#pragma unroll
                        for (int j = 0; j < D; j++) {
                            const df x = df_mul_raw(E, Kb[i & 1][j & 1]);
                            if (k == 0) {
                                v[i][j] = make_float2(x.h, x.l);
                            } else {
                                acc_add(v[i][j].x, v[i][j].y, x);
                            }
                        }
                  }
                } else if (k < cnt) {
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
                    float M[D * D], K[D][D];
                    load_mpair<D>(Ms, m0, M);
                    contract_block<D>(M, G, det, A.lam, A.mu, K);
#pragma unroll
                    for (int i = 0; i < D; i++)
#pragma unroll
                        for (int j = 0; j < D; j++) {
                            // E K as a pair: TwoProd of the head, the tail's product
                            const float kk = K[i][j];
                            const float ph = __fmul_rn(cur.E.x, kk);
                            const float pl = __fmaf_rn(cur.E.y, kk, __fmaf_rn(cur.E.x, kk, -ph));
                            if (k == 0) {
                                v[i][j] = make_float2(ph, pl);
                            } else {
                                acc_add(v[i][j].x, v[i][j].y, df{ph, pl});
                            }
                        }
                }
                m0 = m1;
                rec(k + 2, e1, m1);
            };
            for (int k = 0; k < ct; k += 2) {
                step(c0, c1, k);
                if (k + 1 < ct) step(c1, c0, k + 1);
            }
            // a lane whose pair met an out-of-range modulus redoes it in FP64
            if (__any_sync(kFull, bad) && bad) {
                if constexpr (CACHED) {
                    pair_fp64_cached(A, gbase + rel, cnt, pa, pb, meta, al16);
                } else if constexpr (UNIF) {
                    pair_fp64_unif<D>(A, gbase + rel, cnt, pa, pb, meta, al16);
                } else {
                    pair_fp64<D>(A, Ms, gbase + rel, cnt, pa, pb, meta, al16);
                }
            } else if (cnt > 0) {
                // the values leave as FP64: half the entries widened and added on the
                // FP64 pipe, half with integer operations only
                double d[D][D];
#pragma unroll
                for (int i = 0; i < D; i++)
#pragma unroll
                    for (int j = 0; j < D; j++) {
                        if (((i * D + j) & 1) == 0) {
                            d[i][j] = pair_to_double(v[i][j].x, v[i][j].y);
                        } else {
                            float hh, ll;
                            two_sum(v[i][j].x, v[i][j].y, hh, ll);
                            d[i][j] = df_to_double(hh, ll);
                        }
                    }
                store_block<D>(A.vals + (int64_t)D * pa, (int)((meta >> 10) & 2047u), A.vals + (int64_t)D * pb,
                               (int)(meta >> 21), pa != pb, al16, d);
            }
        }
        if (threadIdx.x == 0) s_ticket = tk;
        __syncthreads();
        c = cn;
        cn = cnn;
        cnn = s_ticket;
        cur ^= 1;
    }
    // the last CTA to finish sets the counter back to zero for the next call
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(A.ticket + 1, 1u) == gridDim.x - 1u) {
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

// The strain-energy density at one point from the reference displacement
// gradient Uv (Uv[i][m] = sum_b u_(b,i) d_m phi_b) and the cell's G.
template <int D, bool PAIR>
__device__ __forceinline__ typename SArith<PAIR>::V
density_from_grad(const typename SArith<PAIR>::V (&Uv)[D][D], const typename SArith<PAIR>::V *G,
                  typename SArith<PAIR>::V lam, typename SArith<PAIR>::V mu)
{
    using S = SArith<PAIR>;
    using V = typename S::V;
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
    return S::val(dens);
}

// Hexahedra of order K = 2, 3: the same sensitivities by sum factorisation.
// The basis is a tensor product of 1D Lagrange polynomials l_j on equispaced
// nodes and the rule a tensor product of n = K + 1 Gauss points, so
//   d_1 phi_b(q) = l'_(b1)(q1) l_(b2)(q2) l_(b3)(q3)   (and so on),
// and the reference displacement gradient at all n^3 points is three passes of
// 1D contractions (8 n^4 multiply-adds per component instead of 3 n^6): a warp
// per cell, the cell's displacements staged in lattice order in shared memory,
// then each pass with the lanes over its n^3 outputs, and the last one over the
// points, which also form the energy density.  sf holds the 1D Gauss weights
// [n], l_j(t_q) [n][n] and l'_j(t_q) [n][n], and each local node's lattice
// index [n^3], as pairs.
template <int K, bool PAIR>
__global__ void __launch_bounds__(128) k_strain_hex_sf(const StrainArgs A, const float2 *__restrict__ sf)
{
    using S = SArith<PAIR>;
    using V = typename S::V;
    constexpr int D = 3, n = K + 1, n2 = n * n, n3 = n2 * n;
    extern __shared__ float2 ush2[];
    __shared__ V s_lv[n2], s_ld[n2], s_w[n];
    __shared__ int s_lat[n3];
    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        s_lv[t] = S::from_pair(sf[n + t]);
        s_ld[t] = S::from_pair(sf[n + n2 + t]);
    }
    for (int t = threadIdx.x; t < n; t += blockDim.x) s_w[t] = S::from_pair(sf[t]);
    for (int t = threadIdx.x; t < n3; t += blockDim.x) s_lat[t] = (int)sf[n + 2 * n2 + t].x;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    V *us = reinterpret_cast<V *>(ush2) + (size_t)warp * 6 * D * n3;   // [D][n3] in lattice order
    V *av = us + D * n3, *ad = av + D * n3, *bvv = ad + D * n3, *bvd = bvv + D * n3, *bdv = bvd + D * n3;
    const double g = A.gscale ? *A.gscale : -1.0;
    const V lam = S::from_pair(A.lam), mu = S::from_pair(A.mu);
    double mine = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * wpb + warp; e < A.nc; e += (int64_t)gridDim.x * wpb) {
        __syncwarp();
        for (int t = lane; t < n3 * D; t += 32) {
            const int b = t / D, i = t - D * b;
            us[i * n3 + s_lat[b]] = S::from_u(A.u[(int64_t)D * A.cell_node[e * n3 + b] + i]);
        }
        __syncwarp();
        // first index: av, ad[i][q1 + n b2 + n2 b3] = sum_b1 l, l'_(b1)(q1) u[i][b1 + n b2 + n2 b3]
        for (int o = lane; o < D * n3; o += 32) {
            const int i = o / n3, r = o - i * n3, q1 = r % n;
            const V *pu = us + i * n3 + (r - q1);
            typename S::Acc sv, sd;
#pragma unroll
            for (int b1 = 0; b1 < n; b1++) {
                S::fma(sv, s_lv[q1 * n + b1], pu[b1]);
                S::fma(sd, s_ld[q1 * n + b1], pu[b1]);
            }
            av[o] = S::val(sv);
            ad[o] = S::val(sd);
        }
        __syncwarp();
        // second index: [i][q1 + n q2 + n2 b3]
        for (int o = lane; o < D * n3; o += 32) {
            const int i = o / n3, r = o - i * n3, q1 = r % n, q2 = (r / n) % n, b3 = r / n2;
            const V *pa = av + i * n3 + q1 + n2 * b3, *pd = ad + i * n3 + q1 + n2 * b3;
            typename S::Acc vv, vd, dv;
#pragma unroll
            for (int b2 = 0; b2 < n; b2++) {
                S::fma(vv, s_lv[q2 * n + b2], pa[n * b2]);
                S::fma(vd, s_ld[q2 * n + b2], pa[n * b2]);
                S::fma(dv, s_lv[q2 * n + b2], pd[n * b2]);
            }
            bvv[o] = S::val(vv);
            bvd[o] = S::val(vd);
            bdv[o] = S::val(dv);
        }
        __syncwarp();
        V G[D * D];
        const float2 *gp = A.geo + e * A.geo_stride;
#pragma unroll
        for (int t = 0; t < D * D; t++) G[t] = S::from_pair(gp[t]);
        const V det = S::from_pair(gp[D * D]);
        // third index at each point q1 + n q2 + n2 q3, and the density there
        V sv = S::from_pair(make_float2(0.f, 0.f));
        for (int p = lane; p < n3; p += 32) {
            const int q1 = p % n, q2 = (p / n) % n, q3 = p / n2;
            V Uv[D][D];
#pragma unroll
            for (int i = 0; i < D; i++) {
                typename S::Acc d1, d2, d3;
                const int bi = i * n3 + q1 + n * q2;
#pragma unroll
                for (int b3 = 0; b3 < n; b3++) {
                    S::fma(d1, s_lv[q3 * n + b3], bdv[bi + n2 * b3]);
                    S::fma(d2, s_lv[q3 * n + b3], bvd[bi + n2 * b3]);
                    S::fma(d3, s_ld[q3 * n + b3], bvv[bi + n2 * b3]);
                }
                Uv[i][0] = S::val(d1);
                Uv[i][1] = S::val(d2);
                Uv[i][2] = S::val(d3);
            }
            const V w = S::mul(S::mul(s_w[q1], s_w[q2]), s_w[q3]);
            sv = S::sum(sv, S::mul(w, density_from_grad<D, PAIR>(Uv, G, lam, mu)));
        }
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

template <int D, bool CACHED, bool UNIF>
cudaError_t pairs_launch(const soptx_mesh_s &m, const double *rho, double *vals, cudaStream_t st)
{
    const auto &h = m.h;
    PairArgs A;
    A.ntiles = m.d.ptiles;
    A.ticket = m.d.cticket;
    A.toff = m.d.ptoff;
    A.ia = m.d.pia;
    A.ib = m.d.pib;
    A.meta = m.d.pmeta;
    A.re = m.d.pre;
    A.rm = m.d.prm;
    A.cgeo = m.d.cgeo;
    A.Mf = m.d.Mf;
    A.nmf = CACHED || UNIF ? 0 : h.nb * h.nb * MPad<D>::n;
    A.Kc = CACHED || UNIF ? static_cast<const float2 *>(m.d.K) : nullptr;
    A.ldof = h.ldof;
    A.blk = CACHED ? m.d.pblk : nullptr;
    A.Edf = m.d.Edf;
    A.rho = rho;
    A.sp = simp_params(m.mat);
    A.lam = (float)m.mat.lam;
    A.mu = (float)m.mat.mu;
    A.vals = vals;
    const size_t smem = 2 * sizeof(ChunkBuf) + (size_t)A.nmf * sizeof(float);
    auto kern = k_contract_pairs<D, CACHED, UNIF>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    // the CTAs that fit at once, each taking chunks from the counter
    int dev = 0, sms = 0, per_sm = 0;
    err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
    if (err != cudaSuccess) return err;
    const int64_t nchunks = (A.ntiles + kChunkTiles - 1) / kChunkTiles;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nchunks, (int64_t)sms * std::max(per_sm, 1)));
    kern<<<grid, 256, smem, st>>>(A);
    return cudaGetLastError();
}

template <int D, int NB, int MINB>
cudaError_t rows_launch(const soptx_mesh_s &m, const double *rho, double *vals, cudaStream_t st)
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

// CTAs per SM each node-owner layout (3D) is compiled for (its register cap).
static int rows_minb(int nb) { return nb >= 20 ? 1 : 2; }

// Whether the contraction serves this cell type.  2D (the pair kernel): the
// reference integrals fit in shared memory and a node's block row, twice its
// degree, fits the tables' 11 bits.  3D (the node-owner kernel): a compiled
// layout, and the reference integrals plus one warp's row accumulators (at the
// largest node degree) fit in a CTA's share of shared memory.
bool contract_fits(int dim, int nb, int max_deg)
{
    if (dim == 2) return nb <= 16 && 2 * max_deg <= 2047;
    // a lane record holds the column block in 9 bits and the local node in 5
    if (dim != 3 || !(nb == 4 || nb == 8 || nb == 10 || nb == 20 || nb == 27) || max_deg > 512) return false;
    const size_t mbytes = (size_t)nb * nb * 12 * sizeof(float);
    const size_t per_warp = (size_t)(32 / nb) * 9 * max_deg * sizeof(float2);
    const size_t cta_smem = std::min<size_t>(200 * 1024, (228 * 1024) / rows_minb(nb) - 1024);
    return mbytes + per_warp <= cta_smem;
}

// At mesh creation: each pair record's 2 x 2 block of the cached FP64 element
// matrices, in record order.
__global__ void k_pair_blocks(int64_t nrec, const int32_t *__restrict__ re, const uint16_t *__restrict__ rm,
                              const float2 *__restrict__ Kc, int ldof, float4 *__restrict__ blk)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrec; r += (int64_t)gridDim.x * blockDim.x) {
        const int m = rm[r];
        const float2 *kb = Kc + (int64_t)re[r] * ldof * ldof + (int64_t)(2 * (m >> 8)) * ldof + 2 * (m & 255);
        blk[2 * r] = *reinterpret_cast<const float4 *>(kb);
        blk[2 * r + 1] = *reinterpret_cast<const float4 *>(kb + ldof);
    }
}

cudaError_t launch_pair_blocks(const soptx_mesh_s &m, int64_t nrec, cudaStream_t st)
{
    if (nrec == 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>((nrec + 255) / 256, 152 * 16);
    k_pair_blocks<<<grid, 256, 0, st>>>(nrec, m.d.pre, m.d.prm, static_cast<const float2 *>(m.d.K), m.h.ldof,
                                        m.d.pblk);
    return cudaGetLastError();
}

// Whether the pair kernel can read a uniform or cached mesh's element matrices:
// local indices in 8 bits each, a block row (d times the degree) in 11 bits.
bool pairs_fit(int dim, int nb, int max_deg)
{
    return (dim == 2 || dim == 3) && nb <= 255 && (int64_t)dim * max_deg <= 2047;
}

// Element moduli as float pairs (k_prep of the gather), then the contraction (or,
// for the cached FP64 element matrices of 2D meshes, the pair kernel reading them).
cudaError_t launch_contract_assemble(const soptx_mesh_s &m, const double *rho, double *vals, cudaStream_t st)
{
    const auto &h = m.h;
    cudaError_t err = launch_prep(m, rho, nullptr, st);
    if (err != cudaSuccess) return err;
    if (m.d.puniform) {
        if (m.d.ptiles == 0) return cudaSuccess;
        return h.dim == 3 ? pairs_launch<3, false, true>(m, rho, vals, st)
                          : pairs_launch<2, false, true>(m, rho, vals, st);
    }
    if (h.dim == 2) {
        if (m.d.ptiles == 0) return cudaSuccess;
        return m.d.pcached ? pairs_launch<2, true, false>(m, rho, vals, st)
                           : pairs_launch<2, false, false>(m, rho, vals, st);
    }
    if (h.nn == 0 || h.nnz == 0) return cudaSuccess;
#define SOPTX_CT(NBB, MINB)                                     \
    if (h.nb == NBB) return rows_launch<3, NBB, MINB>(m, rho, vals, st);
    SOPTX_CT(4, 2) SOPTX_CT(8, 2) SOPTX_CT(10, 2) SOPTX_CT(20, 1) SOPTX_CT(27, 1)
#undef SOPTX_CT
    return cudaErrorInvalidValue;
}

cudaError_t launch_strain_sensitivity(const soptx_mesh_s &m, const double *rho, const double *u, double *out,
                                      double *c, const double *gscale, cudaStream_t st, int max_grid)
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
    if (m.d.ssf && h.dim == 3 && (h.order == 2 || h.order == 3)) {
        // hexahedra of order 2, 3: sum factorisation, a warp per cell, 4 warps per block
        const size_t smem = (size_t)4 * 6 * 3 * h.nb * vb;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((h.nc + 3) / 4, m.d.scratch_len));
        auto k = h.order == 2 ? (f32 ? k_strain_hex_sf<2, false> : k_strain_hex_sf<2, true>)
                              : (f32 ? k_strain_hex_sf<3, false> : k_strain_hex_sf<3, true>);
        cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        k<<<(int)grid, 128, smem, st>>>(A, m.d.ssf);
        return cudaGetLastError();
    }
    if ((int64_t)h.nb * A.nq >= 256) {
        // a warp per cell: 4 warps per block, each staging one cell's displacements
        const size_t smem = (size_t)4 * h.nb * h.dim * vb;
        // (the cap is not applied here: four cells per block, a block per SM would
        // leave this kernel far behind the assembly beside it)
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((h.nc + 3) / 4, m.d.scratch_len));
        auto k = h.dim == 3 ? (f32 ? k_strain_energy_warp<3, false> : k_strain_energy_warp<3, true>)
                            : (f32 ? k_strain_energy_warp<2, false> : k_strain_energy_warp<2, true>);
        cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        k<<<(int)grid, 128, smem, st>>>(A);
        return cudaGetLastError();
    }
    // threads per block: a power of two whose staging fits in 96 KiB
    int T = 128;
    while (T > 32 && (size_t)T * h.nb * h.dim * vb > 96 * 1024) T >>= 1;
    const size_t smem = (size_t)T * h.nb * h.dim * vb;
    int64_t grid = std::max<int64_t>(1, std::min<int64_t>((h.nc + T - 1) / T, m.d.scratch_len));
    if (max_grid > 0) grid = std::min<int64_t>(grid, max_grid);
    void (*k)(StrainArgs) = nullptr;
#define SOPTX_SE(DD, NBB)                                                                                     \
    if (h.dim == DD && (NBB == 0 || h.nb == NBB) && !k)                                                      \
        k = f32 ? k_strain_energy<DD, false, NBB> : k_strain_energy<DD, true, NBB>;
    SOPTX_SE(2, 3) SOPTX_SE(2, 4) SOPTX_SE(2, 6) SOPTX_SE(2, 9) SOPTX_SE(2, 10) SOPTX_SE(2, 0)
    SOPTX_SE(3, 4) SOPTX_SE(3, 8) SOPTX_SE(3, 10) SOPTX_SE(3, 0)
#undef SOPTX_SE
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k<<<(int)grid, T, smem, st>>>(A);
    return cudaGetLastError();
}

}  // namespace soptx
