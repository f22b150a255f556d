// Assembly on an order-1 box lattice (Q1 quads / hexes on a structured grid
// of identical axis-aligned boxes), FP64-accurate on the FP32 pipes.
//
// For node n and a neighbour m = n + delta, the cells shared by n and m are
// the 2^z cells around n on the side(s) delta selects (z = number of zero
// components of delta).  A box is symmetric under the reflection across its
// mid-plane normal to axis k, which swaps the corners along k and flips the
// k-th displacement component, so every shared cell contributes the SAME
// unit-modulus block entry up to a sign:
//     K[(n,i),(m,j)] = kappa_delta[i][j] * sum_{cells c} sigma_c(i,j) E(rho_c),
// with kappa_delta the block of the cell on the high side of n along the
// zero axes and sigma_c = -1 exactly when c lies on the low side along an odd
// number of zero axes that belong to {i, j} (i != j).  The signed sums are
// separable per axis (low L, high H, H+L, H-L), so all 4^d of them come from
// the 2^d moduli around n in d stages of one float-float add per lane.
//
// In 3D each warp takes two consecutive nodes at a time, one lane per
// neighbour offset delta, and hands their 2 d rows (contiguous CSR values) to
// the copy engine; in 2D a warp owns three nodes and stores them coalesced.  The element moduli arrive from k_simp_df
// as float pairs; a node touching a modulus outside [2^-60, 2^60] (flagged by
// a NaN low word) is done in plain FP64 instead: in 2D by its warp at once, in
// 3D by k_simp_df before the assembly (whose warps then skip the node), which
// keeps the rare path out of the assembly kernel's registers.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "df64.cuh"
#include "internal.h"
#include "kernels_common.cuh"

namespace soptx {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ df shfl_df(df v, int src)
{
    return df{__shfl_sync(kFull, v.h, src), __shfl_sync(kFull, v.l, src)};
}

// x with its sign bit flipped when bit 31 of `mask` is set (an integer XOR on
// the high word, no FP64 instruction).
__device__ __forceinline__ double flip_sign(double x, uint32_t mask)
{
    return __hiloint2double(__double2hiint(x) ^ (int)mask, __double2loint(x));
}

// Bulk shared -> global copies by the copy engine (cp.async.bulk, no tensor
// map): both addresses 16-byte aligned, size a multiple of 16.  A warp
// stages a node's rows in shared memory and one lane hands them to the copy
// engine, so the stores do not queue behind the warps' shared-memory and
// shuffle traffic in the load/store unit.
__device__ __forceinline__ void bulk_store(double *gdst, const double *ssrc, uint32_t bytes)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(ssrc);
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(s), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until no committed group is still reading its shared source
__device__ __forceinline__ void bulk_wait_read_0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// wait until every committed group has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// order this thread's generic-proxy shared-memory writes before later async-proxy reads
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// o: 0 -> L, 1 -> H, 2 -> H + L, 3 -> H - L.  `lsel` = (o == 0) and
// `coef` = 0, 1 or -1 (the factor on L) are per-lane constants.
__device__ __forceinline__ df combine(bool lsel, float coef, df L, df H)
{
    const df lhs = lsel ? L : H;
    return df_add(lhs, df{__fmul_rn(coef, L.h), __fmul_rn(coef, L.l)});
}
// The same without the final renormalisation, for the stages whose output
// feeds further float-pair sums.
__device__ __forceinline__ df combine_lazy(bool lsel, float coef, df L, df H)
{
    const df lhs = lsel ? L : H;
    return df_add_lazy(lhs, df{__fmul_rn(coef, L.h), __fmul_rn(coef, L.l)});
}
__device__ __forceinline__ float opt_coef(int o) { return o == 2 ? 1.f : (o == 3 ? -1.f : 0.f); }

__device__ __forceinline__ int axis_opt(int delta, bool in_class)
{
    return delta < 0 ? 0 : (delta > 0 ? 1 : (in_class ? 3 : 2));
}

// Plain-FP64 version of one node's rows (used for out-of-range moduli).
template <int D>
__device__ __forceinline__ void lattice_node_fp64_body(int nx, int ny, int nz, int ix, int iy, int iz, int dl,
                                                       bool valid, int mi, int rowlen, double *base,
                                                       const double *__restrict__ K0, const double *__restrict__ rho,
                                                       const SimpParams &sp)
{
    if (!valid) return;
    const int N[3] = {nx, ny, nz}, idx[3] = {ix, iy, iz};
    const int delta[3] = {dl % 3 - 1, (dl / 3) % 3 - 1, dl / 9 - 1};
    const int ldof = D * (1 << D);
    for (int i = 0; i < D; i++)
        for (int j = 0; j < D; j++) {
            double acc = 0.0;
            for (int c = 0; c < (1 << D); c++) {      // ascending cell order
                int a = 0, b = 0, eidx = 0, stride = 1;
                bool ok = true;
                for (int m = 0; m < D; m++) {
                    const int cm = (c >> m) & 1;
                    const int am = 1 - cm, bm = am + delta[m];
                    const int em = idx[m] - 1 + cm;
                    if (bm < 0 || bm > 1 || em < 0 || em >= N[m]) ok = false;
                    a |= am << m;
                    b |= bm << m;
                    eidx += em * stride;
                    stride *= N[m];
                }
                if (!ok) continue;
                acc += simp_E(sp, rho[eidx]) * K0[(D * a + i) * ldof + D * b + j];
            }
            base[i * rowlen + D * mi + j] = acc;
        }
}
template <int D>
__device__ __noinline__ void lattice_node_fp64(int nx, int ny, int nz, int ix, int iy, int iz, int dl, bool valid,
                                               int mi, int rowlen, double *base, const double *__restrict__ K0,
                                               const double *__restrict__ rho, SimpParams sp)
{
    lattice_node_fp64_body<D>(nx, ny, nz, ix, iy, iz, dl, valid, mi, rowlen, base, K0, rho, sp);
}

// Node chunks per warp: at most kChunk consecutive nodes, so the lattice index
// is decoded once per chunk and then stepped; the next node's moduli are
// fetched before the current node is processed.
constexpr int kChunk = 16;
// Sign classes of a lane's 3 x 3 block: 0 = i == j, 1 = {0,1}, 2 = {0,2},
// 3 = {1,2}.  On a box the two entries of an off-diagonal class are equal or
// opposite: with the Q1 gradients of an axis-aligned box,
//     K[(a,i),(b,j)] = (lam s_ai s_bj + mu s_aj s_bi) f,
//     K[(a,j),(b,i)] = (lam s_aj s_bi + mu s_ai s_bj) f
// (s the signs of the corners along each axis, f the common integral), so
// kappa_delta[j][i] = +-kappa_delta[i][j] and both entries of a class share
// one product (the host checks this before the lattice path is taken).  The
// diagonal class and class {0,1} take one FP64 multiply per product on the
// otherwise idle FP64 pipe (4 of a lane's 6 products), classes {0,2} and
// {1,2} multiply in float pairs and convert each product.

// Row layout of node idx in the CSR values: whether the lane's offset delta is
// a neighbour (valid), its position mi among the node's neighbours and the
// length of each of the node's d rows.
__device__ __forceinline__ void node_layout3(const int idx[3], const int N[3], int dx, int dy, int dz, int lane,
                                             bool &valid, int &mi, int &rowlen)
{
    if (idx[0] > 0 && idx[0] < N[0] && idx[1] > 0 && idx[1] < N[1] && idx[2] > 0 && idx[2] < N[2]) {
        valid = lane < 27;
        mi = lane;
        rowlen = 81;
        return;
    }
    int lo[3], cnt[3];
    for (int m = 0; m < 3; m++) {
        lo[m] = idx[m] > 0 ? -1 : 0;
        cnt[m] = (idx[m] < N[m] ? 1 : 0) - lo[m] + 1;
    }
    valid = lane < 27 && dx >= lo[0] && dx < lo[0] + cnt[0] && dy >= lo[1] && dy < lo[1] + cnt[1] &&
            dz >= lo[2] && dz < lo[2] + cnt[2];
    mi = (dx - lo[0]) + cnt[0] * ((dy - lo[1]) + cnt[1] * (dz - lo[2]));
    rowlen = 3 * cnt[0] * cnt[1] * cnt[2];
}

// The same for a 2D node (lanes 0..8 are the offsets delta).
__device__ __forceinline__ void node_layout2(const int idx[2], int nx, int ny, int dx, int dy, bool lane_ok,
                                             bool &valid, int &mi, int &rowlen)
{
    const int lo0 = idx[0] > 0 ? -1 : 0, lo1 = idx[1] > 0 ? -1 : 0;
    const int c0 = (idx[0] < nx ? 1 : 0) - lo0 + 1, c1 = (idx[1] < ny ? 1 : 0) - lo1 + 1;
    valid = lane_ok && dx >= lo0 && dx < lo0 + c0 && dy >= lo1 && dy < lo1 + c1;
    mi = (dx - lo0) + c0 * (dy - lo1);
    rowlen = 2 * c0 * c1;
}

struct NodeIter {
    int idx[3];
    __device__ void decode(uint32_t n, int nx, int ny)
    {
        idx[0] = (int)(n % (uint32_t)(nx + 1));
        const uint32_t r = n / (uint32_t)(nx + 1);
        idx[1] = (int)(r % (uint32_t)(ny + 1));
        idx[2] = (int)(r / (uint32_t)(ny + 1));
    }
    __device__ void step(int nx, int ny)
    {
        if (++idx[0] > nx) {
            idx[0] = 0;
            if (++idx[1] > ny) {
                idx[1] = 0;
                ++idx[2];
            }
        }
    }
};

// Corner moduli of two nodes: lanes 0..7 those of node a, lanes 8..15 those of node b.
// NC: the moduli were written by an earlier launch (read-only path); otherwise by
// this kernel, before a barrier (coherent loads).
template <bool NC>
__device__ __forceinline__ float2 load_corner_pair(const float2 *__restrict__ Edf, const int ia[3], const int ib[3],
                                                   bool has_b, int lane, int nx, int ny, int nz)
{
    float2 v = make_float2(0.f, 0.f);
    const bool second = lane >= 8;
    if (lane < 8 || (lane < 16 && has_b)) {
        const int l = lane & 7;
        const int *idx = second ? ib : ia;
        const int ex = idx[0] - 1 + (l & 1), ey = idx[1] - 1 + ((l >> 1) & 1), ez = idx[2] - 1 + (l >> 2);
        if (ex >= 0 && ex < nx && ey >= 0 && ey < ny && ez >= 0 && ez < nz)
            v = NC ? __ldg(&Edf[((int64_t)ez * ny + ey) * nx + ex]) : __ldcg(&Edf[((int64_t)ez * ny + ey) * nx + ex]);
    }
    return v;
}

#ifndef SOPTX_LATTICE_MINBLOCKS
#define SOPTX_LATTICE_MINBLOCKS 4
#endif
// Element moduli as float pairs (and, with u given, u as float pairs).  With
// `flag` given, a warp
// whose cells include moduli outside the float-pair range (NaN low word)
// stores `gen` in *flag and writes the rows of the nodes around each such
// cell in plain FP64, lanes over the offsets; the assembly kernel then skips
// those nodes.  A node next to several such cells is written again with the
// same values.
#ifndef SOPTX_SIMP_MINB
#define SOPTX_SIMP_MINB 8
#endif
__device__ __forceinline__ void simp_df_body(int dim, int nx, int ny, int nz, int64_t nc, const double *__restrict__ rho,
                                             SimpParams sp, float2 *__restrict__ Edf,
                                             const int64_t *__restrict__ node_off, const double *__restrict__ K0,
                                             double *__restrict__ vals, unsigned *__restrict__ flag, unsigned gen,
                                             int64_t ndof, const double *__restrict__ u, float2 *__restrict__ udf,
                                             int64_t bid, int64_t nblk)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = nblk * blockDim.x;
    // with u given (one call doing both passes), u as float pairs for the sensitivity
    // kernel, two dofs per thread and pass (16-byte loads and stores when u allows)
    if (u) {
        const bool vec = ((reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(udf)) & 15u) == 0u;
        const int64_t npair = vec ? ndof / 2 : 0;
        for (int64_t r = bid * blockDim.x + threadIdx.x; r < npair; r += stride) {
            const double2 x = __ldcs(reinterpret_cast<const double2 *>(u) + r);
            const df a = df_split(x.x), b = df_split(x.y);
            reinterpret_cast<float4 *>(udf)[r] = make_float4(a.h, a.l, b.h, b.l);
        }
        for (int64_t r = 2 * npair + bid * blockDim.x + threadIdx.x; r < ndof; r += stride) {
            const df v = df_split(u[r]);
            udf[r] = make_float2(v.h, v.l);
        }
    }
    for (int64_t e0 = bid * blockDim.x + (threadIdx.x & ~31); e0 < nc; e0 += stride) {
        const int64_t e = e0 + lane;
        bool isbad = false;
        if (e < nc) {
            const float2 v = simp_E_pair(sp, rho[e]);
            Edf[e] = v;
            isbad = isnan(v.y);
        }
        if (!flag) continue;
        unsigned m = __ballot_sync(kFull, isbad);
        if (!m) continue;
        if (lane == 0) *flag = gen;
        if (dim == 2) {
            const int dl = lane < 9 ? lane : 8;
            const int dx = dl % 3 - 1, dy = dl / 3 - 1;
            while (m) {
                const unsigned k = __ffs(m) - 1;
                m &= m - 1u;
                const uint32_t ce = (uint32_t)(e0 + k);
                for (int corner = 0; corner < 4; corner++) {
                    const int idx[2] = {(int)(ce % (uint32_t)nx) + (corner & 1), (int)(ce / (uint32_t)nx) + (corner >> 1)};
                    const int64_t n = idx[0] + (int64_t)(nx + 1) * idx[1];
                    bool valid;
                    int mi, rowlen;
                    node_layout2(idx, nx, ny, dx, dy, lane < 9, valid, mi, rowlen);
                    lattice_node_fp64<2>(nx, ny, 1, idx[0], idx[1], 0, dl, valid, mi, rowlen, vals + 4 * node_off[n],
                                         K0, rho, sp);
                }
            }
            continue;
        }
        const int dl = lane < 27 ? lane : 26;
        const int dx = dl % 3 - 1, dy = (dl / 3) % 3 - 1, dz = dl / 9 - 1;
        const int N[3] = {nx, ny, nz};
        while (m) {
            const unsigned k = __ffs(m) - 1;
            m &= m - 1u;
            const uint32_t ce = (uint32_t)(e0 + k), r = ce / (uint32_t)nx;
            for (int corner = 0; corner < 8; corner++) {
                const int idx[3] = {(int)(ce % (uint32_t)nx) + (corner & 1), (int)(r % (uint32_t)ny) + ((corner >> 1) & 1),
                                    (int)(r / (uint32_t)ny) + (corner >> 2)};
                const int64_t n = idx[0] + (int64_t)(nx + 1) * (idx[1] + (int64_t)(ny + 1) * idx[2]);
                bool valid;
                int mi, rowlen;
                node_layout3(idx, N, dx, dy, dz, lane, valid, mi, rowlen);
                lattice_node_fp64<3>(nx, ny, nz, idx[0], idx[1], idx[2], dl, valid, mi, rowlen, vals + 9 * node_off[n],
                                     K0, rho, sp);
            }
        }
    }
}

__global__ void __launch_bounds__(256, SOPTX_SIMP_MINB)
k_simp_df(int dim, int nx, int ny, int nz, int64_t nc, const double *__restrict__ rho, SimpParams sp,
          float2 *__restrict__ Edf, const int64_t *__restrict__ node_off, const double *__restrict__ K0,
          double *__restrict__ vals, unsigned *__restrict__ flag, unsigned gen, int64_t ndof,
          const double *__restrict__ u, float2 *__restrict__ udf)
{
    grid_dep_launch();   // the assembly may be scheduled now; it waits for this kernel before reading
    simp_df_body(dim, nx, ny, nz, nc, rho, sp, Edf, node_off, K0, vals, flag, gen, ndof, u, udf, blockIdx.x, gridDim.x);
}

// 3D assembly, two nodes at a time (n, n+1 of a chunk): one corner load, one X
// stage and one hand-off to the copy engine serve both (their rows are
// contiguous in the CSR values); the Y and Z stages and the entries run once
// per node.  Each lane forms its 9 entries from 6 products (see the sign
// classes above): the diagonal class and class {0,1} convert T once and take
// one FP64 multiply per product, the other two multiply in float pairs and
// convert; the second entry of each off-diagonal class is the first with its
// sign bit flipped when the pair is opposite.  One
// staging buffer per warp holds both nodes' rows, each value at the 16-byte
// phase of its destination; before it is refilled the warp waits until the
// copy engine has read the previous pair (one node at a time with two
// buffers was 12% more instructions: 409 against 358 per node).
template <int WPB, bool NC>
__device__ __forceinline__ void lattice_assemble3_body(int nx, int ny, int nz, int64_t nn, int chunk,
                                                       const int64_t *__restrict__ node_off,
                                                       const float2 *__restrict__ Edf,
                                                       const float2 *__restrict__ kappa_g,
                                                       const double *__restrict__ K0, const double *__restrict__ rho,
                                                       SimpParams sp, double *__restrict__ vals,
                                                       const unsigned *__restrict__ flag, unsigned gen,
                                                       uint32_t pbias, double kscale, int64_t bid, int64_t nblk)
{
    const int lane = threadIdx.x & 31;
    const int dl = lane < 27 ? lane : 26;
    const int dx = dl % 3 - 1, dy = (dl / 3) % 3 - 1, dz = dl / 9 - 1;
    int tq[4];
    tq[0] = axis_opt(dx, false) + 4 * axis_opt(dy, false) + 16 * axis_opt(dz, false);   // i == j
    tq[1] = axis_opt(dx, true) + 4 * axis_opt(dy, true) + 16 * axis_opt(dz, false);     // {0, 1}
    tq[2] = axis_opt(dx, true) + 4 * axis_opt(dy, false) + 16 * axis_opt(dz, true);     // {0, 2}
    tq[3] = axis_opt(dx, false) + 4 * axis_opt(dy, true) + 16 * axis_opt(dz, true);     // {1, 2}
    __shared__ float2 kap_s[27 * 9];
    __shared__ double kapd_s[27 * 9];
    __shared__ __align__(16) double stage_s[WPB][2 * 27 * 9 + 2];
    __shared__ float2 tab_s[WPB][2][64];
    for (int t = threadIdx.x; t < 27 * 9; t += blockDim.x) {
        kap_s[t] = kappa_g[t];
        kapd_s[t] = ((double)kappa_g[t].x + (double)kappa_g[t].y) * kscale;
    }
    __syncthreads();
    // the sign of entry (j, i) relative to (i, j) for the classes {0,1}, {0,2}, {1,2}
    // (bit 31 of the high word of the FP64 value)
    uint32_t sflip[3];
    {
        const int ij[3][2] = {{0, 1}, {0, 2}, {1, 2}};
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const float a = kap_s[dl * 9 + ij[q][0] * 3 + ij[q][1]].x, b = kap_s[dl * 9 + ij[q][1] * 3 + ij[q][0]].x;
            sflip[q] = (__float_as_uint(a) ^ __float_as_uint(b)) & 0x80000000u;
        }
    }
    grid_dep_wait();
    grid_dep_launch();
    const int ox = lane & 3, oy = (lane >> 2) & 3;
    const int yzx = (lane >> 2) & 3;            // stage X: (cy, cz) of lanes 0..15 (and 16..31)
    const int xsrc = lane & 16 ? 8 : 0;         // stage X: lanes 16..31 take the second node's corners
    const int czy = (lane >> 4) & 1;            // stage Y: cz of lane
    const int oz0 = (lane < 16) ? 0 : 1, oz1 = oz0 + 2;
    const float cx_ = opt_coef(ox), cy_ = opt_coef(oy), cz0_ = opt_coef(oz0), cz1_ = opt_coef(oz1);
    const int N[3] = {nx, ny, nz};
    const bool anybad = __ldcg(flag) == gen;
    double *stage = stage_s[threadIdx.x >> 5];
    float2(*tab)[64] = tab_s[threadIdx.x >> 5];

    const int64_t nchunks = (nn + chunk - 1) / chunk;
    const int64_t warps = nblk * WPB;
    for (int64_t ch = bid * WPB + (threadIdx.x >> 5); ch < nchunks; ch += warps) {
        const int64_t n_begin = ch * chunk;
        const int64_t n_end = min(n_begin + (int64_t)chunk, nn);
        NodeIter ia;
        ia.decode((uint32_t)n_begin, nx, ny);
        NodeIter ib = ia;
        ib.step(nx, ny);
        float2 cur = load_corner_pair<NC>(Edf, ia.idx, ib.idx, n_begin + 1 < n_end, lane, nx, ny, nz);
        int64_t off = node_off[n_begin];
        for (int64_t n = n_begin; n < n_end; n += 2) {
            const bool has_b = n + 1 < n_end;
            const int idxa[3] = {ia.idx[0], ia.idx[1], ia.idx[2]};
            const int idxb[3] = {ib.idx[0], ib.idx[1], ib.idx[2]};
            // prefetch the next pair's corner moduli and CSR offset
            ia = ib;
            ia.step(nx, ny);
            ib = ia;
            ib.step(nx, ny);
            float2 nxt = make_float2(0.f, 0.f);
            int64_t off_next = 0;
            if (n + 2 < n_end) {
                nxt = load_corner_pair<NC>(Edf, ia.idx, ib.idx, n + 3 < n_end, lane, nx, ny, nz);
                off_next = node_off[n + 2];
            }
            const df Ec = df{cur.x, cur.y};
            unsigned bad_a = 0u, bad_b = 0u;
            if (anybad) {
                bad_a = __ballot_sync(kFull, lane < 8 && isnan(cur.y));
                bad_b = __ballot_sync(kFull, lane >= 8 && lane < 16 && isnan(cur.y));
            }
            bool valid_a, valid_b;
            int mi_a, mi_b, rl_a, rl_b;
            node_layout3(idxa, N, dx, dy, dz, lane, valid_a, mi_a, rl_a);
            node_layout3(idxb, N, dx, dy, dz, lane, valid_b, mi_b, rl_b);
            valid_b = valid_b && has_b;
            double *base = vals + 9 * off;
            // stage X for both nodes: lanes 0..15 node a, 16..31 node b -> (ox, cy, cz)
            const df xL = shfl_df(Ec, xsrc + 2 * yzx), xH = shfl_df(Ec, xsrc + 2 * yzx + 1);
            const df X = combine_lazy(ox == 0, cx_, xL, xH);
#pragma unroll
            for (int k = 0; k < 2; k++) {
                // stage Y: lanes 0..31 -> (ox, oy, cz) of node k
                const df yL = shfl_df(X, 16 * k + ox + 4 * (2 * czy)), yH = shfl_df(X, 16 * k + ox + 4 * (1 + 2 * czy));
                const df Y = combine_lazy(oy == 0, cy_, yL, yH);
                // stage Z: lane holds entries lane (A) and lane + 32 (B) of node k
                const df zL = shfl_df(Y, lane & 15), zH = shfl_df(Y, (lane & 15) + 16);
                const df A = combine(oz0 == 0, cz0_, zL, zH), B = combine(false, cz1_, zL, zH);
                tab[k][lane] = make_float2(A.h, A.l);
                tab[k][lane + 32] = make_float2(B.h, B.l);
            }
            // the buffer is free once the copy engine has read the previous pair
            if (lane == 0) bulk_wait_read_0();
            __syncwarp();
            const int ph = (int)((reinterpret_cast<uintptr_t>(base) >> 3) & 1);
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const bool valid = k ? valid_b : valid_a;
                const int mi = k ? mi_b : mi_a, rowlen = k ? rl_b : rl_a;
                double *st = stage + ph + (k ? 3 * rl_a : 0);
                if (valid) {
                    df T[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const float2 t = tab[k][tq[q]];
                        T[q] = df{t.x, t.y};
                    }
                    const double T0 = df_to_double_biased(T[0].h, T[0].l, 0x38000000u);
                    const double T1 = df_to_double_biased(T[1].h, T[1].l, 0x38000000u);
                    double *r0 = st + 3 * mi, *r1 = r0 + rowlen, *r2 = r1 + rowlen;
                    const double *kd = kapd_s + dl * 9;
                    r0[0] = kd[0] * T0;
                    r1[1] = kd[4] * T0;
                    r2[2] = kd[8] * T0;
                    const double v01 = kd[1] * T1;
                    r0[1] = v01;
                    r1[0] = flip_sign(v01, sflip[0]);
                    const float2 k02 = kap_s[dl * 9 + 2], k12 = kap_s[dl * 9 + 5];
                    const df p02 = df_mul_raw(df{k02.x, k02.y}, T[2]), p12 = df_mul_raw(df{k12.x, k12.y}, T[3]);
                    const double v02 = df_to_double_biased(p02.h, p02.l, pbias);
                    const double v12 = df_to_double_biased(p12.h, p12.l, pbias);
                    r0[2] = v02;
                    r2[0] = flip_sign(v02, sflip[1]);
                    r1[2] = v12;
                    r2[1] = flip_sign(v12, sflip[2]);
                }
            }
            fence_proxy_async_smem();
            __syncwarp();
            const int blk_a = 3 * rl_a, blk = blk_a + (has_b ? 3 * rl_b : 0);
            if (!bad_a && !bad_b) {
                // a value at an odd 8-byte phase at either end goes out by a plain store
                const int head = ph, mid = (blk - head) & ~1, tail = blk - head - mid;
                if (lane == 0 && mid > 0) {
                    bulk_store(base + head, stage + ph + head, (uint32_t)(8 * mid));
                    bulk_commit();
                }
                if (lane == 1 && head) __stcs(base, stage[ph]);
                if (lane == 2 && tail) __stcs(base + blk - 1, stage[ph + blk - 1]);
            } else {
                // a node next to an out-of-range modulus was written by k_simp_df: only
                // the other node's rows go out, by plain stores
                const int t0 = bad_a ? blk_a : 0, t1 = (bad_b || !has_b) ? blk_a : blk;
                for (int t = t0 + lane; t < t1; t += 32) __stcs(base + t, stage[ph + t]);
            }
            cur = nxt;
            off = off_next;
        }
    }
    if (lane == 0) bulk_wait_all();
}

template <int WPB>
__global__ void __launch_bounds__(WPB * 32, SOPTX_LATTICE_MINBLOCKS)
k_lattice_assemble3(int nx, int ny, int nz, int64_t nn, int chunk, const int64_t *__restrict__ node_off,
                    const float2 *__restrict__ Edf, const float2 *__restrict__ kappa_g,
                    const double *__restrict__ K0, const double *__restrict__ rho, SimpParams sp,
                    double *__restrict__ vals, const unsigned *__restrict__ flag, unsigned gen, uint32_t pbias,
                    double kscale)
{
    lattice_assemble3_body<WPB, true>(nx, ny, nz, nn, chunk, node_off, Edf, kappa_g, K0, rho, sp, vals, flag, gen,
                                      pbias, kscale, blockIdx.x, gridDim.x);
}

// 2D: a warp takes chunks of up to 48 consecutive nodes, three at a time, lanes
// 9g .. 9g+8 serving node g (one lane per offset delta).  Lanes 9g .. 9g+3 load
// node g's corner moduli, which reach its lanes by shuffles; each lane forms
// the diagonal-class and the {0,1}-class signed sums directly (one combine per
// axis and row), its two diagonal entries with one FP64 multiply each and its
// two others in float pairs (kappa pairs scaled as in 3D), stages the three
// nodes' rows (contiguous in the CSR values) and the warp stores them
// coalesced.  Nodes next to an out-of-range modulus were written by k_simp_df
// and are skipped.
// The corner moduli of the node of lane 9g + c (c < 4) at lattice index (ix, iy).
// NC: the moduli were written by an earlier launch (read-only path); otherwise
// by this kernel, before a barrier (coherent loads).
template <bool NC>
__device__ __forceinline__ float2 corner2(const float2 *__restrict__ Edf, int ix, int iy, int cl, bool live, int nx,
                                          int ny)
{
    float2 v = make_float2(0.f, 0.f);
    if (live && cl < 4) {
        const int ex = ix - 1 + (cl & 1), ey = iy - 1 + (cl >> 1);
        if (ex >= 0 && ex < nx && ey >= 0 && ey < ny)
            v = NC ? __ldg(&Edf[(int64_t)ey * nx + ex]) : __ldcg(&Edf[(int64_t)ey * nx + ex]);
    }
    return v;
}

template <int WPB, bool NC>
__device__ __forceinline__ void lattice_assemble2_body(int nx, int ny, int64_t nn, int chunk,
                                                       const int64_t *__restrict__ node_off,
                                                       const float2 *__restrict__ Edf,
                                                       const float2 *__restrict__ kappa_g, double *__restrict__ vals,
                                                       const unsigned *__restrict__ flag, unsigned gen, uint32_t pbias,
                                                       double kscale, int64_t bid, int64_t nblk)
{
    __shared__ double stage_s[WPB][3 * 9 * 4];   // three nodes' rows
    const int lane = threadIdx.x & 31;
    const int g = lane < 27 ? lane / 9 : 2;
    const int cl = lane < 27 ? lane - 9 * g : 8;
    const int dl = cl;
    const int dx = dl % 3 - 1, dy = dl / 3 - 1;
    // the lane's kappa: diagonal entries in FP64, the off-diagonal pair as one
    // (scaled) float pair: kappa[1][0] = +-kappa[0][1] on a box (see the sign
    // classes of the 3D kernel), so one product serves both entries
    const float2 k01 = kappa_g[dl * 4 + 1];
    const uint32_t sflip = (__float_as_uint(k01.x) ^ __float_as_uint(kappa_g[dl * 4 + 2].x)) & 0x80000000u;
    const double k00 = ((double)kappa_g[dl * 4].x + (double)kappa_g[dl * 4].y) * kscale;
    const double k11 = ((double)kappa_g[dl * 4 + 3].x + (double)kappa_g[dl * 4 + 3].y) * kscale;
    // axis options: the low cell (L), the high one (H), or both: H + L on the
    // diagonal class, H - L on the {0,1} class (axes with delta 0)
    const bool lx = dx < 0, ly = dy < 0;
    const float cdx = dx == 0 ? 1.f : 0.f, cdy = dy == 0 ? 1.f : 0.f;
    grid_dep_wait();
    grid_dep_launch();
    const bool anybad = __ldcg(flag) == gen;
    double *stage = stage_s[threadIdx.x >> 5];
    const int64_t nchunks = (nn + chunk - 1) / chunk;
    const int64_t warps = nblk * WPB;
    for (int64_t ch = bid * WPB + (threadIdx.x >> 5); ch < nchunks; ch += warps) {
        const int64_t nb = ch * chunk, ne = min(nb + (int64_t)chunk, nn);
        int ix = (int)((nb + g) % (nx + 1)), iy = (int)((nb + g) / (nx + 1));
        int64_t vbase = 4 * node_off[nb];
        // node g's corner moduli from lanes 9g .. 9g+3, fetched one pass ahead
        float2 vn = corner2<NC>(Edf, ix, iy, cl, lane < 27 && nb + g < ne, nx, ny);
        for (int64_t n0 = nb; n0 < ne; n0 += 3) {
            const int64_t n = n0 + g;
            const bool live = lane < 27 && n < ne;
            const float2 v = vn;
            const int idx[2] = {ix, iy};
            ix += 3;
            while (ix > nx) {
                ix -= nx + 1;
                iy++;
            }
            vn = corner2<NC>(Edf, ix, iy, cl, lane < 27 && n + 3 < ne, nx, ny);
            unsigned badm = 0u;
            if (anybad) badm = __ballot_sync(kFull, live && cl < 4 && isnan(v.y));
            df E[4];
#pragma unroll
            for (int c = 0; c < 4; c++) {
                E[c] = df{__shfl_sync(kFull, v.x, 9 * g + c), __shfl_sync(kFull, v.y, 9 * g + c)};
            }
            bool valid;
            int mi, rowlen;
            node_layout2(idx, nx, ny, dx, dy, live, valid, mi, rowlen);
            const int blk = live ? 2 * rowlen : 0;
            // offsets of the three nodes' blocks in the staged span
            const int b0 = __shfl_sync(kFull, blk, 0), b1 = __shfl_sync(kFull, blk, 9), b2 = __shfl_sync(kFull, blk, 18);
            const int sbase = g == 0 ? 0 : (g == 1 ? b0 : b0 + b1);
            const int span = b0 + b1 + b2;
            if (valid) {
                // along x in each row (cy = 0: cells 0, 1; cy = 1: cells 2, 3), then along y
                const df d0 = df_add(lx ? E[0] : E[1], df{cdx * E[0].h, cdx * E[0].l});
                const df d1 = df_add(lx ? E[2] : E[3], df{cdx * E[2].h, cdx * E[2].l});
                const df p0 = df_add(lx ? E[0] : E[1], df{-cdx * E[0].h, -cdx * E[0].l});
                const df p1 = df_add(lx ? E[2] : E[3], df{-cdx * E[2].h, -cdx * E[2].l});
                const df Td = df_add(ly ? d0 : d1, df{cdy * d0.h, cdy * d0.l});
                const df Tp = df_add(ly ? p0 : p1, df{-cdy * p0.h, -cdy * p0.l});
                const double tdd = df_to_double_biased(Td.h, Td.l, 0x38000000u);
                double *r0 = stage + sbase + 2 * mi, *r1 = r0 + rowlen;
                r0[0] = k00 * tdd;
                r1[1] = k11 * tdd;
                const df v01 = df_mul_raw(df{k01.x, k01.y}, Tp);
                const double o01 = df_to_double_biased(v01.h, v01.l, pbias);
                r0[1] = o01;
                r1[0] = flip_sign(o01, sflip);
            }
            __syncwarp();
            if (!badm) {
                for (int t = lane; t < span; t += 32) __stcs(vals + vbase + t, stage[t]);
            } else {
                // skip the rows of nodes whose corner lanes saw an out-of-range modulus
                for (int t = lane; t < span; t += 32) {
                    const int gg = t < b0 ? 0 : (t < b0 + b1 ? 1 : 2);
                    if (!(badm & (0xfu << (9 * gg)))) __stcs(vals + vbase + t, stage[t]);
                }
            }
            __syncwarp();
            vbase += span;
        }
    }
}

template <int WPB>
__global__ void __launch_bounds__(WPB * 32)
k_lattice_assemble2(int nx, int ny, int64_t nn, int chunk, const int64_t *__restrict__ node_off,
                    const float2 *__restrict__ Edf, const float2 *__restrict__ kappa_g,
                    double *__restrict__ vals, const unsigned *__restrict__ flag, unsigned gen, uint32_t pbias,
                    double kscale)
{
    lattice_assemble2_body<WPB, true>(nx, ny, nn, chunk, node_off, Edf, kappa_g, vals, flag, gen, pbias, kscale,
                                      blockIdx.x, gridDim.x);
}

// Sensitivity on the box lattice.  The reflections of a box across its
// mid-planes commute with K^0, so in the Walsh basis of each displacement
// component, f_t(a) = (-1)^(t.a) over the 2^d corners a, K^0 splits into 2^d
// independent d x d blocks: sector c couples the modes t = c xor e_i of the
// components i.  With w_{t,i} = sum_a f_t(a) u_{a,i} (a fast Walsh transform),
//     u_e^T K^0 u_e = sum_c sum_ij w_{c^e_i, i} B_c[i][j] w_{c^e_j, j},
// B_c[i][j] = f_{c^e_i}^T K^0_{ij} f_{c^e_j} / 4^d, each term of the outer sum
// a non-negative energy.  One thread per cell, float-pair arithmetic; the
// blocks arrive as kernel parameters (constant bank, read as instruction
// operands); 64 registers, 8 blocks per SM.
#ifndef SOPTX_SENS_MINB
#define SOPTX_SENS_MINB 8
#endif
// Displacement entries: doubles split on the fly, or float pairs made once per call.
__device__ __forceinline__ df load_u(const double *__restrict__ u, int64_t r) { return df_split(u[r]); }
__device__ __forceinline__ df load_u(const float2 *__restrict__ u, int64_t r)
{
    const float2 v = u[r];
    return df{v.x, v.y};
}

template <int D, typename UT>
__device__ __forceinline__ void lattice_sens_body(int nx, int ny, int64_t nc, const double *__restrict__ rho,
                                                  const UT *__restrict__ u, SimpParams sp, const SectorTable<D> B,
                                                  const double *__restrict__ gscale, double *__restrict__ out,
                                                  double *__restrict__ partial, unsigned *__restrict__ counter,
                                                  double *__restrict__ c, int64_t bid, int64_t nblk, int vthreads)
{
    constexpr int NCR = 1 << D;
    const double g = gscale ? *gscale : -1.0;
    double mine = 0.0;
    // block bid of nblk blocks of vthreads threads (threads from vthreads on add nothing)
    const int64_t e0 = (int)threadIdx.x < vthreads ? bid * vthreads + threadIdx.x : nc;
    for (int64_t e = e0; e < nc; e += nblk * vthreads) {
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
            for (int i = 0; i < D; i++) w[a][i] = load_u(u, D * node + i);
        }
        // in-place Walsh transform along each axis
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
        // compensated sum of the sector energies: S + C
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
                    const float2 bb = B.b[(c * D + i) * D + j];     // off-diagonal entries pre-doubled
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
        out[e] = g * simp_dE(sp, re) * sd;
        mine += simp_E(sp, re) * sd;
    }
    if (c) grid_sum_last_block_n(mine, partial, counter, c, (unsigned)bid, (unsigned)nblk);
}

template <int D, typename UT>
__global__ void __launch_bounds__(128, SOPTX_SENS_MINB)
k_lattice_sens(int nx, int ny, int64_t nc, const double *__restrict__ rho, const UT *__restrict__ u,
               SimpParams sp, const SectorTable<D> B, const double *__restrict__ gscale,
               double *__restrict__ out, double *__restrict__ partial, unsigned *__restrict__ counter,
               double *__restrict__ c)
{
    lattice_sens_body<D, UT>(nx, ny, nc, rho, u, sp, B, gscale, out, partial, counter, c, blockIdx.x, gridDim.x,
                             blockDim.x);
}

// Grouped step of small box lattices (2D and 3D): one cluster of kGroupCtas CTAs per
// request of a table that arrives as the kernel's parameter.  The cluster's
// CTAs share the moduli (and u's float pairs); after a cluster barrier they
// share the assembly of the mesh's nodes (the warps take the node chunks; the
// moduli come through coherent loads, having been written in this launch) and
// the sensitivities, taking the blocks of the single step's sensitivity launch
// (sgrid blocks of 128 threads) in turn, with the same last-block sum -- the
// same arithmetic in the same order as the three kernels of a single step, so
// K, dc and c are bitwise theirs; one launch serves the whole group.
template <int D> struct LatReq {
    int nx, ny, nz, chunk, sgrid;
    unsigned gen;
    uint32_t pbias;
    int64_t nn, nc, ndof;
    double kscale;
    SimpParams sp;
    SectorTable<D> B;
    const double *rho, *u, *gscale, *K0;
    double *vals, *dc, *c, *partial;
    float2 *Edf, *udf;
    const int64_t *node_off;
    unsigned *flag, *counter;
    const float2 *kappa;
};
constexpr int kGroupMax = 32;
constexpr int kGroupCtas = 8;   // a portable cluster size
template <int D> struct LatGroup {
    int n;
    LatReq<D> r[kGroupMax];
};
static_assert(sizeof(LatGroup<3>) < 32000, "the request table travels as the kernel's parameter");

template <int D>
__global__ void __launch_bounds__(256) k_lattice_step_group(const __grid_constant__ LatGroup<D> G)
{
    const int rank = (int)(blockIdx.x % kGroupCtas);   // the CTA's rank in its cluster
    const LatReq<D> &R = G.r[blockIdx.x / kGroupCtas];
    simp_df_body(D, R.nx, R.ny, R.nz, R.nc, R.rho, R.sp, R.Edf, R.node_off, R.K0, R.vals, R.flag, R.gen, R.ndof, R.u,
                 R.udf, rank, kGroupCtas);
    // the moduli and u's pairs of the whole cluster written before any CTA reads them
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    if constexpr (D == 2)
        lattice_assemble2_body<8, false>(R.nx, R.ny, R.nn, R.chunk, R.node_off, R.Edf, R.kappa, R.vals, R.flag, R.gen,
                                         R.pbias, R.kscale, rank, kGroupCtas);
    else
        lattice_assemble3_body<8, false>(R.nx, R.ny, R.nz, R.nn, R.chunk, R.node_off, R.Edf, R.kappa, R.K0, R.rho,
                                         R.sp, R.vals, R.flag, R.gen, R.pbias, R.kscale, rank, kGroupCtas);
    for (int vb = rank; vb < R.sgrid; vb += kGroupCtas)
        lattice_sens_body<D, float2>(R.nx, R.ny, R.nc, R.rho, R.udf, R.sp, R.B, R.gscale, R.dc, R.partial, R.counter,
                                     R.c, vb, R.sgrid, 128);
}

}  // namespace

constexpr int kSensThreads = 128;
int lattice_sens_grid(int64_t nc)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((nc + kSensThreads - 1) / kSensThreads, 152 * 8));
}

template <int D>
static SectorTable<D> sector_table(const std::vector<float2> &v)
{
    SectorTable<D> B;
    for (int t = 0; t < (1 << D) * D * D; t++) B.b[t] = v[t];
    return B;
}

template <typename UT>
static cudaError_t lattice_sens_t(const soptx_mesh_s &m, const double *rho, const UT *u, double *out, double *c,
                                  const double *gscale, cudaStream_t st, bool after_assembly = false)
{
    const auto &h = m.h;
    const int grid = lattice_sens_grid(h.nc);
    if ((int)h.sectors.size() != (h.dim << h.dim) * h.dim) return cudaErrorInvalidValue;
    if (after_assembly && h.dim == 3) {
        // in the one-call step, right after the 3D assembly, whose blocks let it start
        // once the moduli kernel (the producer of u's pairs) has completed (as a
        // dependent launch after the 2D assembly the sensitivity made some steps
        // several times longer)
        return launch_dependent(k_lattice_sens<3, UT>, grid, kSensThreads, st, h.lat_n[0], h.lat_n[1], h.nc, rho,
                                u, simp_params(m.mat), sector_table<3>(h.sectors), gscale, out, m.d.scratch,
                                m.d.counter, c);
    }
    if (h.dim == 3)
        k_lattice_sens<3, UT><<<grid, kSensThreads, 0, st>>>(h.lat_n[0], h.lat_n[1], h.nc, rho, u,
                                                             simp_params(m.mat), sector_table<3>(h.sectors), gscale,
                                                             out, m.d.scratch, m.d.counter, c);
    else
        k_lattice_sens<2, UT><<<grid, kSensThreads, 0, st>>>(h.lat_n[0], h.lat_n[1], h.nc, rho, u,
                                                             simp_params(m.mat), sector_table<2>(h.sectors), gscale,
                                                             out, m.d.scratch, m.d.counter, c);
    return cudaGetLastError();
}

cudaError_t launch_lattice_sensitivity(const soptx_mesh_s &m, const double *rho, const double *u, double *out,
                                       double *c, const double *gscale, cudaStream_t st)
{
    return lattice_sens_t(m, rho, u, out, c, gscale, st);
}

// Sector blocks B_c[i][j] of a box element's K^0 (see k_lattice_sens), the
// off-diagonal ones doubled (only i <= j is summed), the entries that vanish
// on every box (sector_zero) checked against zero_tol relative to the largest
// sector entry and stored as zeros; returns
// false when K^0 does not split into the 2^d sectors (then the general
// sensitivity kernel is used).
bool build_lattice_sectors(int dim, const std::vector<double> &K0, double zero_tol, std::vector<float2> &B)
{
    const int ncr = 1 << dim, ldof = dim * ncr;
    auto f = [](int t, int a) { return (__builtin_popcount(t & a) & 1) ? -1.0 : 1.0; };
    double fmax = 0.0, offmax = 0.0;
    std::vector<double> F((size_t)ncr * dim * ncr * dim);
    for (int t = 0; t < ncr; t++)
        for (int i = 0; i < dim; i++)
            for (int t2 = 0; t2 < ncr; t2++)
                for (int j = 0; j < dim; j++) {
                    double s = 0.0;
                    for (int a = 0; a < ncr; a++)
                        for (int b = 0; b < ncr; b++) s += f(t, a) * K0[(size_t)(dim * a + i) * ldof + dim * b + j] * f(t2, b);
                    F[(((size_t)t * dim + i) * ncr + t2) * dim + j] = s;
                    fmax = std::max(fmax, std::fabs(s));
                    if ((t ^ (1 << i)) != (t2 ^ (1 << j))) offmax = std::max(offmax, std::fabs(s));
                }
    if (!(offmax <= 1e-13 * fmax)) return false;
    const double norm = 1.0 / ((double)ncr * ncr);
    // the entries the kernel skips must vanish (to the rounding of K^0: zero_tol)
    for (int c = 0; c < ncr; c++)
        for (int i = 0; i < dim; i++)
            for (int j = 0; j < dim; j++)
                if (sector_zero(c, i, j) &&
                    !(std::fabs(F[(((size_t)(c ^ (1 << i)) * dim + i) * ncr + (c ^ (1 << j))) * dim + j]) <= zero_tol * fmax))
                    return false;
    B.assign((size_t)ncr * dim * dim, make_float2(0.f, 0.f));
    for (int c = 0; c < ncr; c++)
        for (int i = 0; i < dim; i++)
            for (int j = 0; j < dim; j++) {
                // the entries that vanish on every box are stored as exact zeros
                const double x = sector_zero(c, i, j) ? 0.0 : (i == j ? 1.0 : 2.0) * norm *
                                 F[(((size_t)(c ^ (1 << i)) * dim + i) * ncr + (c ^ (1 << j))) * dim + j];
                const float hh = (float)x;
                B[((size_t)c * dim + i) * dim + j] = make_float2(hh, (float)(x - (double)hh));
            }
    return true;
}

// The assembly; with u given (and m.d.udf), the moduli kernel also leaves u
// as float pairs in m.d.udf for the sensitivity of the same step.
static cudaError_t lattice_assemble_u(const soptx_mesh_s &m, const double *rho, const double *u, double *vals,
                                      cudaStream_t st, cudaEvent_t moduli_done = nullptr)
{
    const auto &h = m.h;
    const SimpParams sp = simp_params(m.mat);
    const int eb = 256;
    const int64_t items = std::max<int64_t>(h.nc, (u && m.d.udf) ? h.ndof / 2 : 0);
    const int egrid = (int)std::min<int64_t>((items + eb - 1) / eb, 152 * 8);
    // a fresh nonzero generation per call marks this call's out-of-range flag
    unsigned gen = ++m.lattice_gen;
    if (gen == 0u) gen = ++m.lattice_gen;
    k_simp_df<<<std::max(egrid, 1), eb, 0, st>>>(h.dim, h.lat_n[0], h.lat_n[1], h.lat_n[2], h.nc, rho, sp,
                                                 (float2 *)m.d.Edf, m.d.node_off, m.d.K0, vals, m.d.lat_bad, gen,
                                                 h.ndof,
                                                 m.d.udf ? u : nullptr, m.d.udf);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    if (moduli_done) {
        err = cudaEventRecord(moduli_done, st);
        if (err != cudaSuccess) return err;
    }
    constexpr int WPB = 8;
    if (h.dim == 3) {
        const int64_t chunks = (h.nn + kChunk - 1) / kChunk;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((chunks + WPB - 1) / WPB, 152 * 4));
        // the chunk length (at most kChunk, even) that gives every warp the same
        // number of chunks, give or take one: no warp runs a round alone at the end
        const int64_t warps = (int64_t)grid * WPB;
        const int64_t rounds = (h.nn + warps * kChunk - 1) / (warps * kChunk);
        int chunk = (int)std::max<int64_t>(1, (h.nn + warps * rounds - 1) / (warps * rounds));
        chunk += chunk & 1;
        // scheduled while the moduli kernel runs (see grid_dep_wait)
        err = launch_dependent(k_lattice_assemble3<WPB>, grid, WPB * 32, st, h.lat_n[0], h.lat_n[1], h.lat_n[2],
                               h.nn, chunk, m.d.node_off, (const float2 *)m.d.Edf, (const float2 *)m.d.kappa, m.d.K0,
                               rho, sp, vals, m.d.lat_bad, gen, 0x38000000u + ((uint32_t)h.lat_kshift << 20),
                               std::ldexp(1.0, h.lat_kshift));
        if (err != cudaSuccess) return err;
    } else {
        // chunks of 3 .. 48 nodes: long enough to amortise a chunk's set-up, short
        // enough to give every warp slot of the GPU work on small meshes
        const int64_t groups = (h.nn + 2) / 3;
        const int chunk = 3 * (int)std::max<int64_t>(1, std::min<int64_t>(16, groups / (152 * 4 * WPB)));
        const int64_t chunks = (h.nn + chunk - 1) / chunk;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((chunks + WPB - 1) / WPB, 152 * 8));
        err = launch_dependent(k_lattice_assemble2<WPB>, grid, WPB * 32, st, h.lat_n[0], h.lat_n[1], h.nn, chunk,
                               m.d.node_off, (const float2 *)m.d.Edf, (const float2 *)m.d.kappa, vals, m.d.lat_bad,
                               gen, 0x38000000u + ((uint32_t)h.lat_kshift << 20), std::ldexp(1.0, h.lat_kshift));
        if (err != cudaSuccess) return err;
    }
    return cudaGetLastError();
}

cudaError_t launch_lattice_assemble(const soptx_mesh_s &m, const double *rho, double *vals, cudaStream_t st)
{
    return lattice_assemble_u(m, rho, nullptr, vals, st);
}

// One call doing both passes: u is split into float pairs once, by the moduli
// kernel, instead of at every corner of every cell.
cudaError_t launch_lattice_step(const soptx_mesh_s &m, const double *rho, const double *u, double *vals, double *dc,
                                double *c, cudaStream_t st, const double *gscale)
{
    if (!m.d.udf || !u) {
        cudaError_t err = lattice_assemble_u(m, rho, nullptr, vals, st);
        if (err != cudaSuccess) return err;
        return launch_lattice_sensitivity(m, rho, u, dc, c, gscale, st);
    }
    if (m.h.dim == 2 && m.d.side) {
        // 2D: the sensitivity runs on the mesh's second stream beside the assembly
        // (it needs the moduli kernel's u pairs, not K); the assembly's grid is
        // not one full wave, so the two share the SMs
        cudaError_t err = lattice_assemble_u(m, rho, u, vals, st, m.d.ev[0]);
        if (err != cudaSuccess) return err;
        err = cudaStreamWaitEvent(m.d.side, m.d.ev[0], 0);
        if (err != cudaSuccess) return err;
        err = lattice_sens_t(m, rho, (const float2 *)m.d.udf, dc, c, gscale, m.d.side);
        if (err != cudaSuccess) return err;
        err = cudaEventRecord(m.d.ev[1], m.d.side);
        if (err != cudaSuccess) return err;
        return cudaStreamWaitEvent(st, m.d.ev[1], 0);
    }
    cudaError_t err = lattice_assemble_u(m, rho, u, vals, st);
    if (err != cudaSuccess) return err;
    return lattice_sens_t(m, rho, (const float2 *)m.d.udf, dc, c, gscale, st, true);
}

// kappa_delta[i][j] = K0[(a*, i), (b*, j)] for every offset delta (x fastest),
// a*, b* the corners of n and n + delta in the reference cell (high side on
// zero axes).
static std::vector<double> lattice_kappa_values(int dim, const std::vector<double> &K0)
{
    const int nd = dim == 3 ? 27 : 9, ldof = dim * (1 << dim);
    std::vector<double> kap((size_t)nd * dim * dim, 0.0);
    for (int dl = 0; dl < nd; dl++) {
        int a = 0, b = 0, r = dl;
        for (int m = 0; m < dim; m++) {
            const int delta = r % 3 - 1;
            r /= 3;
            const int am = delta < 0 ? 1 : 0, bm = am + delta;
            a |= am << m;
            b |= bm << m;
        }
        for (int i = 0; i < dim; i++)
            for (int j = 0; j < dim; j++)
                kap[(size_t)dl * dim * dim + i * dim + j] = K0[(size_t)(dim * a + i) * ldof + dim * b + j];
    }
    return kap;
}

// The 3D assembly multiplies float pairs of kappa 2^-shift, |kappa| 2^-shift in
// [2^-24, 2), and lets the conversion to FP64 put 2^shift back; with element
// moduli in [2^-60, 2^60] its products then stay below 2^84, and a product
// that falls below the FP32 normal range is off by less than 1e-12 of its
// entry's scale.  False when the kappa entries span more than 2^24 (entries
// below 2^-40 of the largest count as zeros); those boxes take the general path.
bool lattice_kappa_shift(int dim, const std::vector<double> &K0, int &shift)
{
    const std::vector<double> kap = lattice_kappa_values(dim, K0);
    double kmax = 0.0, kmin = INFINITY;
    for (double x : kap) kmax = std::max(kmax, std::fabs(x));
    for (double x : kap)
        if (std::fabs(x) > std::ldexp(kmax, -40)) kmin = std::min(kmin, std::fabs(x));
    if (!(kmax > 0.0) || !std::isfinite(kmax) || !(kmin >= std::ldexp(kmax, -24))) return false;
    // the kernels form entry (j, i) of each block as +-entry (i, j): the pairs
    // must agree to the rounding of K^0 (a few ulps), with the sign the kernels
    // read off the two stored entries
    const int nd = dim == 3 ? 27 : 9;
    for (int dl = 0; dl < nd; dl++)
        for (int i = 0; i < dim; i++)
            for (int j = i + 1; j < dim; j++) {
                const double a = kap[(size_t)dl * dim * dim + i * dim + j], b = kap[(size_t)dl * dim * dim + j * dim + i];
                // (entries that vanish in exact arithmetic may carry rounding noise of
                // either sign: the absolute term covers them)
                const double tol = 1e-14 * std::max(std::fabs(a), std::fabs(b)) + 1e-15 * kmax;
                const bool same = std::signbit(a) == std::signbit(b);
                if (!(std::fabs(same ? a - b : a + b) <= tol)) return false;
            }
    shift = std::ilogb(kmax);
    return shift > -900 && shift < 900;
}

// The kappa table times 2^-shift as float pairs.
void build_lattice_kappa(int dim, const std::vector<double> &K0, int shift, std::vector<float2> &kappa)
{
    const std::vector<double> kap = lattice_kappa_values(dim, K0);
    kappa.resize(kap.size());
    for (size_t t = 0; t < kap.size(); t++) {
        const double x = std::ldexp(kap[t], -shift);
        const float hh = (float)x;
        kappa[t] = make_float2(hh, (float)(x - (double)hh));
    }
}

// ------------------------------------------------------------- grouped steps
// Meshes the grouped step serves: 2D and 3D box lattices whose sensitivity
// splits into Walsh sectors, up to kGroupCells cells in 2D and kGroupCells3 in
// 3D (a cluster of kGroupCtas CTAs does the whole step; a larger 3D mesh's step
// takes longer on one cluster than its three launches across the GPU).
constexpr int64_t kGroupCells = 4096;
constexpr int64_t kGroupCells3 = 1024;
static_assert(kSensThreads == 128, "the grouped step replays the 128-thread sensitivity blocks");
// its 256 threads then sum at most 128 block partials as the 128 of the single step do
static_assert((kGroupCells + 127) / 128 <= 128, "the grouped step's last-block sum needs <= 128 partials");

bool lattice_groupable(const soptx_mesh_s &m)
{
    const auto &h = m.h;
    return m.path == SOPTX_PATH_LATTICE && (h.dim == 2 || h.dim == 3) && m.d.sectors && m.d.udf && m.d.Edf &&
           h.nc > 0 && h.nc <= (h.dim == 2 ? kGroupCells : kGroupCells3) &&
           (int)h.sectors.size() == (h.dim << h.dim) * h.dim;
}

template <int D>
static cudaError_t launch_group_d(const std::vector<int> &ks, const soptx_mesh_s *const *ms, const double *const *rho,
                                  const double *const *u, double *const *vals, double *const *dc, double *const *c,
                                  cudaStream_t st)
{
    const int n = (int)ks.size();
    for (int k0 = 0; k0 < n; k0 += kGroupMax) {
        static thread_local LatGroup<D> G;   // ~24 KB: off the stack
        G = LatGroup<D>{};
        G.n = std::min(kGroupMax, n - k0);
        for (int k = 0; k < G.n; k++) {
            const int j = ks[k0 + k];
            const soptx_mesh_s &m = *ms[j];
            const auto &h = m.h;
            LatReq<D> &R = G.r[k];
            unsigned gen = ++m.lattice_gen;
            if (gen == 0u) gen = ++m.lattice_gen;
            R.nx = h.lat_n[0];
            R.ny = h.lat_n[1];
            R.nz = D == 3 ? h.lat_n[2] : 1;
            constexpr int warps = 8 * kGroupCtas;
            if (D == 2) {
                // node chunks of 3 .. 48 for the cluster's warps
                const int64_t groups = (h.nn + 2) / 3;
                R.chunk = 3 * (int)std::max<int64_t>(1, std::min<int64_t>(16, groups / warps));
            } else {
                // even chunks of at most kChunk nodes, about as many per warp (as in the single step)
                const int64_t rounds = (h.nn + warps * kChunk - 1) / (warps * kChunk);
                int chunk = (int)std::max<int64_t>(1, (h.nn + warps * rounds - 1) / (warps * rounds));
                R.chunk = chunk + (chunk & 1);
            }
            R.sgrid = lattice_sens_grid(h.nc);
            R.gen = gen;
            R.pbias = 0x38000000u + ((uint32_t)h.lat_kshift << 20);
            R.nn = h.nn;
            R.nc = h.nc;
            R.ndof = h.ndof;
            R.kscale = std::ldexp(1.0, h.lat_kshift);
            R.sp = simp_params(m.mat);
            R.B = sector_table<D>(h.sectors);
            R.rho = rho[j];
            R.u = u[j];
            R.gscale = nullptr;
            R.K0 = m.d.K0;
            R.vals = vals[j];
            R.dc = dc[j];
            R.c = c[j];
            R.partial = m.d.scratch;
            R.Edf = (float2 *)m.d.Edf;
            R.udf = m.d.udf;
            R.node_off = m.d.node_off;
            R.flag = m.d.lat_bad;
            R.counter = m.d.counter;
            R.kappa = (const float2 *)m.d.kappa;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(G.n * kGroupCtas));
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = kGroupCtas;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaError_t err = cudaLaunchKernelEx(&cfg, k_lattice_step_group<D>, G);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

cudaError_t launch_lattice_group(const soptx_mesh_s *const *ms, const double *const *rho, const double *const *u,
                                 double *const *vals, double *const *dc, double *const *c, int n, cudaStream_t st)
{
    std::vector<int> k2, k3;
    for (int k = 0; k < n; k++) (ms[k]->h.dim == 2 ? k2 : k3).push_back(k);
    cudaError_t err = k2.empty() ? cudaSuccess : launch_group_d<2>(k2, ms, rho, u, vals, dc, c, st);
    if (err == cudaSuccess && !k3.empty()) err = launch_group_d<3>(k3, ms, rho, u, vals, dc, c, st);
    return err;
}

}  // namespace soptx
