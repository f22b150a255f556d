// The C ABI (include/soptx.h): argument validation, device residency of a mesh
// and dispatch to the kernels.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "internal.h"

namespace soptx {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_fail_after{0};
static std::atomic<int> g_no_sectors{0};

void set_error(const std::string &msg) { g_last_error = msg; }

cudaError_t dev_alloc(void **p, size_t bytes)
{
    *p = nullptr;
    int64_t n = g_fail_after.load();
    if (n > 0) {
        if (n == 1) {
            g_fail_after.store(0);
            return cudaErrorMemoryAllocation;
        }
        g_fail_after.store(n - 1);
    }
    if (bytes == 0) bytes = 16;
    return cudaMalloc(p, bytes);
}

static void free_device(DeviceMesh &d)
{
    void *ptrs[] = {d.indptr, d.indices, d.cell_node, d.node_off, d.inc_ptr, d.inc,
                    d.pos, d.geo, d.M, d.K, d.scratch, d.Edf, d.kappa, d.K0, d.sectors, d.udf, d.part,
                    d.inc_e, d.inc_a, d.counter, d.xcell, d.qw, d.qdphi, d.qdgeo, d.cg, d.lat_bad, d.stage,
                    d.kvals, d.sgeo, d.sq, d.ssf, d.cgeo, d.Mf, d.ptoff, d.pia, d.pib, d.pmeta, d.pre, d.prm, d.pblk,
                    d.cnrec, d.cinc_e, d.cinc_a, d.crec, d.cticket};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (d.cg_exec) cudaGraphExecDestroy(d.cg_exec);
    if (d.cg_cap) cudaStreamDestroy(d.cg_cap);
    for (cudaEvent_t e : d.ev)
        if (e) cudaEventDestroy(e);
    if (d.side) cudaStreamDestroy(d.side);
    d = DeviceMesh{};
}

// The mesh's second stream and its two events, made once (the host-buffer step and
// the 2D lattice step use them).
static cudaError_t ensure_side(soptx_mesh_s &m)
{
    auto &d = m.d;
    if (d.side) return cudaSuccess;
    cudaStream_t side = nullptr;
    cudaEvent_t ev[2] = {};
    // meshes with the strain-energy sensitivities run their assembly (3D) or
    // their sensitivities (2D) on this stream in the one-call step, at the
    // highest priority (see launch_step)
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess)
        e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, d.strain ? greatest : least);
    for (int i = 0; i < 2 && e == cudaSuccess; i++) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        for (cudaEvent_t x : ev)
            if (x) cudaEventDestroy(x);
        if (side) cudaStreamDestroy(side);
        return e;
    }
    d.side = side;
    for (int i = 0; i < 2; i++) d.ev[i] = ev[i];
    return cudaSuccess;
}

static soptx_status cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return SOPTX_OK;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SOPTX_ENOMEM : SOPTX_ECUDA;
}

template <typename T>
static soptx_status upload(T **dst, const std::vector<T> &src, cudaStream_t st, int64_t &bytes, const char *what)
{
    size_t n = src.size() * sizeof(T);
    cudaError_t e = dev_alloc((void **)dst, n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e, what);
    }
    bytes += (int64_t)(n ? n : 16);
    if (n) {
        e = cudaMemcpyAsync(*dst, src.data(), n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_status(e, what);
    }
    return SOPTX_OK;
}

static float2 split_pair(double x)
{
    const float hh = (float)x;
    return make_float2(hh, (float)(x - (double)hh));
}

// Tables of the strain-energy sensitivities (k_strain_energy).
static soptx_status setup_strain(soptx_mesh_s &m, const RefElement &ref, cudaStream_t st)
{
    const HostMesh &h = m.h;
    RefQuad q;
    if (is_simplex(h.cell)) build_simplex_quadrature(ref, q);
    else build_tensor_quadrature(ref, q);
    std::vector<float2> tab((size_t)q.nq * (1 + h.nb * h.dim));
    for (int p = 0; p < q.nq; p++) tab[p] = split_pair(q.w[p]);
    for (size_t t = 0; t < q.dphi.size(); t++) tab[q.nq + t] = split_pair(q.dphi[t]);
    const int ng = h.dim * h.dim + 1;
    const int64_t ncg = m.path == SOPTX_PATH_UNIFORM ? 1 : h.nc;
    std::vector<float2> sg((size_t)ncg * ng);
    for (size_t t = 0; t < sg.size(); t++) sg[t] = split_pair(h.geo[t]);
    soptx_status s = upload(&m.d.sq, tab, st, m.device_bytes, "quadrature table");
    if (s == SOPTX_OK) s = upload(&m.d.sgeo, sg, st, m.device_bytes, "cell geometry pairs");
    if (s == SOPTX_OK && h.dim == 3 && !is_simplex(h.cell) && (h.order == 2 || h.order == 3)) {
        // the 1D factors of the tensor rule, for the sum-factorised kernel
        std::vector<double> w1, val, der;
        tensor_1d_factors(h.order, w1, val, der);
        const int n = h.order + 1;
        std::vector<float2> sf;
        for (double x : w1) sf.push_back(split_pair(x));
        for (double x : val) sf.push_back(split_pair(x));
        for (double x : der) sf.push_back(split_pair(x));
        for (int a = 0; a < h.nb; a++) {
            const int *la = ref.lat[(size_t)a].data();
            sf.push_back(make_float2((float)(la[0] + n * la[1] + n * n * la[2]), 0.f));
        }
        s = upload(&m.d.ssf, sf, st, m.device_bytes, "1D factors of the rule");
    }
    if (s == SOPTX_OK) {
        m.d.snq = q.nq;
        m.d.strain = true;
    }
    return s;
}

// Tables of the per-call contraction of 2D cells (k_contract_pairs): G and
// |det J| per cell in FP32 (whole float4s), the reference integrals
// [a][b][k][l] in FP32, and the node pairs.  K is symmetric, so the block pair
// (a, b), (b, a) of two nodes
// that share a cell is assembled once, by whichever of them comes first in the
// processing order, and each node's diagonal block by the node itself.  The
// order takes nodes by their first cell (then id), so it sweeps the mesh and
// both row blocks of a pair are written close together in time.  A pair's
// records are the cells holding both nodes, in ascending order, each with the
// reference-integral pair a_loc nb + b_loc.  The pairs of a window of
// consecutive owners (about kPairWindow pairs) are sorted by cell count, most
// first, and cut into tiles of 32, so the lanes of a warp walk about as many
// cells each; a window's last tile is padded with empty pairs (no cells).
// The same tables serve the cached FP64 element matrices of 2D cells (cached:
// each record's 2 x 2 block is also gathered into record order) and the one
// FP64 matrix of a uniform mesh (unif); for those the local pair is stored as
// a_loc << 8 | b_loc.  In 3D (uniform meshes) every node takes all of its own
// column blocks instead of the pairs after it, so no block is written
// transposed.
static constexpr size_t kPairWindow = 4096;

struct PairTables {
    std::vector<uint32_t> ia, ib, meta;   // per pair, tiles of 32 lanes
    std::vector<uint32_t> toff;           // [tiles + 1] record offsets / 32
    std::vector<int32_t> re;              // per record: the cell
    std::vector<uint16_t> rm;             // per record: the local pair
    int64_t ntiles = 0;
};

// The pair tables, on the host.  bytes: the local pair as a_loc << 8 | b_loc,
// else a_loc nb + b_loc.  False when a node meets more than 1023 cells or a
// value index / d needs more than 32 bits (a pair's cell count has 10 bits in
// the tables): such meshes keep the cached gather.
static bool build_pair_tables(const HostMesh &h, bool bytes, PairTables &T)
{
    const int d = h.dim, nb = h.nb;
    // 3D: every node assembles all of its own row blocks (the symmetric layout's
    // transposed 24-byte pieces leave L2 sectors partly filled)
    const bool sym = d == 2;
    for (int64_t n = 0; n < h.nn; n++)
        if (h.inc_ptr[(size_t)n + 1] - h.inc_ptr[(size_t)n] > 1023) return false;
    if ((int64_t)d * h.node_off[(size_t)h.nn] > (int64_t)UINT32_MAX) return false;
    // processing order: nodes by first cell (the incidences are in ascending cell
    // order), then id; a counting sort
    std::vector<int32_t> order((size_t)h.nn), rank((size_t)h.nn);
    {
        auto first = [&](int64_t n) -> int64_t {
            return h.inc_ptr[(size_t)n + 1] > h.inc_ptr[(size_t)n] ? h.inc_e[(size_t)h.inc_ptr[(size_t)n]] : h.nc;
        };
        std::vector<int64_t> start((size_t)h.nc + 2, 0);
        for (int64_t n = 0; n < h.nn; n++) start[(size_t)first(n) + 1]++;
        for (size_t c = 1; c < start.size(); c++) start[c] += start[c - 1];
        for (int64_t n = 0; n < h.nn; n++) order[(size_t)start[(size_t)first(n)]++] = (int32_t)n;
        for (int64_t i = 0; i < h.nn; i++) rank[(size_t)order[(size_t)i]] = (int32_t)i;
    }
    // the incidence of each (cell, local node)
    std::vector<int32_t> cinc((size_t)h.nc * nb, 0);
    for (int64_t n = 0; n < h.nn; n++)
        for (int32_t q = h.inc_ptr[(size_t)n]; q < h.inc_ptr[(size_t)n + 1]; q++)
            cinc[(size_t)h.inc_e[(size_t)q] * nb + h.inc_a[(size_t)q]] = q;
    auto &ia = T.ia, &ib = T.ib, &meta = T.meta, &toff = T.toff;
    auto &re = T.re;
    auto &rm = T.rm;
    ia.clear();
    ib.clear();
    meta.clear();
    toff.assign(1, 0u);
    re.clear();
    rm.clear();
    struct WPair {
        uint32_t pa, pb, meta;
        size_t r0;
    };
    std::vector<WPair> win;
    std::vector<int32_t> wre, scnt, sstart, sfill, te;
    std::vector<uint16_t> wrm, tm;
    std::vector<size_t> idx;
    auto flush = [&]() {
        if (win.empty()) return;
        idx.resize(win.size());
        for (size_t k = 0; k < idx.size(); k++) idx[k] = k;
        std::stable_sort(idx.begin(), idx.end(),
                         [&](size_t x, size_t y) { return (win[x].meta & 1023u) > (win[y].meta & 1023u); });
        for (size_t t0 = 0; t0 < win.size(); t0 += 32) {
            const int ct = (int)(win[idx[t0]].meta & 1023u);
            for (size_t l = 0; l < 32; l++) {
                const bool real = t0 + l < win.size();
                const WPair &w = win[idx[real ? t0 + l : t0]];
                ia.push_back(real ? w.pa : 0u);
                ib.push_back(real ? w.pb : 0u);
                meta.push_back(real ? w.meta : 0u);
            }
            for (int k = 0; k < ct; k++)
                for (size_t l = 0; l < 32; l++) {
                    const bool real = t0 + l < win.size();
                    const WPair &w = win[idx[real ? t0 + l : t0]];
                    const bool has = real && k < (int)(w.meta & 1023u);
                    re.push_back(has ? wre[w.r0 + (size_t)k] : 0);
                    rm.push_back(has ? wrm[w.r0 + (size_t)k] : (uint16_t)0);
                }
            toff.push_back(toff.back() + (uint32_t)ct);
        }
        win.clear();
        wre.clear();
        wrm.clear();
    };
    for (int64_t i = 0; i < h.nn; i++) {
        const int32_t a = order[(size_t)i];
        const int32_t q0 = h.inc_ptr[(size_t)a], q1 = h.inc_ptr[(size_t)a + 1];
        const int64_t off = h.node_off[(size_t)a];
        const int deg = (int)(h.node_off[(size_t)a + 1] - off);
        // the owner's records grouped by column block, ascending cells within each
        scnt.assign((size_t)deg, 0);
        for (int32_t q = q0; q < q1; q++) {
            const int32_t *cn = &h.cell_node[(size_t)h.inc_e[(size_t)q] * nb];
            for (int j = 0; j < nb; j++)
                if (!sym || cn[j] == a || rank[(size_t)cn[j]] > i) scnt[h.pos[(size_t)q * nb + j]]++;
        }
        sstart.assign((size_t)deg + 1, 0);
        for (int p = 0; p < deg; p++) sstart[(size_t)p + 1] = sstart[(size_t)p] + scnt[(size_t)p];
        sfill.assign(sstart.begin(), sstart.end() - 1);
        te.resize((size_t)sstart[(size_t)deg]);
        tm.resize((size_t)sstart[(size_t)deg]);
        for (int32_t q = q0; q < q1; q++) {
            const int32_t e = h.inc_e[(size_t)q];
            const int32_t *cn = &h.cell_node[(size_t)e * nb];
            const int al = h.inc_a[(size_t)q];
            for (int j = 0; j < nb; j++)
                if (!sym || cn[j] == a || rank[(size_t)cn[j]] > i) {
                    const int32_t f = sfill[h.pos[(size_t)q * nb + j]]++;
                    te[(size_t)f] = e;
                    tm[(size_t)f] = (uint16_t)(bytes ? al << 8 | j : al * nb + j);
                }
        }
        for (int p = 0; p < deg; p++) {
            const int32_t c = scnt[(size_t)p];
            if (c == 0) continue;
            const int32_t b = h.nbr[(size_t)(off + p)];
            // the block of a in b's rows, from the pair's first cell
            const int32_t e = te[(size_t)sstart[(size_t)p]];
            const int t0 = tm[(size_t)sstart[(size_t)p]];
            const int al = bytes ? t0 >> 8 : t0 / nb, bl = bytes ? t0 & 255 : t0 % nb;
            const int pba = h.pos[(size_t)cinc[(size_t)e * nb + bl] * nb + al];
            const int64_t offb = h.node_off[(size_t)b];
            const int degb = (int)(h.node_off[(size_t)b + 1] - offb);
            const uint32_t pa = (uint32_t)(d * off + p), pb = sym ? (uint32_t)(d * offb + pba) : pa;
            const uint32_t rla = (uint32_t)(d * deg), rlb = (uint32_t)(d * (sym ? degb : deg));
            win.push_back(WPair{pa, pb, (uint32_t)c | rla << 10 | rlb << 21, wre.size()});
            wre.insert(wre.end(), te.begin() + sstart[(size_t)p], te.begin() + sstart[(size_t)p + 1]);
            wrm.insert(wrm.end(), tm.begin() + sstart[(size_t)p], tm.begin() + sstart[(size_t)p + 1]);
        }
        if (win.size() >= kPairWindow) flush();
    }
    flush();
    // the kernel stages chunks of 8 tiles: whole chunks of pairs, and 16 record
    // offsets from each chunk's first
    const int64_t ntiles = (int64_t)toff.size() - 1, nchunks = (ntiles + 7) / 8;
    toff.resize((size_t)(nchunks * 8 + 16), toff.back());
    ia.resize((size_t)(nchunks * 8 * 32), 0u);
    ib.resize((size_t)(nchunks * 8 * 32), 0u);
    meta.resize((size_t)(nchunks * 8 * 32), 0u);
    T.ntiles = ntiles;
    return true;
}

static soptx_status setup_contract_pairs(soptx_mesh_s &m, const RefElement &ref, cudaStream_t st, bool cached,
                                        bool unif = false)
{
    const HostMesh &h = m.h;
    const int d = h.dim, nb = h.nb, ng = d * d + 1, n4 = d == 3 ? 3 : 2, mp = d == 3 ? 12 : 4;
    const bool bytes = cached || unif;   // local pair as a_loc << 8 | b_loc
    PairTables T;
    if (!build_pair_tables(h, bytes, T)) return SOPTX_OK;
    std::vector<float4> cg((size_t)h.nc * n4, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int64_t e = 0; e < h.nc; e++) {
        float *dst = reinterpret_cast<float *>(&cg[(size_t)e * n4]);
        for (int t = 0; t < ng; t++) dst[t] = (float)h.geo[(size_t)e * ng + t];
    }
    std::vector<float> mf((size_t)nb * nb * mp, 0.f);
    for (int a = 0; a < nb; a++)
        for (int b = 0; b < nb; b++)
            for (int k = 0; k < d; k++)
                for (int l = 0; l < d; l++)
                    mf[((size_t)a * nb + b) * mp + k * d + l] = (float)ref.M[(((size_t)k * d + l) * nb + a) * nb + b];
    soptx_status s = SOPTX_OK;
    if (!bytes) s = upload(&m.d.cgeo, cg, st, m.device_bytes, "cell geometry");
    if (s == SOPTX_OK && !bytes) s = upload(&m.d.Mf, mf, st, m.device_bytes, "reference integrals (FP32)");
    if (s == SOPTX_OK) s = upload(&m.d.ptoff, T.toff, st, m.device_bytes, "pair tiles");
    if (s == SOPTX_OK) s = upload(&m.d.pia, T.ia, st, m.device_bytes, "pair blocks");
    if (s == SOPTX_OK) s = upload(&m.d.pib, T.ib, st, m.device_bytes, "pair transposed blocks");
    if (s == SOPTX_OK) s = upload(&m.d.pmeta, T.meta, st, m.device_bytes, "pair counts and row lengths");
    if (s == SOPTX_OK) s = upload(&m.d.pre, T.re, st, m.device_bytes, "pair cells");
    if (s == SOPTX_OK) s = upload(&m.d.prm, T.rm, st, m.device_bytes, "pair reference integrals");
    if (s == SOPTX_OK) s = upload(&m.d.cticket, std::vector<unsigned>(2, 0u), st, m.device_bytes, "chunk counter");
    if (s == SOPTX_OK && cached) {
        // each record's block of the cache, gathered once here so the kernel reads
        // them in record order
        const int64_t nrec = (int64_t)T.re.size();
        cudaError_t e = dev_alloc((void **)&m.d.pblk, (size_t)std::max<int64_t>(nrec, 1) * 2 * sizeof(float4));
        if (e == cudaSuccess) e = launch_pair_blocks(m, nrec, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s = cuda_status(e, "pair blocks");
        } else {
            m.device_bytes += std::max<int64_t>(nrec, 1) * 2 * (int64_t)sizeof(float4);
        }
    }
    if (s == SOPTX_OK) {
        m.d.ptiles = T.ntiles;
        (unif ? m.d.puniform : cached ? m.d.pcached : m.d.contract) = true;
    }
    return s;
}

// Tables of the node-owner contraction of 3D cells (k_contract_rows), on the
// host.  False when a node meets 65536 cells or more (a node record holds the
// incident-cell count in 16 bits): such fans keep the cached gather.
struct RowTables {
    // per node in processing order: its row block offset (node_off, low and
    // high words), first incidence, cell count << 16 | degree
    std::vector<int4> nrec;
    std::vector<int32_t> ce;      // per incidence, each node's cells in chain order
    std::vector<uint8_t> ca;      // the node's local index in that cell
    std::vector<uint16_t> rec;    // per (incidence, lane): p | b << 9 | first << 14 | last << 15
};

static bool build_row_tables(const HostMesh &h, RowTables &T)
{
    const int nb = h.nb;
    for (int64_t n = 0; n < h.nn; n++)
        if (h.inc_ptr[(size_t)n + 1] - h.inc_ptr[(size_t)n] >= 65536) return false;
    // processing order: nodes by incident-cell count, largest first, ascending ids
    // within a count (a counting sort), so a warp's node groups walk as many cells
    std::vector<int32_t> order((size_t)h.nn);
    {
        int32_t cmax = 0;
        for (int64_t n = 0; n < h.nn; n++) cmax = std::max(cmax, h.inc_ptr[n + 1] - h.inc_ptr[n]);
        std::vector<int64_t> start((size_t)cmax + 2, 0);
        for (int64_t n = 0; n < h.nn; n++) start[(size_t)(cmax - (h.inc_ptr[n + 1] - h.inc_ptr[n])) + 1]++;
        for (size_t c = 1; c < start.size(); c++) start[c] += start[c - 1];
        for (int64_t n = 0; n < h.nn; n++)
            order[(size_t)start[(size_t)(cmax - (h.inc_ptr[n + 1] - h.inc_ptr[n]))]++] = (int32_t)n;
    }
    // Each node's cells as a chain: the next cell is the unvisited one that holds
    // the most of the nodes the group's lanes hold now (ties: the lowest cell id);
    // a lane keeps its node when the next cell has it, and the cell's other nodes
    // go to the free lanes in local order.  A lane whose column block continues
    // into the next cell keeps its row sums in registers instead of a round trip
    // through shared memory.  Per (incidence, lane): column block p (bits 0-8),
    // local node b (bits 9-13), and whether this is the first (bit 14) or the last
    // (bit 15) time the node's chain meets that block.
    const int64_t ninc = h.inc_ptr[(size_t)h.nn];
    auto &ce = T.ce;
    auto &ca = T.ca;
    auto &rec = T.rec;
    ce.assign((size_t)ninc, 0);
    ca.assign((size_t)ninc, 0);
    rec.assign((size_t)ninc * nb, 0);
    {
        std::vector<int64_t> lane_mark((size_t)h.nn, -1), cell_mark((size_t)h.nn, -1);
        std::vector<int32_t> cell_loc((size_t)h.nn, 0);
        std::vector<int32_t> lanes(nb), next(nb);
        std::vector<char> used, taken(nb), seen;
        int64_t stamp = 0;
        for (int64_t n = 0; n < h.nn; n++) {
            const int32_t q0 = h.inc_ptr[(size_t)n], cnt = h.inc_ptr[(size_t)n + 1] - q0;
            used.assign((size_t)cnt, 0);
            int32_t t = 0;
            for (int32_t k = 0; k < cnt; k++) {
                if (k > 0) {
                    // the unvisited cell sharing the most nodes with the lanes
                    ++stamp;
                    for (int L = 0; L < nb; L++) lane_mark[(size_t)lanes[L]] = stamp;
                    int best = -1, bshare = -1;
                    for (int32_t c = 0; c < cnt; c++) {
                        if (used[(size_t)c]) continue;
                        const int32_t *cn = &h.cell_node[(size_t)h.inc_e[(size_t)(q0 + c)] * nb];
                        int share = 0;
                        for (int b = 0; b < nb; b++) share += lane_mark[(size_t)cn[b]] == stamp;
                        if (share > bshare) { bshare = share; best = c; }
                    }
                    t = best;
                }
                used[(size_t)t] = 1;
                const int32_t qo = q0 + t, e = h.inc_e[(size_t)qo];
                const int32_t *cn = &h.cell_node[(size_t)e * nb];
                if (k == 0) {
                    for (int L = 0; L < nb; L++) next[L] = L;
                } else {
                    ++stamp;
                    for (int b = 0; b < nb; b++) { cell_mark[(size_t)cn[b]] = stamp; cell_loc[(size_t)cn[b]] = b; }
                    std::fill(taken.begin(), taken.end(), 0);
                    for (int L = 0; L < nb; L++) {
                        next[L] = cell_mark[(size_t)lanes[L]] == stamp ? cell_loc[(size_t)lanes[L]] : -1;
                        if (next[L] >= 0) taken[next[L]] = 1;
                    }
                    int b = 0;
                    for (int L = 0; L < nb; L++) {
                        if (next[L] >= 0) continue;
                        while (taken[b]) b++;
                        next[L] = b;
                        taken[b] = 1;
                    }
                }
                const int64_t qn = q0 + k;
                ce[(size_t)qn] = e;
                ca[(size_t)qn] = h.inc_a[(size_t)qo];
                for (int L = 0; L < nb; L++) {
                    lanes[L] = cn[next[L]];
                    rec[(size_t)qn * nb + L] = (uint16_t)((next[L] << 9) | h.pos[(size_t)qo * nb + next[L]]);
                }
            }
            // first and last meeting of each column block along the chain
            const int deg = (int)(h.node_off[(size_t)n + 1] - h.node_off[(size_t)n]);
            seen.assign((size_t)deg, 0);
            for (int64_t qn = q0; qn < q0 + cnt; qn++)
                for (int L = 0; L < nb; L++) {
                    uint16_t &r = rec[(size_t)qn * nb + L];
                    if (!seen[r & 511u]) { seen[r & 511u] = 1; r = (uint16_t)(r | 0x4000u); }
                }
            seen.assign((size_t)deg, 0);
            for (int64_t qn = q0 + cnt - 1; qn >= q0; qn--)
                for (int L = 0; L < nb; L++) {
                    uint16_t &r = rec[(size_t)qn * nb + L];
                    if (!seen[r & 511u]) { seen[r & 511u] = 1; r = (uint16_t)(r | 0x8000u); }
                }
        }
    }
    auto &nrec = T.nrec;
    nrec.assign((size_t)h.nn, make_int4(0, 0, 0, 0));
    for (int64_t i = 0; i < h.nn; i++) {
        const int64_t n = order[(size_t)i], off = h.node_off[(size_t)n];
        const int32_t deg = (int32_t)(h.node_off[(size_t)n + 1] - off), q0 = h.inc_ptr[(size_t)n],
                      cnt = h.inc_ptr[(size_t)n + 1] - q0;
        nrec[(size_t)i] =
            make_int4((int)(uint32_t)off, (int)(off >> 32), q0, (int)(((uint32_t)cnt << 16) | (uint32_t)deg));
    }
    return true;
}

static soptx_status setup_contract_rows(soptx_mesh_s &m, const RefElement &ref, cudaStream_t st)
{
    const HostMesh &h = m.h;
    const int d = h.dim, nb = h.nb, ng = d * d + 1, n4 = d == 3 ? 3 : 2, mp = d == 3 ? 12 : 4;
    RowTables T;
    if (!build_row_tables(h, T)) return SOPTX_OK;
    std::vector<float4> cg((size_t)h.nc * n4, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int64_t e = 0; e < h.nc; e++) {
        float *dst = reinterpret_cast<float *>(&cg[(size_t)e * n4]);
        for (int t = 0; t < ng; t++) dst[t] = (float)h.geo[(size_t)e * ng + t];
    }
    std::vector<float> mf((size_t)nb * nb * mp, 0.f);
    for (int a = 0; a < nb; a++)
        for (int b = 0; b < nb; b++)
            for (int k = 0; k < d; k++)
                for (int l = 0; l < d; l++)
                    mf[((size_t)a * nb + b) * mp + k * d + l] = (float)ref.M[(((size_t)k * d + l) * nb + a) * nb + b];
    soptx_status s = upload(&m.d.cgeo, cg, st, m.device_bytes, "cell geometry");
    if (s == SOPTX_OK) s = upload(&m.d.Mf, mf, st, m.device_bytes, "reference integrals (FP32)");
    if (s == SOPTX_OK) s = upload(&m.d.cnrec, T.nrec, st, m.device_bytes, "node records");
    if (s == SOPTX_OK) s = upload(&m.d.cinc_e, T.ce, st, m.device_bytes, "contraction cell chains");
    if (s == SOPTX_OK) s = upload(&m.d.cinc_a, T.ca, st, m.device_bytes, "contraction local indices");
    if (s == SOPTX_OK) s = upload(&m.d.crec, T.rec, st, m.device_bytes, "contraction lane records");
    if (s == SOPTX_OK) s = upload(&m.d.cticket, std::vector<unsigned>(2, 0u), st, m.device_bytes, "round counter");
    if (s == SOPTX_OK) m.d.contract = true;
    return s;
}

// FP32 element matrices of affine cells: the tables of the per-call contraction.
static soptx_status setup_contract(soptx_mesh_s &m, const RefElement &ref, cudaStream_t st)
{
    return m.h.dim == 2 ? setup_contract_pairs(m, ref, st, false) : setup_contract_rows(m, ref, st);
}

static bool material_ok(const soptx_material *m, int dim, Material &out, std::string &err)
{
    if (!m) { err = "material is NULL"; return false; }
    if (!std::isfinite(m->E0) || !std::isfinite(m->Emin) || !std::isfinite(m->nu) || !std::isfinite(m->p)) {
        err = "material parameters must be finite";
        return false;
    }
    if (!(m->Emin >= 0.0) || !(m->E0 > m->Emin)) { err = "need E0 > Emin >= 0"; return false; }
    if (!(m->nu > -1.0 && m->nu < 0.5)) { err = "need -1 < nu < 0.5"; return false; }
    if (!(m->p >= 1.0)) { err = "need p >= 1"; return false; }
    out.E0 = m->E0;
    out.Emin = m->Emin;
    out.nu = m->nu;
    out.p = m->p;
    out.dE = m->E0 - m->Emin;
    out.p_int = (m->p == std::floor(m->p) && m->p <= 16.0) ? (int)m->p : 0;
    const double nu = m->nu;
    out.mu = 1.0 / (2.0 * (1.0 + nu));
    if (dim == 2 && !m->plane_strain) out.lam = nu / (1.0 - nu * nu);      // plane stress lambda*
    else out.lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    return true;
}

}  // namespace soptx

using namespace soptx;

extern "C" {

const char *soptx_last_error(void) { return g_last_error.c_str(); }
const char *soptx_version(void) { return "soptx-gb300 0.1 (sm_103a)"; }
void soptx_debug_fail_alloc_after(int64_t n) { g_fail_after.store(n > 0 ? n : 0); }
void soptx_debug_lattice_no_sectors(int32_t enable) { g_no_sectors.store(enable ? 1 : 0); }

soptx_status soptx_mesh_create(int dim, soptx_cell cell, int order, int64_t n_vertices, const double *coords,
                               int64_t n_cells, const int32_t *cell_vertices, const soptx_material *mat,
                               soptx_elem_prec prec, void *stream, soptx_mesh *out)
{
    g_last_error.clear();
    if (!out) SOPTX_FAIL(SOPTX_EINVAL, "out is NULL");
    *out = nullptr;
    if ((int)cell < SOPTX_TRI || (int)cell > SOPTX_HEX) SOPTX_FAIL(SOPTX_EINVAL, "unknown cell type");
    if (cell_dim(cell) != dim) SOPTX_FAIL(SOPTX_EINVAL, "dim does not match the cell type");
    if (order < 1 || order > 3) SOPTX_FAIL(SOPTX_EINVAL, "order must be 1, 2 or 3");
    if (prec != SOPTX_ELEM_FP64 && prec != SOPTX_ELEM_FP32) SOPTX_FAIL(SOPTX_EINVAL, "unknown element precision");
    if (n_vertices < 1 || n_cells < 0) SOPTX_FAIL(SOPTX_EINVAL, "need n_vertices >= 1 and n_cells >= 0");
    if (n_vertices >= ((int64_t)1 << 31) || n_cells >= ((int64_t)1 << 31))
        SOPTX_FAIL(SOPTX_EINVAL, "vertex and cell counts must stay below 2^31");
    if (!coords || (n_cells > 0 && !cell_vertices)) SOPTX_FAIL(SOPTX_EINVAL, "coords / cell_vertices is NULL");
    Material mt;
    std::string err;
    if (!material_ok(mat, dim, mt, err)) SOPTX_FAIL(SOPTX_EINVAL, err);

    soptx_mesh_s *m = new (std::nothrow) soptx_mesh_s();
    if (!m) SOPTX_FAIL(SOPTX_ENOMEM, "host allocation failed");
    m->mat = mt;
    m->user_mat = *mat;
    m->prec = prec;
    RefElement ref;
    try {
        if (!build_ref_element(cell, order, ref, err) ||
            !setup_host_mesh(dim, cell, order, n_vertices, coords, n_cells, cell_vertices, ref, m->h, err)) {
            delete m;
            SOPTX_FAIL(SOPTX_EINVAL, err);
        }
    } catch (const std::bad_alloc &) {
        delete m;
        SOPTX_FAIL(SOPTX_ENOMEM, "host allocation failed during mesh setup");
    }
    HostMesh &h = m->h;
    m->path = h.lattice ? SOPTX_PATH_LATTICE : (h.uniform ? SOPTX_PATH_UNIFORM : SOPTX_PATH_CACHED);

    cudaStream_t st = (cudaStream_t)stream;
    soptx_status s = SOPTX_OK;
    int64_t &B = m->device_bytes;
    std::vector<int64_t> indptr;
    std::vector<int32_t> indices;
    try {
        build_csr(h, indptr, indices);
    } catch (const std::bad_alloc &) {
        delete m;
        SOPTX_FAIL(SOPTX_ENOMEM, "host allocation failed building the CSR pattern");
    }
    DeviceMesh &d = m->d;
#define UP(dst, src, what)                                  \
    if (s == SOPTX_OK) s = upload(&(dst), (src), st, B, what);
    UP(d.indptr, indptr, "indptr");
    UP(d.indices, indices, "indices");
    UP(d.cell_node, h.cell_node, "cell_node");
    UP(d.node_off, h.node_off, "node_off");
    UP(d.inc_ptr, h.inc_ptr, "inc_ptr");
    UP(d.inc, h.inc, "inc");
    UP(d.inc_e, h.inc_e, "inc_e");
    UP(d.inc_a, h.inc_a, "inc_a");
    UP(d.pos, h.pos, "pos");
    UP(d.M, ref.M, "reference integrals");
    if (h.nonaffine) {
        // general bilinear / trilinear cells: corner coordinates and the
        // reference Gauss rule with the basis gradients at its points
        RefQuad rq;
        build_tensor_quadrature(ref, rq);
        d.nq = rq.nq;
        UP(d.xcell, h.xcell, "corner coordinates");
        UP(d.qw, rq.w, "quadrature weights");
        UP(d.qdphi, rq.dphi, "basis gradients");
        UP(d.qdgeo, rq.dgeo, "vertex-basis gradients");
    }
#undef UP
    // geometry: all cells when cached, one otherwise
    if (s == SOPTX_OK) {
        std::vector<double> geo = h.geo;
        if (m->path != SOPTX_PATH_CACHED && h.nc > 0) geo.resize((size_t)(h.dim * h.dim + 1));
        s = upload(&d.geo, geo, st, B, "geometry");
    }
    const int64_t n_elem_mats = (m->path == SOPTX_PATH_CACHED) ? h.nc : (h.nc > 0 ? 1 : 0);
    if (s == SOPTX_OK) {
        size_t esz = (prec == SOPTX_ELEM_FP32) ? 4 : 8;   // float, or a float pair
        size_t bytes = (size_t)std::max<int64_t>(n_elem_mats, 1) * h.ldof * h.ldof * esz;
        cudaError_t e = dev_alloc(&d.K, bytes);
        if (e != cudaSuccess) { cudaGetLastError(); s = cuda_status(e, "element matrices"); }
        else B += (int64_t)bytes;
    }
    if (s == SOPTX_OK) {
        d.scratch_len = std::max<int64_t>(std::max<int64_t>(sensitivity_scratch_len(*m), lattice_sens_grid(h.nc)), 1);
        cudaError_t e = dev_alloc((void **)&d.scratch, d.scratch_len * sizeof(double));
        if (e != cudaSuccess) { cudaGetLastError(); s = cuda_status(e, "scratch"); }
        else B += d.scratch_len * (int64_t)sizeof(double);
    }
    if (s == SOPTX_OK) {
        cudaError_t e = dev_alloc((void **)&d.counter, 16);
        if (e == cudaSuccess) e = cudaMemsetAsync(d.counter, 0, 16, st);
        if (e != cudaSuccess) { cudaGetLastError(); s = cuda_status(e, "grid-sum ticket"); }
        else B += 16;
    }
    if (s == SOPTX_OK) s = cuda_status(launch_element_matrices(*m, n_elem_mats, st), "element matrices kernel");
    if (s == SOPTX_OK) s = cuda_status(cudaStreamSynchronize(st), "mesh setup");
    std::vector<double> K0;
    if (s == SOPTX_OK && m->path == SOPTX_PATH_LATTICE) {
        // the lattice kernels read one FP64 K^0, its reference blocks as float
        // pairs, and per-call element moduli
        const size_t n2 = (size_t)h.ldof * h.ldof;
        K0.assign(n2, 0.0);
        if (prec == SOPTX_ELEM_FP32) {
            std::vector<float> Kf(n2);
            s = cuda_status(cudaMemcpy(Kf.data(), d.K, n2 * sizeof(float), cudaMemcpyDeviceToHost), "K0");
            for (size_t q = 0; q < n2; q++) K0[q] = Kf[q];
        } else {
            std::vector<float2> Kp(n2);
            s = cuda_status(cudaMemcpy(Kp.data(), d.K, n2 * sizeof(float2), cudaMemcpyDeviceToHost), "K0");
            for (size_t q = 0; q < n2; q++) K0[q] = (double)Kp[q].x + (double)Kp[q].y;
        }
        if (s == SOPTX_OK && !lattice_kappa_shift(h.dim, K0, h.lat_kshift)) m->path = SOPTX_PATH_UNIFORM;
    }
    if (s == SOPTX_OK && m->path == SOPTX_PATH_LATTICE) {
        std::vector<float2> kappa;
        build_lattice_kappa(h.dim, K0, h.lat_kshift, kappa);
        if (s == SOPTX_OK) s = upload(&d.K0, K0, st, B, "K0");
        if (s == SOPTX_OK) s = upload(&d.kappa, kappa, st, B, "kappa");
        std::vector<float2> sectors;
        // FP32 element matrices carry their rounding into K^0: zeros hold to about 2^-24 there
        const double zero_tol = prec == SOPTX_ELEM_FP32 ? 1e-5 : 1e-13;
        if (s == SOPTX_OK && !g_no_sectors.load() && build_lattice_sectors(h.dim, K0, zero_tol, sectors)) {
            s = upload(&d.sectors, sectors, st, B, "sectors");
            h.sectors = sectors;
        }
        if (s == SOPTX_OK) {
            cudaError_t e = dev_alloc((void **)&d.Edf, (size_t)std::max<int64_t>(h.nc, 1) * sizeof(float2));
            if (e != cudaSuccess) { cudaGetLastError(); s = cuda_status(e, "element moduli"); }
            else B += std::max<int64_t>(h.nc, 1) * (int64_t)sizeof(float2);
        }
        if (s == SOPTX_OK) {
            const size_t bytes = 16;
            cudaError_t e = dev_alloc((void **)&d.lat_bad, bytes);
            if (e == cudaSuccess) e = cudaMemsetAsync(d.lat_bad, 0, bytes, st);
            if (e != cudaSuccess) { cudaGetLastError(); s = cuda_status(e, "out-of-range flag"); }
            else B += (int64_t)bytes;
        }
        if (s == SOPTX_OK && d.sectors) {
            // u as float pairs, made once per call by the one-call step
            cudaError_t e = dev_alloc((void **)&d.udf, (size_t)std::max<int64_t>(h.ndof, 1) * sizeof(float2));
            if (e != cudaSuccess) { cudaGetLastError(); s = cuda_status(e, "displacement pairs"); }
            else B += std::max<int64_t>(h.ndof, 1) * (int64_t)sizeof(float2);
        }
        if (s == SOPTX_OK) s = cuda_status(cudaStreamSynchronize(st), "mesh setup");
    }
    if (s == SOPTX_OK && m->path != SOPTX_PATH_LATTICE && !h.nonaffine && h.nc > 0) {
        // affine cells off the lattice: the sensitivities from the strain energy at
        // the points of a rule exact for it (G and |det J| per cell as float pairs,
        // the weights and reference gradients of the rule)
        s = setup_strain(*m, ref, st);
        // FP32 element matrices: the assembly contracts the reference integrals with
        // each cell's Jacobian per call (FP32 tables), the cache is not read
        if (s == SOPTX_OK && prec == SOPTX_ELEM_FP32 && m->path == SOPTX_PATH_CACHED &&
            contract_fits(h.dim, h.nb, h.max_deg))
            s = setup_contract(*m, ref, st);
        // FP64 element matrices of 2D cells: the pair kernel reads each node pair's
        // blocks of the cache once for both row blocks
        if (s == SOPTX_OK && prec == SOPTX_ELEM_FP64 && m->path == SOPTX_PATH_CACHED && h.dim == 2 &&
            contract_fits(h.dim, h.nb, h.max_deg))
            s = setup_contract_pairs(*m, ref, st, true);
        // FP64 element matrix of a uniform mesh (boxes of order 2 and 3): the pair
        // kernel reads its blocks through L1
        if (s == SOPTX_OK && prec == SOPTX_ELEM_FP64 && m->path == SOPTX_PATH_UNIFORM &&
            pairs_fit(h.dim, h.nb, h.max_deg))
            s = setup_contract_pairs(*m, ref, st, false, true);
    }
    if (s == SOPTX_OK && (m->path != SOPTX_PATH_LATTICE || !d.sectors)) {
        // per-call float-pair moduli and displacements, per-(cell, node) partials
        // of the general path (also the sensitivity of a lattice whose element
        // matrix does not split into Walsh sectors)
        void *p1 = nullptr, *p2 = nullptr, *p3 = nullptr;
        cudaError_t e = d.Edf ? cudaSuccess : dev_alloc(&p1, (size_t)std::max<int64_t>(h.nc, 1) * sizeof(float2));
        if (e == cudaSuccess) e = dev_alloc(&p2, (size_t)std::max<int64_t>(h.ndof, 1) * sizeof(float2));
        if (e == cudaSuccess) e = dev_alloc(&p3, (size_t)std::max<int64_t>(h.nc * h.nb, 1) * sizeof(double));
        if (!d.Edf) d.Edf = (float2 *)p1;
        d.udf = (float2 *)p2;
        d.part = (double *)p3;
        if (e != cudaSuccess) { cudaGetLastError(); s = cuda_status(e, "general-path scratch"); }
        else B += (p1 ? std::max<int64_t>(h.nc, 1) * 8 : 0) + std::max<int64_t>(h.ndof, 1) * 8 +
                  std::max<int64_t>(h.nc * h.nb, 1) * 8;
    }
    if (s != SOPTX_OK) {
        std::string msg = g_last_error;
        cudaStreamSynchronize(st);
        free_device(m->d);
        delete m;
        set_error(msg);
        return s;
    }
    // host copies that the kernels do not need any more
    std::vector<uint16_t>().swap(h.pos);
    std::vector<int32_t>().swap(h.inc);
    std::vector<int32_t>().swap(h.inc_e);
    std::vector<uint8_t>().swap(h.inc_a);
    std::vector<double>().swap(h.xcell);
    *out = m;
    return SOPTX_OK;
}

// The validation, numbering and pattern of soptx_mesh_create, on the host.
static soptx_status plan_on_host(int dim, soptx_cell cell, int order, int64_t n_vertices, const double *coords,
                                 int64_t n_cells, const int32_t *cell_vertices, RefElement &ref, HostMesh &h)
{
    g_last_error.clear();
    if ((int)cell < SOPTX_TRI || (int)cell > SOPTX_HEX) SOPTX_FAIL(SOPTX_EINVAL, "unknown cell type");
    if (cell_dim(cell) != dim) SOPTX_FAIL(SOPTX_EINVAL, "dim does not match the cell type");
    if (order < 1 || order > 3) SOPTX_FAIL(SOPTX_EINVAL, "order must be 1, 2 or 3");
    if (n_vertices < 1 || n_cells < 0) SOPTX_FAIL(SOPTX_EINVAL, "need n_vertices >= 1 and n_cells >= 0");
    if (!coords || (n_cells > 0 && !cell_vertices)) SOPTX_FAIL(SOPTX_EINVAL, "coords / cell_vertices is NULL");
    std::string err;
    if (!build_ref_element(cell, order, ref, err) ||
        !setup_host_mesh(dim, cell, order, n_vertices, coords, n_cells, cell_vertices, ref, h, err))
        SOPTX_FAIL(SOPTX_EINVAL, err);
    return SOPTX_OK;
}

soptx_status soptx_host_plan(int dim, soptx_cell cell, int order, int64_t n_vertices, const double *coords,
                             int64_t n_cells, const int32_t *cell_vertices, int64_t *ndof, int64_t *nnz,
                             int32_t *nb, soptx_path *path, int64_t *indptr, int32_t *indices,
                             int32_t *cell_nodes)
{
    RefElement ref;
    HostMesh h;
    try {
        const soptx_status s = plan_on_host(dim, cell, order, n_vertices, coords, n_cells, cell_vertices, ref, h);
        if (s != SOPTX_OK) return s;
        if (ndof) *ndof = h.ndof;
        if (nnz) *nnz = h.nnz;
        if (nb) *nb = h.nb;
        if (path) *path = h.lattice ? SOPTX_PATH_LATTICE : (h.uniform ? SOPTX_PATH_UNIFORM : SOPTX_PATH_CACHED);
        if (indptr || indices) {
            std::vector<int64_t> ip;
            std::vector<int32_t> ix;
            build_csr(h, ip, ix);
            if (indptr) std::memcpy(indptr, ip.data(), ip.size() * sizeof(int64_t));
            if (indices && !ix.empty()) std::memcpy(indices, ix.data(), ix.size() * sizeof(int32_t));
        }
        if (cell_nodes && !h.cell_node.empty())
            std::memcpy(cell_nodes, h.cell_node.data(), h.cell_node.size() * sizeof(int32_t));
    } catch (const std::bad_alloc &) {
        SOPTX_FAIL(SOPTX_ENOMEM, "host allocation failed");
    }
    return SOPTX_OK;
}

soptx_status soptx_host_pair_tables(int dim, soptx_cell cell, int order, int64_t n_vertices, const double *coords,
                                    int64_t n_cells, const int32_t *cell_vertices, int32_t local_pair_bytes,
                                    int64_t *n_tiles, int64_t *n_records, uint32_t *tile_offsets,
                                    uint32_t *pair_block, uint32_t *pair_block_t, uint32_t *pair_meta,
                                    int32_t *record_cell, uint16_t *record_pair)
{
    RefElement ref;
    HostMesh h;
    try {
        const soptx_status s = plan_on_host(dim, cell, order, n_vertices, coords, n_cells, cell_vertices, ref, h);
        if (s != SOPTX_OK) return s;
        PairTables T;
        if (!pairs_fit(h.dim, h.nb, h.max_deg) || !build_pair_tables(h, local_pair_bytes != 0, T)) {
            if (n_tiles) *n_tiles = -1;
            if (n_records) *n_records = 0;
            return SOPTX_OK;
        }
        const int64_t nt = T.ntiles, nrec = (int64_t)T.toff[(size_t)nt] * 32;
        if (n_tiles) *n_tiles = nt;
        if (n_records) *n_records = nrec;
        if (tile_offsets) std::memcpy(tile_offsets, T.toff.data(), (size_t)(nt + 1) * sizeof(uint32_t));
        if (pair_block && nt) std::memcpy(pair_block, T.ia.data(), (size_t)nt * 32 * sizeof(uint32_t));
        if (pair_block_t && nt) std::memcpy(pair_block_t, T.ib.data(), (size_t)nt * 32 * sizeof(uint32_t));
        if (pair_meta && nt) std::memcpy(pair_meta, T.meta.data(), (size_t)nt * 32 * sizeof(uint32_t));
        if (record_cell && nrec) std::memcpy(record_cell, T.re.data(), (size_t)nrec * sizeof(int32_t));
        if (record_pair && nrec) std::memcpy(record_pair, T.rm.data(), (size_t)nrec * sizeof(uint16_t));
    } catch (const std::bad_alloc &) {
        SOPTX_FAIL(SOPTX_ENOMEM, "host allocation failed");
    }
    return SOPTX_OK;
}

soptx_status soptx_host_row_tables(int dim, soptx_cell cell, int order, int64_t n_vertices, const double *coords,
                                   int64_t n_cells, const int32_t *cell_vertices, int64_t *n_nodes,
                                   int64_t *n_incidences, int32_t *nb, int32_t *node_records, int32_t *chain_cell,
                                   uint8_t *chain_local, uint16_t *lane_records)
{
    RefElement ref;
    HostMesh h;
    try {
        const soptx_status s = plan_on_host(dim, cell, order, n_vertices, coords, n_cells, cell_vertices, ref, h);
        if (s != SOPTX_OK) return s;
        if (nb) *nb = h.nb;
        RowTables T;
        if (h.dim != 3 || !contract_fits(h.dim, h.nb, h.max_deg) || !build_row_tables(h, T)) {
            if (n_nodes) *n_nodes = -1;
            if (n_incidences) *n_incidences = 0;
            return SOPTX_OK;
        }
        const int64_t ninc = (int64_t)T.ce.size();
        if (n_nodes) *n_nodes = h.nn;
        if (n_incidences) *n_incidences = ninc;
        if (node_records && h.nn) std::memcpy(node_records, T.nrec.data(), (size_t)h.nn * sizeof(int4));
        if (chain_cell && ninc) std::memcpy(chain_cell, T.ce.data(), (size_t)ninc * sizeof(int32_t));
        if (chain_local && ninc) std::memcpy(chain_local, T.ca.data(), (size_t)ninc * sizeof(uint8_t));
        if (lane_records && ninc) std::memcpy(lane_records, T.rec.data(), (size_t)ninc * h.nb * sizeof(uint16_t));
    } catch (const std::bad_alloc &) {
        SOPTX_FAIL(SOPTX_ENOMEM, "host allocation failed");
    }
    return SOPTX_OK;
}

soptx_status soptx_mesh_info(soptx_mesh m, int64_t *ndof, int64_t *nnz, int64_t *n_cells, int32_t *ldof)
{
    if (!m) SOPTX_FAIL(SOPTX_EINVAL, "mesh is NULL");
    if (ndof) *ndof = m->h.ndof;
    if (nnz) *nnz = m->h.nnz;
    if (n_cells) *n_cells = m->h.nc;
    if (ldof) *ldof = m->h.ldof;
    return SOPTX_OK;
}

soptx_status soptx_mesh_pattern(soptx_mesh m, const int64_t **d_indptr, const int32_t **d_indices)
{
    if (!m) SOPTX_FAIL(SOPTX_EINVAL, "mesh is NULL");
    if (d_indptr) *d_indptr = m->d.indptr;
    if (d_indices) *d_indices = m->d.indices;
    return SOPTX_OK;
}

soptx_status soptx_mesh_cell_nodes(soptx_mesh m, const int32_t **d_cell_nodes, int32_t *nb)
{
    if (!m) SOPTX_FAIL(SOPTX_EINVAL, "mesh is NULL");
    if (d_cell_nodes) *d_cell_nodes = m->d.cell_node;
    if (nb) *nb = m->h.nb;
    return SOPTX_OK;
}

soptx_status soptx_mesh_copy_pattern(soptx_mesh m, int64_t *d_indptr, int32_t *d_indices, void *stream)
{
    if (!m) SOPTX_FAIL(SOPTX_EINVAL, "mesh is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (d_indptr) {
        soptx_status s = cuda_status(cudaMemcpyAsync(d_indptr, m->d.indptr, (m->h.ndof + 1) * sizeof(int64_t),
                                                     cudaMemcpyDeviceToDevice, st), "copy indptr");
        if (s != SOPTX_OK) return s;
    }
    if (d_indices && m->h.nnz > 0)
        return cuda_status(cudaMemcpyAsync(d_indices, m->d.indices, m->h.nnz * sizeof(int32_t),
                                           cudaMemcpyDeviceToDevice, st), "copy indices");
    return SOPTX_OK;
}

soptx_status soptx_mesh_copy_cell_nodes(soptx_mesh m, int32_t *d_cell_nodes, void *stream)
{
    if (!m || !d_cell_nodes) SOPTX_FAIL(SOPTX_EINVAL, "mesh or d_cell_nodes is NULL");
    if (m->h.nc == 0) return SOPTX_OK;
    return cuda_status(cudaMemcpyAsync(d_cell_nodes, m->d.cell_node, m->h.nc * m->h.nb * sizeof(int32_t),
                                       cudaMemcpyDeviceToDevice, (cudaStream_t)stream), "copy cell nodes");
}

soptx_status soptx_mesh_path(soptx_mesh m, soptx_path *path)
{
    if (!m || !path) SOPTX_FAIL(SOPTX_EINVAL, "mesh or path is NULL");
    *path = m->path;
    return SOPTX_OK;
}

soptx_status soptx_mesh_routes(soptx_mesh m, int32_t *assembly, int32_t *sensitivity)
{
    if (!m) SOPTX_FAIL(SOPTX_EINVAL, "mesh is NULL");
    if (assembly)
        *assembly = m->path == SOPTX_PATH_LATTICE ? 0 : m->d.contract ? 2 : (m->d.pcached || m->d.puniform) ? 3 : 1;
    if (sensitivity) *sensitivity = (m->path == SOPTX_PATH_LATTICE && m->d.sectors) ? 0 : (m->d.strain ? 2 : 1);
    return SOPTX_OK;
}

soptx_status soptx_mesh_device_bytes(soptx_mesh m, int64_t *bytes)
{
    if (!m || !bytes) SOPTX_FAIL(SOPTX_EINVAL, "mesh or bytes is NULL");
    *bytes = m->device_bytes;
    return SOPTX_OK;
}

soptx_status soptx_assemble_K(soptx_mesh m, const double *d_rho, double *d_vals, void *stream)
{
    if (!m) SOPTX_FAIL(SOPTX_EINVAL, "mesh is NULL");
    if ((!d_rho && m->h.nc > 0) || (!d_vals && m->h.nnz > 0)) SOPTX_FAIL(SOPTX_EINVAL, "d_rho / d_vals is NULL");
    return cuda_status(launch_assemble(*m, d_rho, d_vals, (cudaStream_t)stream), "soptx_assemble_K");
}

soptx_status soptx_sensitivity(soptx_mesh m, const double *d_rho, const double *d_u, double *d_dc, double *d_c,
                               void *stream)
{
    if (!m) SOPTX_FAIL(SOPTX_EINVAL, "mesh is NULL");
    if (m->h.nc > 0 && (!d_rho || !d_u || !d_dc)) SOPTX_FAIL(SOPTX_EINVAL, "d_rho / d_u / d_dc is NULL");
    return cuda_status(launch_sensitivity(*m, d_rho, d_u, d_dc, d_c, -1.0, nullptr, (cudaStream_t)stream),
                       "soptx_sensitivity");
}

soptx_status soptx_assemble_and_sensitivity(soptx_mesh m, const double *d_rho, const double *d_u, double *d_vals,
                                            double *d_dc, double *d_c, void *stream)
{
    if (!m) SOPTX_FAIL(SOPTX_EINVAL, "mesh is NULL");
    if ((!d_vals && m->h.nnz > 0) || (m->h.nc > 0 && (!d_rho || !d_u || !d_dc)))
        SOPTX_FAIL(SOPTX_EINVAL, "d_rho / d_u / d_vals / d_dc is NULL");
    if (((m->path == SOPTX_PATH_LATTICE && m->h.dim == 2 && m->d.sectors) || m->d.strain) && m->h.nc > 0) {
        cudaError_t e = ensure_side(*m);
        if (e != cudaSuccess) return cuda_status(e, "soptx_assemble_and_sensitivity stream");
    }
    return cuda_status(launch_step(*m, d_rho, d_u, d_vals, d_dc, d_c, (cudaStream_t)stream),
                       "soptx_assemble_and_sensitivity");
}

soptx_status soptx_assemble_and_sensitivity_group(int32_t n, const soptx_mesh *meshes, const double *const *d_rho,
                                                  const double *const *d_u, double *const *d_vals,
                                                  double *const *d_dc, double *const *d_c, void *stream)
{
    if (n < 0) SOPTX_FAIL(SOPTX_EINVAL, "n must be >= 0");
    if (n == 0) return SOPTX_OK;
    if (!meshes || !d_rho || !d_u || !d_vals || !d_dc || !d_c) SOPTX_FAIL(SOPTX_EINVAL, "an argument array is NULL");
    std::vector<const soptx_mesh_s *> grp;
    std::vector<const double *> gr, gu;
    std::vector<double *> gv, gd, gc;
    for (int32_t k = 0; k < n; k++) {
        soptx_mesh m = meshes[k];
        if (!m) SOPTX_FAIL(SOPTX_EINVAL, "mesh is NULL");
        for (int32_t k2 = 0; k2 < k; k2++)
            if (meshes[k2] == m) SOPTX_FAIL(SOPTX_EINVAL, "a mesh appears twice in the group");
        if ((!d_vals[k] && m->h.nnz > 0) || (m->h.nc > 0 && (!d_rho[k] || !d_u[k] || !d_dc[k])))
            SOPTX_FAIL(SOPTX_EINVAL, "d_rho / d_u / d_vals / d_dc is NULL");
    }
    for (int32_t k = 0; k < n; k++) {
        soptx_mesh m = meshes[k];
        if (lattice_groupable(*m)) {
            grp.push_back(m);
            gr.push_back(d_rho[k]);
            gu.push_back(d_u[k]);
            gv.push_back(d_vals[k]);
            gd.push_back(d_dc[k]);
            gc.push_back(d_c[k]);
            continue;
        }
        soptx_status s = soptx_assemble_and_sensitivity(m, d_rho[k], d_u[k], d_vals[k], d_dc[k], d_c[k], stream);
        if (s != SOPTX_OK) return s;
    }
    if (grp.empty()) return SOPTX_OK;
    return cuda_status(launch_lattice_group(grp.data(), gr.data(), gu.data(), gv.data(), gd.data(), gc.data(),
                                            (int)grp.size(), (cudaStream_t)stream),
                       "soptx_assemble_and_sensitivity_group");
}

soptx_status soptx_step_host(soptx_mesh m, const double *h_rho, const double *h_u, double *d_vals, double *h_dc,
                             double *h_c, void *stream)
{
    if (!m) SOPTX_FAIL(SOPTX_EINVAL, "mesh is NULL");
    const auto &h = m->h;
    if ((!d_vals && h.nnz > 0) || (h.nc > 0 && !h_dc) || (h.nc > 0 && !h_rho) || (h.ndof > 0 && !h_u))
        SOPTX_FAIL(SOPTX_EINVAL, "h_rho / h_u / d_vals / h_dc is NULL");
    auto &d = m->d;
    cudaError_t e = cudaSuccess;
    if (!d.stage) {
        const size_t bytes = (size_t)(2 * h.nc + h.ndof + 1) * sizeof(double);
        void *p = nullptr;
        e = dev_alloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_status(e, "soptx_step_host staging");
        }
        d.stage = (double *)p;
        m->device_bytes += (int64_t)bytes;
    }
    e = ensure_side(*m);
    if (e != cudaSuccess) return cuda_status(e, "soptx_step_host stream");
    cudaStream_t st = (cudaStream_t)stream;
    double *rho_d = d.stage, *u_d = rho_d + h.nc, *dc_d = u_d + h.ndof, *c_d = dc_d + h.nc;
    const size_t rb = (size_t)h.nc * sizeof(double), ub = (size_t)h.ndof * sizeof(double);
    // dc and c back: one copy when the caller's c follows its dc
    auto copy_back = [&](cudaStream_t s) -> cudaError_t {
        if (h_dc && h_c && h_c == h_dc + h.nc)
            return cudaMemcpyAsync(h_dc, dc_d, rb + sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaError_t r = rb ? cudaMemcpyAsync(h_dc, dc_d, rb, cudaMemcpyDeviceToHost, s) : cudaSuccess;
        if (r == cudaSuccess && h_c) r = cudaMemcpyAsync(h_c, c_d, sizeof(double), cudaMemcpyDeviceToHost, s);
        return r;
    };
#define SOPTX_TRY(x)                                                            \
    do {                                                                        \
        e = (x);                                                                \
        if (e != cudaSuccess) return cuda_status(e, "soptx_step_host");         \
    } while (0)
    if (m->path == SOPTX_PATH_LATTICE && d.sectors && h.nc > 0) {
        // the sensitivities need rho and u but not K: they run on the side stream
        // while the moduli and the assembly run on `stream`.  rho goes first (the
        // assembly waits for it); u's copy follows it and overlaps the assembly.
        SOPTX_TRY(cudaMemcpyAsync(rho_d, h_rho, rb, cudaMemcpyHostToDevice, st));
        SOPTX_TRY(cudaEventRecord(d.ev[0], st));
        SOPTX_TRY(cudaStreamWaitEvent(d.side, d.ev[0], 0));
        SOPTX_TRY(cudaMemcpyAsync(u_d, h_u, ub, cudaMemcpyHostToDevice, d.side));
        SOPTX_TRY(launch_lattice_sensitivity(*m, rho_d, u_d, dc_d, c_d, nullptr, d.side));
        SOPTX_TRY(copy_back(d.side));
        SOPTX_TRY(cudaEventRecord(d.ev[1], d.side));
        SOPTX_TRY(launch_lattice_assemble(*m, rho_d, d_vals, st));
        SOPTX_TRY(cudaStreamWaitEvent(st, d.ev[1], 0));
    } else {
        if (rb) SOPTX_TRY(cudaMemcpyAsync(rho_d, h_rho, rb, cudaMemcpyHostToDevice, st));
        if (ub) SOPTX_TRY(cudaMemcpyAsync(u_d, h_u, ub, cudaMemcpyHostToDevice, st));
        SOPTX_TRY(launch_step(*m, rho_d, u_d, d_vals, dc_d, c_d, st));
        SOPTX_TRY(copy_back(st));
    }
#undef SOPTX_TRY
    return SOPTX_OK;
}

soptx_status soptx_compliance_vjp(soptx_mesh m, const double *d_rho, const double *d_u, const double *d_gout,
                                  double *d_grad_rho, double *d_grad_u, void *stream)
{
    if (!m) SOPTX_FAIL(SOPTX_EINVAL, "mesh is NULL");
    if (!d_gout) SOPTX_FAIL(SOPTX_EINVAL, "d_gout is NULL");
    if (m->h.nc > 0 && (!d_rho || !d_u || !d_grad_rho)) SOPTX_FAIL(SOPTX_EINVAL, "d_rho / d_u / d_grad_rho is NULL");
    if (d_grad_u && m->h.ndof > 0 && !d_u) SOPTX_FAIL(SOPTX_EINVAL, "d_u is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    auto &d = m->d;
    if (d_grad_u && !d.kvals && m->h.nnz > 0) {
        // K(rho) for 2 g K(rho) u goes into a mesh-owned scratch of 8 nnz bytes, made once;
        // where that memory cannot be had the product is formed matrix-free instead
        void *p = nullptr;
        if (dev_alloc(&p, (size_t)m->h.nnz * sizeof(double)) == cudaSuccess) {
            d.kvals = (double *)p;
            m->device_bytes += (int64_t)m->h.nnz * (int64_t)sizeof(double);
        } else {
            cudaGetLastError();
        }
    }
    if (d_grad_u && m->h.nnz == 0) {
        // no element couples any dof: K(rho) = 0
        soptx_status s = cuda_status(launch_sensitivity(*m, d_rho, d_u, d_grad_rho, nullptr, 1.0, d_gout, st),
                                     "soptx_compliance_vjp");
        if (s != SOPTX_OK || m->h.ndof == 0) return s;
        return cuda_status(cudaMemsetAsync(d_grad_u, 0, (size_t)m->h.ndof * sizeof(double), st),
                           "soptx_compliance_vjp");
    }
    if (d_grad_u && d.kvals) {
        // one step (K(rho) and the rho-gradient g E' s) then the product with u
        soptx_status s = cuda_status(launch_step(*m, d_rho, d_u, d.kvals, d_grad_rho, nullptr, st, d_gout),
                                     "soptx_compliance_vjp");
        if (s != SOPTX_OK) return s;
        return cuda_status(launch_scaled_product(*m, d.kvals, d_u, d_gout, d_grad_u, st), "soptx_compliance_vjp");
    }
    soptx_status s = cuda_status(launch_sensitivity(*m, d_rho, d_u, d_grad_rho, nullptr, 1.0, d_gout, st),
                                 "soptx_compliance_vjp");
    if (s != SOPTX_OK || !d_grad_u) return s;
    return cuda_status(launch_Ku(*m, d_rho, d_u, d_gout, d_grad_u, st), "soptx_compliance_vjp");
}

soptx_status soptx_mesh_destroy(soptx_mesh m)
{
    if (!m) return SOPTX_OK;
    cudaDeviceSynchronize();
    free_device(m->d);
    delete m;
    return SOPTX_OK;
}

}  // extern "C"
