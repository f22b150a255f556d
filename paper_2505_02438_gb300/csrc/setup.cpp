// Host-side mesh setup, done once per mesh (the counterpart of the paper's
// "1st assembly", Sec. 5.5): validation, per-cell geometry, Lagrange node
// numbering, the CSR pattern and the gather maps the kernels use.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace soptx {
namespace {

// Local vertex set (bitmask over the cell's vertices) of the entity carrying
// local node a, and that entity's dimension.
void classify(const RefElement &ref, int a, unsigned &mask, int &edim)
{
    const int k = ref.order, dim = ref.dim, nvc = cell_nverts(ref.cell);
    mask = 0;
    if (is_simplex(ref.cell)) {
        int lam[4] = {ref.lat[a][3], ref.lat[a][0], ref.lat[a][1], ref.lat[a][2]};
        int n = 0;
        for (int v = 0; v <= dim; v++)
            if (lam[v] > 0) { mask |= 1u << v; n++; }
        edim = n - 1;
    } else {
        int nfree = 0;
        for (int v = 0; v < nvc; v++) {
            bool ok = true;
            for (int m = 0; m < dim; m++) {
                int c = ref.lat[a][m], bit = (v >> m) & 1;
                if ((c == 0 && bit) || (c == k && !bit)) ok = false;
            }
            if (ok) mask |= 1u << v;
        }
        for (int m = 0; m < dim; m++)
            if (ref.lat[a][m] != 0 && ref.lat[a][m] != k) nfree++;
        edim = nfree;
    }
    (void)k;
}

// Sorted unique keys grouped by their first vertex (CSR over vertices).
struct EntityTable {
    int width = 0;                              // vertices per key
    std::vector<int64_t> ptr;                   // [nv+1]
    std::vector<std::array<int32_t, 3>> rest;   // remaining vertices, sorted per group
    void build(int64_t nv, int w, std::vector<std::array<int32_t, 4>> &keys)
    {
        width = w;
        std::sort(keys.begin(), keys.end());
        keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
        ptr.assign(nv + 1, 0);
        for (auto &x : keys) ptr[x[0] + 1]++;
        for (int64_t v = 0; v < nv; v++) ptr[v + 1] += ptr[v];
        rest.resize(keys.size());
        for (size_t i = 0; i < keys.size(); i++) rest[i] = {keys[i][1], keys[i][2], keys[i][3]};
    }
    int64_t find(const std::array<int32_t, 4> &key) const
    {
        std::array<int32_t, 3> r{key[1], key[2], key[3]};
        auto b = rest.begin() + ptr[key[0]], e = rest.begin() + ptr[key[0] + 1];
        auto it = std::lower_bound(b, e, r);
        return (it != e && *it == r) ? (int64_t)(it - rest.begin()) : -1;
    }
    int64_t size() const { return (int64_t)rest.size(); }
};

// The vertex ids of an edge or face (n <= 4) in ascending order, padded with -1.
std::array<int32_t, 4> sorted_key(const int32_t *v, int n)
{
    std::array<int32_t, 4> k{-1, -1, -1, -1};
    n = std::min(n, 4);
    for (int i = 0; i < n; i++) {
        int32_t x = v[i];
        int j = i;
        for (; j > 0 && k[j - 1] > x; j--) k[j] = k[j - 1];
        k[j] = x;
    }
    return k;
}

bool geometry(HostMesh &hm, const double *coords, const int32_t *cv, std::string &err)
{
    const int d = hm.dim, nvc = hm.nvc;
    const int ng = d * d + 1;
    hm.geo.assign((size_t)hm.nc * ng, 0.0);
    hm.uniform = hm.nc > 0;
    double J0[9] = {0};
    for (int64_t e = 0; e < hm.nc; e++) {
        const int32_t *c = cv + e * nvc;
        const double *x0 = coords + (int64_t)c[0] * d;
        double J[9] = {0};   // J[i*d + m] = d x_i / d xi_m
        for (int m = 0; m < d; m++) {
            int vm = is_simplex(hm.cell) ? m + 1 : (1 << m);
            const double *xm = coords + (int64_t)c[vm] * d;
            for (int i = 0; i < d; i++) J[i * d + m] = xm[i] - x0[i];
        }
        double scale = 0.0;
        for (int q = 0; q < d * d; q++) scale = std::max(scale, std::fabs(J[q]));
        if (!is_simplex(hm.cell)) {
            // affine check: every corner at x0 + sum_m bit_m J[:, m]; a general
            // (bilinear / trilinear) cell is integrated by Gauss quadrature
            bool affine = true;
            for (int v = 0; v < nvc && affine; v++) {
                const double *xv = coords + (int64_t)c[v] * d;
                for (int i = 0; i < d; i++) {
                    double want = x0[i];
                    for (int m = 0; m < d; m++)
                        if ((v >> m) & 1) want += J[i * d + m];
                    if (std::fabs(xv[i] - want) > 1e-10 * scale) affine = false;
                }
            }
            if (!affine) {
                // the Jacobian at every corner (edges toward the corner's
                // neighbours along each axis) must keep one sign
                hm.nonaffine = true;
                double sgn = 0.0;
                for (int v = 0; v < nvc; v++) {
                    double Jc[9];
                    const double *xv = coords + (int64_t)c[v] * d;
                    for (int m = 0; m < d; m++) {
                        const double *xn = coords + (int64_t)c[v ^ (1 << m)] * d;
                        const double s = ((v >> m) & 1) ? -1.0 : 1.0;
                        for (int i = 0; i < d; i++) Jc[i * d + m] = s * (xn[i] - xv[i]);
                    }
                    const double dc = d == 2 ? Jc[0] * Jc[3] - Jc[1] * Jc[2]
                                             : Jc[0] * (Jc[4] * Jc[8] - Jc[5] * Jc[7]) -
                                                   Jc[1] * (Jc[3] * Jc[8] - Jc[5] * Jc[6]) +
                                                   Jc[2] * (Jc[3] * Jc[7] - Jc[4] * Jc[6]);
                    if (!std::isfinite(dc) || std::fabs(dc) <= 1e-12 * std::pow(scale, d) ||
                        (sgn != 0.0 && (dc > 0.0) != (sgn > 0.0))) {
                        err = "cell " + std::to_string(e) + " is inverted or degenerate at corner " + std::to_string(v);
                        return false;
                    }
                    sgn = dc;
                }
            }
        }
        double det, G[9];
        if (d == 2) {
            det = J[0] * J[3] - J[1] * J[2];
            G[0] = J[3] / det; G[1] = -J[1] / det;
            G[2] = -J[2] / det; G[3] = J[0] / det;
        } else {
            double c00 = J[4] * J[8] - J[5] * J[7];
            double c01 = J[5] * J[6] - J[3] * J[8];
            double c02 = J[3] * J[7] - J[4] * J[6];
            det = J[0] * c00 + J[1] * c01 + J[2] * c02;
            // G = adj(J) / det, G[m*3 + i] = (J^-1)_{m i}
            G[0] = c00 / det;
            G[1] = (J[2] * J[7] - J[1] * J[8]) / det;
            G[2] = (J[1] * J[5] - J[2] * J[4]) / det;
            G[3] = c01 / det;
            G[4] = (J[0] * J[8] - J[2] * J[6]) / det;
            G[5] = (J[2] * J[3] - J[0] * J[5]) / det;
            G[6] = c02 / det;
            G[7] = (J[1] * J[6] - J[0] * J[7]) / det;
            G[8] = (J[0] * J[4] - J[1] * J[3]) / det;
        }
        if (!std::isfinite(det) || std::fabs(det) <= 1e-12 * std::pow(scale, d) || scale == 0.0) {
            err = "cell " + std::to_string(e) + " is degenerate (det J = " + std::to_string(det) + ")";
            return false;
        }
        double *g = &hm.geo[(size_t)e * ng];
        for (int q = 0; q < d * d; q++) g[q] = G[q];
        g[d * d] = std::fabs(det);
        // uniform: every Jacobian equals the first to within rounding of the
        // coordinates (1e-14 of its largest entry), so one K^0 serves all cells
        if (e == 0) {
            std::memcpy(J0, J, sizeof(J));
        } else if (hm.uniform) {
            double j0max = 0.0;
            for (int q = 0; q < d * d; q++) j0max = std::max(j0max, std::fabs(J0[q]));
            for (int q = 0; q < d * d; q++)
                if (std::fabs(J[q] - J0[q]) > 1e-14 * j0max) hm.uniform = false;
        }
    }
    if (hm.nonaffine) {
        hm.uniform = false;
        hm.xcell.resize((size_t)hm.nc * nvc * d);
        for (int64_t e = 0; e < hm.nc; e++)
            for (int v = 0; v < nvc; v++)
                for (int i = 0; i < d; i++)
                    hm.xcell[((size_t)e * nvc + v) * d + i] = coords[(int64_t)cv[e * nvc + v] * d + i];
    }
    return true;
}

// Order-1 box lattice in the canonical layout: vertices lexicographic (x
// fastest), cells lexicographic, corners lexicographic, axis-aligned boxes.
void detect_lattice(HostMesh &hm, const double *coords, const int32_t *cv)
{
    hm.lattice = false;
    if (hm.order != 1 || is_simplex(hm.cell) || !hm.uniform || hm.nc == 0) return;
    const int d = hm.dim, nvc = hm.nvc;
    const double *g = &hm.geo[0];
    for (int i = 0; i < d; i++)
        for (int m = 0; m < d; m++)
            if (i != m && g[i * d + m] != 0.0) return;   // J diagonal <=> G diagonal
    int64_t s1 = cv[1 << 1] - cv[0];
    int64_t n[3] = {s1 - 1, 1, 1};
    if (n[0] < 1 || cv[1] - cv[0] != 1) return;
    if (d == 3) {
        int64_t s2 = cv[1 << 2] - cv[0];
        if (s2 % s1) return;
        n[1] = s2 / s1 - 1;
        if (n[1] < 1) return;
        if (hm.nc % (n[0] * n[1])) return;
        n[2] = hm.nc / (n[0] * n[1]);
    } else {
        if (hm.nc % n[0]) return;
        n[1] = hm.nc / n[0];
    }
    int64_t nvl = 1;
    for (int m = 0; m < d; m++) nvl *= n[m] + 1;
    if (nvl != hm.nv || cv[0] != 0) return;
    // every cell's corners and every vertex's position
    for (int64_t e = 0; e < hm.nc; e++) {
        int64_t r = e, idx[3] = {0, 0, 0};
        for (int m = 0; m < d; m++) { idx[m] = r % n[m]; r /= n[m]; }
        for (int v = 0; v < nvc; v++) {
            int64_t vid = 0, stride = 1;
            for (int m = 0; m < d; m++) {
                vid += (idx[m] + ((v >> m) & 1)) * stride;
                stride *= n[m] + 1;
            }
            if (cv[e * nvc + v] != vid) return;
        }
    }
    double h[3], x0[3];
    for (int m = 0; m < d; m++) {
        x0[m] = coords[m];
        h[m] = coords[(int64_t)cv[1 << m] * d + m] - x0[m];
        if (!(h[m] > 0.0)) return;
    }
    for (int64_t v = 0; v < hm.nv; v++) {
        int64_t r = v;
        for (int m = 0; m < d; m++) {
            int64_t i = r % (n[m] + 1);
            r /= n[m] + 1;
            double want = x0[m] + (double)i * h[m];
            if (std::fabs(coords[v * d + m] - want) > 1e-12 * (std::fabs(want) + h[m])) return;
        }
    }
    for (int m = 0; m < 3; m++) hm.lat_n[m] = (int)n[m];
    hm.lattice = true;
}

}  // namespace

bool setup_host_mesh(int dim, int cell, int order, int64_t nv, const double *coords, int64_t nc,
                     const int32_t *cv, const RefElement &ref, HostMesh &hm, std::string &err)
{
    hm.dim = dim;
    hm.cell = cell;
    hm.order = order;
    hm.nb = ref.nb;
    hm.ldof = dim * ref.nb;
    hm.nvc = cell_nverts(cell);
    hm.nv = nv;
    hm.nc = nc;
    const int nb = ref.nb, nvc = hm.nvc, k = order;

    for (int64_t i = 0; i < nv * dim; i++)
        if (!std::isfinite(coords[i])) { err = "coordinates must be finite"; return false; }
    for (int64_t i = 0; i < nc * nvc; i++)
        if (cv[i] < 0 || cv[i] >= nv) {
            err = "cell_vertices[" + std::to_string(i) + "] = " + std::to_string(cv[i]) + " is out of range";
            return false;
        }
    for (int64_t e = 0; e < nc; e++)
        for (int a = 0; a < nvc; a++)
            for (int b = a + 1; b < nvc; b++)
                if (cv[e * nvc + a] == cv[e * nvc + b]) {
                    err = "cell " + std::to_string(e) + " repeats a vertex";
                    return false;
                }
    if (!geometry(hm, coords, cv, err)) return false;

    // ---- classify local nodes
    std::vector<unsigned> mask(nb);
    std::vector<int> edim(nb), interior_rank(nb, -1);
    int n_int = 0;
    for (int a = 0; a < nb; a++) {
        classify(ref, a, mask[a], edim[a]);
        if (edim[a] == dim) interior_rank[a] = n_int++;
    }
    auto verts_of = [&](int64_t e, unsigned msk, int32_t *out) {
        int n = 0;
        for (int v = 0; v < nvc; v++)
            if (msk >> v & 1) out[n++] = cv[e * nvc + v];
        return n;
    };

    // ---- edge and face tables
    EntityTable edges, faces;
    if (k > 1) {
        std::vector<std::array<int32_t, 4>> keys;
        keys.reserve((size_t)nc * 12);
        for (int64_t e = 0; e < nc; e++)
            for (int a = 0; a < nb; a++)
                if (edim[a] == 1) {
                    int32_t vv[8];
                    verts_of(e, mask[a], vv);
                    keys.push_back(sorted_key(vv, 2));
                }
        edges.build(nv, 2, keys);
        if (dim == 3) {
            keys.clear();
            for (int64_t e = 0; e < nc; e++)
                for (int a = 0; a < nb; a++)
                    if (edim[a] == 2) {
                        int32_t vv[8];
                        int n = verts_of(e, mask[a], vv);
                        keys.push_back(sorted_key(vv, n));
                    }
            faces.build(nv, is_simplex(cell) ? 3 : 4, keys);
        }
    }
    const int per_edge = k - 1;
    const int per_face = (dim == 3 && k > 1) ? (is_simplex(cell) ? (k - 1) * (k - 2) / 2 : (k - 1) * (k - 1)) : 0;
    const int64_t off_edge = nv;
    const int64_t off_face = off_edge + (k > 1 ? edges.size() * per_edge : 0);
    const int64_t off_int = off_face + (per_face ? faces.size() * per_face : 0);
    hm.nn = off_int + nc * n_int;
    hm.ndof = hm.nn * dim;
    if (hm.ndof >= ((int64_t)1 << 31) - 1) { err = "ndof must stay below 2^31"; return false; }
    if (nc * nb >= ((int64_t)1 << 31)) { err = "n_cells * nodes per cell must stay below 2^31"; return false; }

    // ---- cell -> node map
    hm.cell_node.assign((size_t)nc * nb, -1);
    for (int64_t e = 0; e < nc; e++) {
        const int32_t *g = cv + e * nvc;
        for (int a = 0; a < nb; a++) {
            int32_t &out = hm.cell_node[(size_t)e * nb + a];
            if (edim[a] == 0) {
                out = g[__builtin_ctz(mask[a])];
            } else if (edim[a] == dim) {
                out = (int32_t)(off_int + e * n_int + interior_rank[a]);
            } else if (edim[a] == 1) {
                int32_t vv[2];
                int lv[2], n = 0;
                for (int v = 0; v < nvc; v++)
                    if (mask[a] >> v & 1) { lv[n] = v; vv[n++] = g[v]; }
                int64_t id = edges.find(sorted_key(vv, 2));
                int hi = (g[lv[0]] > g[lv[1]]) ? lv[0] : lv[1];   // larger-id end
                int t;   // lattice steps from the smaller-id end
                if (is_simplex(cell)) {
                    t = (hi == 0) ? ref.lat[a][3] : ref.lat[a][hi - 1];
                } else {
                    int m = 0;
                    while (((lv[0] ^ lv[1]) >> m & 1) == 0) m++;
                    t = ((hi >> m) & 1) ? ref.lat[a][m] : k - ref.lat[a][m];
                }
                out = (int32_t)(off_edge + id * per_edge + (t - 1));
            } else {
                int32_t vv[4];
                int n = verts_of(e, mask[a], vv);
                int64_t id = faces.find(sorted_key(vv, n));
                int idx = 0;
                if (!is_simplex(cell)) {
                    // quad face of a hex: frame of the smallest-id corner o
                    int lo = -1;
                    for (int v = 0; v < nvc; v++)
                        if (mask[a] >> v & 1)
                            if (lo < 0 || g[v] < g[lo]) lo = v;
                    int ax[2], na = 0;
                    for (int m = 0; m < dim; m++)
                        if (ref.lat[a][m] != 0 && ref.lat[a][m] != k) ax[na++] = m;
                    int dist[2];
                    for (int q = 0; q < 2; q++)
                        dist[q] = ((lo >> ax[q]) & 1) ? k - ref.lat[a][ax[q]] : ref.lat[a][ax[q]];
                    int first = (g[lo ^ (1 << ax[0])] < g[lo ^ (1 << ax[1])]) ? 0 : 1;
                    idx = (dist[first] - 1) + (k - 1) * (dist[1 - first] - 1);
                }
                out = (int32_t)(off_face + id * per_face + idx);
            }
        }
    }

    // ---- node -> (cell, local) incidence, ascending cell
    hm.inc_ptr.assign(hm.nn + 1, 0);
    for (int64_t i = 0; i < nc * nb; i++) hm.inc_ptr[hm.cell_node[i] + 1]++;
    for (int64_t n = 0; n < hm.nn; n++) hm.inc_ptr[n + 1] += hm.inc_ptr[n];
    hm.ninc = nc * nb;
    hm.inc.assign(hm.ninc, 0);
    {
        std::vector<int32_t> fill(hm.inc_ptr.begin(), hm.inc_ptr.end() - 1);
        for (int64_t e = 0; e < nc; e++)
            for (int a = 0; a < nb; a++) {
                int32_t n = hm.cell_node[(size_t)e * nb + a];
                hm.inc[fill[n]++] = (int32_t)(e * nb + a);
            }
        hm.inc_e.resize(hm.ninc);
        hm.inc_a.resize(hm.ninc);
        for (int64_t q = 0; q < hm.ninc; q++) {
            hm.inc_e[q] = hm.inc[q] / nb;
            hm.inc_a[q] = (uint8_t)(hm.inc[q] % nb);
        }
    }

    // ---- node adjacency (sorted neighbour nodes) and the position map
    hm.node_off.assign(hm.nn + 1, 0);
    std::vector<int32_t> scratch;
    for (int64_t n = 0; n < hm.nn; n++) {
        scratch.clear();
        for (int32_t t = hm.inc_ptr[n]; t < hm.inc_ptr[n + 1]; t++) {
            int64_t e = hm.inc[t] / nb;
            for (int b = 0; b < nb; b++) scratch.push_back(hm.cell_node[e * nb + b]);
        }
        std::sort(scratch.begin(), scratch.end());
        int64_t deg = std::unique(scratch.begin(), scratch.end()) - scratch.begin();
        hm.node_off[n + 1] = hm.node_off[n] + deg;
    }
    hm.nbr.resize(hm.node_off[hm.nn]);
    hm.pos.assign((size_t)hm.ninc * nb, 0);
    hm.max_deg = 0;
    for (int64_t n = 0; n < hm.nn; n++) {
        scratch.clear();
        for (int32_t t = hm.inc_ptr[n]; t < hm.inc_ptr[n + 1]; t++) {
            int64_t e = hm.inc[t] / nb;
            for (int b = 0; b < nb; b++) scratch.push_back(hm.cell_node[e * nb + b]);
        }
        std::sort(scratch.begin(), scratch.end());
        scratch.erase(std::unique(scratch.begin(), scratch.end()), scratch.end());
        std::copy(scratch.begin(), scratch.end(), hm.nbr.begin() + hm.node_off[n]);
        hm.max_deg = std::max<int>(hm.max_deg, (int)scratch.size());
        if (scratch.size() > 65535) { err = "a node has more than 65535 neighbours"; return false; }
        for (int32_t t = hm.inc_ptr[n]; t < hm.inc_ptr[n + 1]; t++) {
            int64_t e = hm.inc[t] / nb;
            for (int b = 0; b < nb; b++) {
                int32_t m = hm.cell_node[e * nb + b];
                hm.pos[(size_t)t * nb + b] =
                    (uint16_t)(std::lower_bound(scratch.begin(), scratch.end(), m) - scratch.begin());
            }
        }
    }
    hm.nnz = (int64_t)dim * dim * hm.node_off[hm.nn];
    detect_lattice(hm, coords, cv);
    return true;
}

// CSR over dofs: the d rows of node n are d*node_off[n] .. apart; row (n, i)
// lists the columns d*m + j for m in nbr(n) ascending, j = 0..d-1.
void build_csr(const HostMesh &hm, std::vector<int64_t> &indptr, std::vector<int32_t> &indices)
{
    const int d = hm.dim;
    indptr.assign(hm.ndof + 1, 0);
    indices.resize(hm.nnz);
    for (int64_t n = 0; n < hm.nn; n++) {
        int64_t deg = hm.node_off[n + 1] - hm.node_off[n];
        int64_t base = (int64_t)d * d * hm.node_off[n];
        for (int i = 0; i < d; i++) {
            int64_t r = d * n + i;
            indptr[r] = base + i * d * deg;
            int64_t w = indptr[r];
            for (int64_t q = hm.node_off[n]; q < hm.node_off[n + 1]; q++)
                for (int j = 0; j < d; j++) indices[w++] = d * hm.nbr[q] + j;
        }
    }
    indptr[hm.ndof] = hm.nnz;
}

}  // namespace soptx
