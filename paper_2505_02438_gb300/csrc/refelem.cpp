// Reference element of the library: local node lattice and the exact reference
// integrals  M[k][l][a][b] = int_ref d_k phi_a  d_l phi_b.
//
// This is the "symbolic" half of the paper's symbolic fast assembly (Sec. 3.2.2,
// Sec. 5.5): the element-independent integrals are computed exactly, once, in
// rational arithmetic, and only rounded to double at the end.  Per element, the
// device contracts them with the element's inverse Jacobian (kernels.cu).
//
//  * Simplices (P_k): the basis function of the node with barycentric lattice
//    index alpha (sum = k) is  prod_v prod_{s < alpha_v} (k lam_v - s)/(s + 1),
//    a polynomial in the barycentric coordinates lam_0..lam_d; d/dxi_m =
//    d/dlam_m - d/dlam_0; and  int_ref lam^beta = prod(beta_v!) / (|beta| + d)!.
//  * Tensor cells (Q_k): products of 1D Lagrange polynomials on the equispaced
//    nodes i/k of [0,1]; the integral factorises into 1D integrals of
//    l_i l_j, l_i' l_j and l_i' l_j'.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <numeric>

#include "internal.h"

namespace soptx {
namespace {

// Exact rational with 128-bit numerator / denominator, always reduced.
struct Q {
    __int128 n = 0, d = 1;
    Q() = default;
    Q(long long v) : n(v), d(1) {}
    Q(__int128 a, __int128 b) : n(a), d(b) { norm(); }
    static __int128 g(__int128 a, __int128 b)
    {
        if (a < 0) a = -a;
        if (b < 0) b = -b;
        while (b) {
            __int128 t = a % b;
            a = b;
            b = t;
        }
        return a ? a : 1;
    }
    void norm()
    {
        if (d < 0) { n = -n; d = -d; }
        __int128 q = g(n, d);
        n /= q;
        d /= q;
    }
    Q operator+(const Q &o) const { return Q(n * o.d + o.n * d, d * o.d); }
    Q operator-(const Q &o) const { return Q(n * o.d - o.n * d, d * o.d); }
    Q operator*(const Q &o) const { return Q(n * o.n, d * o.d); }
    Q operator/(const Q &o) const { return Q(n * o.d, d * o.n); }
    bool zero() const { return n == 0; }
    double to_double() const { return (double)((long double)n / (long double)d); }
};

// Polynomial in up to 4 variables: exponent tuple -> coefficient.
using Mono = std::array<int, 4>;
using Poly = std::map<Mono, Q>;

Poly pmul(const Poly &a, const Poly &b)
{
    Poly r;
    for (auto &x : a)
        for (auto &y : b) {
            Mono m;
            for (int i = 0; i < 4; i++) m[i] = x.first[i] + y.first[i];
            r[m] = r[m] + x.second * y.second;
        }
    for (auto it = r.begin(); it != r.end();) it = it->second.zero() ? r.erase(it) : std::next(it);
    return r;
}

Poly pdiff(const Poly &a, int var)
{
    Poly r;
    for (auto &x : a) {
        if (x.first[var] == 0) continue;
        Mono m = x.first;
        Q c = x.second * Q((long long)m[var]);
        m[var] -= 1;
        r[m] = r[m] + c;
    }
    return r;
}

Poly psub(const Poly &a, const Poly &b)
{
    Poly r = a;
    for (auto &y : b) r[y.first] = r[y.first] - y.second;
    return r;
}

long long fact(int n)
{
    long long f = 1;
    for (int i = 2; i <= n; i++) f *= i;
    return f;
}

// int over the unit simplex of prod lam_v^beta_v (Dirichlet integral)
Q simplex_integral(const Poly &p, int dim)
{
    Q s(0);
    for (auto &x : p) {
        long long num = 1;
        int tot = 0;
        for (int v = 0; v <= dim; v++) {
            num *= fact(x.first[v]);
            tot += x.first[v];
        }
        s = s + x.second * Q((__int128)num, (__int128)fact(tot + dim));
    }
    return s;
}

}  // namespace

bool build_ref_element(int cell, int order, RefElement &ref, std::string &err)
{
    if (order < 1 || order > 3) {
        err = "order must be 1, 2 or 3";
        return false;
    }
    const int k = order, dim = cell_dim(cell);
    ref.cell = cell;
    ref.order = order;
    ref.dim = dim;
    ref.lat.clear();
    if (is_simplex(cell)) {
        // barycentric multi-indices: vertices first (vertex v carries lam_v = k),
        // then the rest in lexicographic order of (lam_1, ..., lam_d)
        std::vector<std::array<int, 4>> rest;
        for (int v = 0; v <= dim; v++) {
            std::array<int, 4> L{0, 0, 0, 0};
            if (v == 0) L[3] = k; else L[v - 1] = k;
            ref.lat.push_back(L);
        }
        for (int c = 0; c <= (dim == 3 ? k : 0); c++)
            for (int b = 0; b <= k; b++)
                for (int a = 0; a <= k; a++) {
                    int s = a + b + c;
                    if (s > k) continue;
                    std::array<int, 4> L{a, b, c, k - s};
                    int nz = (a > 0) + (b > 0) + (c > 0) + (k - s > 0);
                    if (nz == 1) continue;   // a vertex, already listed
                    rest.push_back(L);
                }
        ref.lat.insert(ref.lat.end(), rest.begin(), rest.end());
    } else {
        for (int c = 0; c <= (dim == 3 ? k : 0); c++)
            for (int b = 0; b <= k; b++)
                for (int a = 0; a <= k; a++) ref.lat.push_back({a, b, c, 0});
    }
    const int nb = (int)ref.lat.size();
    ref.nb = nb;
    ref.M.assign((size_t)dim * dim * nb * nb, 0.0);

    if (is_simplex(cell)) {
        // basis polynomials in lam_0..lam_dim (variable index v); lam_0 <-> lat[3]
        std::vector<Poly> phi(nb);
        for (int a = 0; a < nb; a++) {
            int alpha[4] = {ref.lat[a][3], ref.lat[a][0], ref.lat[a][1], ref.lat[a][2]};
            Poly p;
            p[Mono{0, 0, 0, 0}] = Q(1);
            for (int v = 0; v <= dim; v++)
                for (int s = 0; s < alpha[v]; s++) {
                    Poly f;   // (k lam_v - s) / (s + 1)
                    Mono mv{0, 0, 0, 0};
                    mv[v] = 1;
                    f[mv] = Q((__int128)k, (__int128)(s + 1));
                    if (s) f[Mono{0, 0, 0, 0}] = Q((__int128)-s, (__int128)(s + 1));
                    p = pmul(p, f);
                }
            phi[a] = p;
        }
        std::vector<std::vector<Poly>> grad(nb, std::vector<Poly>(dim));
        for (int a = 0; a < nb; a++) {
            Poly d0 = pdiff(phi[a], 0);
            for (int m = 0; m < dim; m++) grad[a][m] = psub(pdiff(phi[a], m + 1), d0);
        }
        for (int kk = 0; kk < dim; kk++)
            for (int l = 0; l < dim; l++)
                for (int a = 0; a < nb; a++)
                    for (int b = 0; b < nb; b++) {
                        Q v = simplex_integral(pmul(grad[a][kk], grad[b][l]), dim);
                        ref.M[(((size_t)kk * dim + l) * nb + a) * nb + b] = v.to_double();
                    }
    } else {
        // 1D Lagrange polynomials on t_i = i/k, as coefficient vectors
        std::vector<std::vector<Q>> ell(k + 1);
        for (int i = 0; i <= k; i++) {
            std::vector<Q> c{Q(1)};
            Q den(1);
            for (int j = 0; j <= k; j++) {
                if (j == i) continue;
                // multiply by (t - j/k)
                std::vector<Q> nc(c.size() + 1, Q(0));
                for (size_t q = 0; q < c.size(); q++) {
                    nc[q + 1] = nc[q + 1] + c[q];
                    nc[q] = nc[q] - c[q] * Q((__int128)j, (__int128)k);
                }
                c = nc;
                den = den * Q((__int128)(i - j), (__int128)k);
            }
            for (auto &x : c) x = x / den;
            ell[i] = c;
        }
        auto deriv = [](const std::vector<Q> &c) {
            std::vector<Q> r;
            for (size_t q = 1; q < c.size(); q++) r.push_back(c[q] * Q((long long)q));
            if (r.empty()) r.push_back(Q(0));
            return r;
        };
        auto integ = [](const std::vector<Q> &a, const std::vector<Q> &b) {
            Q s(0);
            for (size_t p = 0; p < a.size(); p++)
                for (size_t q = 0; q < b.size(); q++)
                    s = s + a[p] * b[q] * Q((__int128)1, (__int128)(p + q + 1));
            return s;
        };
        std::vector<std::vector<Q>> I0(k + 1, std::vector<Q>(k + 1)), I1 = I0, I2 = I0;
        for (int i = 0; i <= k; i++)
            for (int j = 0; j <= k; j++) {
                I0[i][j] = integ(ell[i], ell[j]);
                I1[i][j] = integ(deriv(ell[i]), ell[j]);        // derivative on the first
                I2[i][j] = integ(deriv(ell[i]), deriv(ell[j]));
            }
        for (int kk = 0; kk < dim; kk++)
            for (int l = 0; l < dim; l++)
                for (int a = 0; a < nb; a++)
                    for (int b = 0; b < nb; b++) {
                        Q v(1);
                        for (int m = 0; m < dim; m++) {
                            int ia = ref.lat[a][m], ib = ref.lat[b][m];
                            if (m == kk && m == l) v = v * I2[ia][ib];
                            else if (m == kk) v = v * I1[ia][ib];
                            else if (m == l) v = v * I1[ib][ia];
                            else v = v * I0[ia][ib];
                        }
                        ref.M[(((size_t)kk * dim + l) * nb + a) * nb + b] = v.to_double();
                    }
    }
    return true;
}

// Gauss-Legendre nodes and weights on [0, 1]: roots of the Legendre polynomial
// P_n by Newton's method from the asymptotic guesses cos(pi (i + 3/4) / (n + 1/2)),
// P_n and P_n' from the three-term recurrence; w = 2 / ((1 - x^2) P_n'(x)^2) on
// [-1, 1], halved for [0, 1].
static void gauss_legendre01(int n, std::vector<double> &t, std::vector<double> &w)
{
    t.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; i++) {
        double x = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int j = 1; j < n; j++) {
                const double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            const double pn = n == 0 ? 1.0 : p1, pm = n == 1 ? 1.0 : p0;
            dp = n * (x * pn - pm) / (x * x - 1.0);
            const double dx = pn / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-17) break;
        }
        // ascending order on [0, 1]
        t[n - 1 - i] = 0.5 * (x + 1.0);
        w[n - 1 - i] = 1.0 / ((1.0 - x * x) * dp * dp);
    }
}

// 1D Lagrange polynomial l_i on the equispaced nodes j/k and its derivative at t
static void lagrange1d(int k, int i, double t, double &val, double &der)
{
    val = 1.0;
    der = 0.0;
    for (int j = 0; j <= k; j++) {
        if (j == i) continue;
        const double den = (double)(i - j) / k;
        der = der * ((t - (double)j / k) / den) + val / den;
        val *= (t - (double)j / k) / den;
    }
}

// The one-dimensional factors of the tensor rule below: weights w[q] of the
// order + 1 Gauss points t_q on [0, 1], and val[q][j] = l_j(t_q),
// der[q][j] = l_j'(t_q) for the Lagrange polynomials on the nodes j / order.
void tensor_1d_factors(int order, std::vector<double> &w, std::vector<double> &val, std::vector<double> &der)
{
    const int n = order + 1;
    std::vector<double> t;
    gauss_legendre01(n, t, w);
    val.assign((size_t)n * n, 0.0);
    der.assign((size_t)n * n, 0.0);
    for (int q = 0; q < n; q++)
        for (int j = 0; j < n; j++) lagrange1d(order, j, t[q], val[(size_t)q * n + j], der[(size_t)q * n + j]);
}

void build_tensor_quadrature(const RefElement &ref, RefQuad &q)
{
    const int dim = ref.dim, k = ref.order, n = k + 1, nb = ref.nb;
    const int nvc = 1 << dim;
    std::vector<double> t1, w1;
    gauss_legendre01(n, t1, w1);
    q.nvc = nvc;
    q.nq = 1;
    for (int m = 0; m < dim; m++) q.nq *= n;
    q.w.assign(q.nq, 0.0);
    q.dphi.assign((size_t)q.nq * nb * dim, 0.0);
    q.dgeo.assign((size_t)q.nq * nvc * dim, 0.0);
    for (int p = 0; p < q.nq; p++) {
        int idx[3] = {p % n, (p / n) % n, p / (n * n)};
        double xi[3] = {0, 0, 0}, w = 1.0;
        for (int m = 0; m < dim; m++) {
            xi[m] = t1[idx[m]];
            w *= w1[idx[m]];
        }
        q.w[p] = w;
        for (int a = 0; a < nb; a++) {
            double val[3], der[3];
            for (int m = 0; m < dim; m++) lagrange1d(k, ref.lat[a][m], xi[m], val[m], der[m]);
            for (int m = 0; m < dim; m++) {
                double g = der[m];
                for (int o = 0; o < dim; o++)
                    if (o != m) g *= val[o];
                q.dphi[((size_t)p * nb + a) * dim + m] = g;
            }
        }
        for (int v = 0; v < nvc; v++)
            for (int m = 0; m < dim; m++) {
                double g = ((v >> m) & 1) ? 1.0 : -1.0;
                for (int o = 0; o < dim; o++)
                    if (o != m) g *= ((v >> o) & 1) ? xi[o] : 1.0 - xi[o];
                q.dgeo[((size_t)p * nvc + v) * dim + m] = g;
            }
    }
}

// Reference gradients of the simplex basis at xi: with the barycentric
// coordinates lam_0 = 1 - sum xi, lam_m = xi_m, the basis function of node a
// is prod_v f_v(lam_v), f_v(t) = prod_{s < alpha_v} (k t - s) / (s + 1), and
// d/dxi_m = d/dlam_m - d/dlam_0.
static void simplex_basis_grad(const RefElement &ref, const double *xi, double *dphi)
{
    const int dim = ref.dim, k = ref.order, nb = ref.nb;
    double lam[4] = {1.0, 0.0, 0.0, 0.0};
    for (int m = 0; m < dim; m++) {
        lam[m + 1] = xi[m];
        lam[0] -= xi[m];
    }
    for (int a = 0; a < nb; a++) {
        const int alpha[4] = {ref.lat[a][3], ref.lat[a][0], ref.lat[a][1], ref.lat[a][2]};
        double f[4], df[4];
        for (int v = 0; v <= dim; v++) {
            double val = 1.0, der = 0.0;
            for (int s = 0; s < alpha[v]; s++) {
                const double c = (k * lam[v] - s) / (s + 1.0), dc = k / (s + 1.0);
                der = der * c + val * dc;
                val *= c;
            }
            f[v] = val;
            df[v] = der;
        }
        double dl[4];
        for (int v = 0; v <= dim; v++) {
            double g = df[v];
            for (int w = 0; w <= dim; w++)
                if (w != v) g *= f[w];
            dl[v] = g;
        }
        for (int m = 0; m < dim; m++) dphi[(size_t)a * dim + m] = dl[m + 1] - dl[0];
    }
}

// Quadrature of the reference simplex exact for polynomials of degree
// 2 (k - 1), the degree of the strain energy density of a P_k field:
//   k = 1: the centroid;
//   k = 2: triangle, the three edge midpoints (weights 1/6); tetrahedron, the
//          symmetric four-point rule with barycentric coordinates
//          (alpha, beta, beta, beta), alpha = (5 + 3 sqrt 5) / 20,
//          beta = (5 - sqrt 5) / 20, weights 1/24;
//   k = 3: the conical product of Gauss-Legendre rules (the collapsed square /
//          cube: xi_1 = u, xi_2 = v (1 - u), xi_3 = w (1 - u)(1 - v), Jacobian
//          (1 - u)^(d-1) (1 - v)^(d-2)), 3 x 3 points on the triangle and
//          4 x 3 x 3 on the tetrahedron: the substituted integrand has degree
//          p + d - 1 in u, p + d - 2 in v and p in w, p = 4.
void build_simplex_quadrature(const RefElement &ref, RefQuad &q)
{
    const int dim = ref.dim, k = ref.order, nb = ref.nb;
    std::vector<std::array<double, 3>> pts;
    std::vector<double> wts;
    if (k == 1) {
        pts.push_back({1.0 / (dim + 1), 1.0 / (dim + 1), dim == 3 ? 0.25 : 0.0});
        wts.push_back(dim == 3 ? 1.0 / 6 : 0.5);
    } else if (k == 2 && dim == 2) {
        pts = {{0.5, 0.0, 0.0}, {0.5, 0.5, 0.0}, {0.0, 0.5, 0.0}};
        wts.assign(3, 1.0 / 6);
    } else if (k == 2) {
        const double al = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, be = (5.0 - std::sqrt(5.0)) / 20.0;
        // lam_0 = alpha (the origin vertex), then alpha on each unit vertex
        pts = {{be, be, be}, {al, be, be}, {be, al, be}, {be, be, al}};
        wts.assign(4, 1.0 / 24);
    } else if (k == 3 && dim == 2) {
        // Radon's seven-point rule (Stroud T2:5-1), exact for degree 5 (the
        // energy density of P3 is degree 4): the centroid and two orbits of three
        // points (a, a, b) in barycentric coordinates, area 1/2
        const double r = std::sqrt(15.0);
        const double a1 = (6.0 - r) / 21.0, b1 = (9.0 + 2.0 * r) / 21.0, w1 = (155.0 - r) / 2400.0;
        const double a2 = (6.0 + r) / 21.0, b2 = (9.0 - 2.0 * r) / 21.0, w2 = (155.0 + r) / 2400.0;
        pts = {{1.0 / 3, 1.0 / 3, 0.0}, {a1, a1, 0.0}, {a1, b1, 0.0}, {b1, a1, 0.0},
               {a2, a2, 0.0}, {a2, b2, 0.0}, {b2, a2, 0.0}};
        wts = {9.0 / 80, w1, w1, w1, w2, w2, w2};
    } else {
        std::vector<double> tu, wu, tv, wv;
        gauss_legendre01(dim == 3 ? 4 : 3, tu, wu);
        gauss_legendre01(3, tv, wv);
        for (size_t iu = 0; iu < tu.size(); iu++)
            for (size_t iv = 0; iv < tv.size(); iv++)
                for (size_t iw = 0; iw < (dim == 3 ? tv.size() : 1); iw++) {
                    const double u = tu[iu], v = tv[iv];
                    if (dim == 2) {
                        pts.push_back({u, v * (1.0 - u), 0.0});
                        wts.push_back(wu[iu] * wv[iv] * (1.0 - u));
                    } else {
                        const double w = tv[iw];
                        pts.push_back({u, v * (1.0 - u), w * (1.0 - u) * (1.0 - v)});
                        wts.push_back(wu[iu] * wv[iv] * wv[iw] * (1.0 - u) * (1.0 - u) * (1.0 - v));
                    }
                }
    }
    q.nq = (int)pts.size();
    q.nvc = 0;
    q.w = wts;
    q.dphi.assign((size_t)q.nq * nb * dim, 0.0);
    q.dgeo.clear();
    for (int p = 0; p < q.nq; p++) simplex_basis_grad(ref, pts[p].data(), &q.dphi[(size_t)p * nb * dim]);
}

}  // namespace soptx
