/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the SIMP stiffness assembly and
 * the element compliance sensitivities of density-based topology optimisation
 * (SOPTX, arXiv 2505.02438).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file: it is used by the tests, by the smoke check and by the timed CPU
 * baseline of the benchmark.  It shares no code, header, table or constant
 * generator with the CUDA library; the two agree only through the numbers they
 * produce.
 *
 * What it computes, step by step, in the order the paper states the problem:
 *
 *   (1) Modified SIMP interpolation (Sec. 2.1):
 *           E(rho) = Emin + rho^p (E0 - Emin).
 *   (2) The element matrix for unit Young's modulus, K_e^0 (Sec. 2.2, the
 *       discrete problem, "K_e^0 is the elemental matrix for unit Young's
 *       modulus"), by the standard finite-element definition
 *           K_e^0 = int_e B^T D B dx,
 *       evaluated by numerical quadrature at every element -- the paper's
 *       "original assembly" (Sec. 5.5, Table "assembly comparison").  B is the
 *       Voigt strain-displacement matrix with engineering shear, D the
 *       isotropic elasticity matrix (plane stress, plane strain or 3D) at E = 1
 *       (Sec. 3.2.1, material module: Lame constants, elasticity and strain
 *       matrices).
 *   (3) The global stiffness K(rho) = sum_e E(rho_e) K_e^0 (Sec. 2.2) into a
 *       CSR matrix: COO triplets generated element by element, stably sorted
 *       by (row, column), each run summed left to right -- so each entry is
 *       summed in ascending element order.  Every structural pair is kept,
 *       including entries that cancel to zero.
 *   (4) The compliance sensitivity dc_e = -E'(rho_e) u_e^T K_e^0 u_e with
 *       E'(rho) = p rho^(p-1) (E0 - Emin) (the per-element compliance
 *       E u_e^T K_e^0 u_e differentiated in rho, Appendix D), and
 *       c = sum_e E(rho_e) u_e^T K_e^0 u_e = u^T K(rho) u.
 *
 * Lagrange basis: for order k on a reference cell the basis is the unique
 * polynomial basis of P_k (simplices) or Q_k (tensor cells) that is 1 at one
 * node of the equispaced lattice and 0 at the others.  It is obtained by
 * inverting the Vandermonde matrix of monomials at the lattice nodes (double
 * LU with iterative refinement in long double), not from a closed formula.
 *
 * Quadrature: Gauss-Legendre on [0,1] with k+1 points per direction, tensor
 * product on squares/cubes, collapsed (Duffy) product on triangles and
 * tetrahedra.  For affine cells this integrates every entry of K_e^0 exactly.
 *
 * Global node numbering (independent implementation of the library's
 * convention): vertices keep their ids; then edge nodes, edges sorted by
 * (min vertex, max vertex), the k-1 nodes of an edge ordered from the min
 * vertex toward the max vertex; then face nodes (3D cells only), faces sorted
 * by their sorted vertex tuple; then the interior nodes of each cell, cell by
 * cell.  Degrees of freedom are node-interleaved: dof = d*node + component.
 * Reference cells: simplex vertex 0 at the origin, vertex m at the unit vector
 * e_m; tensor cells [0,1]^d with vertices in lexicographic order, x fastest.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_TRI = 0, OR_TET = 1, OR_QUAD = 2, OR_HEX = 3 };
enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2 };

#define OR_MAXNB 64          /* hex Q3 */
#define OR_MAXLDOF 192
#define OR_MAXQ 64           /* 4^3 quadrature points */

static int cell_dim(int cell) { return (cell == OR_TRI || cell == OR_QUAD) ? 2 : 3; }
static int is_simplex(int cell) { return cell == OR_TRI || cell == OR_TET; }
static int n_cell_vertices(int cell)
{
    switch (cell) {
    case OR_TRI: return 3;
    case OR_TET: return 4;
    case OR_QUAD: return 4;
    default: return 8;
    }
}
static int valid_cell(int cell, int k)
{
    return cell >= OR_TRI && cell <= OR_HEX && k >= 1 && k <= 3;
}

/* ---------------------------------------------------------------------------
 * Reference lattice: local node a has integer coordinates L[a] and reference
 * position xi = L[a] / k.  Simplex: all L >= 0 with sum <= k; tensor: [0,k]^d.
 * Enumeration: last axis outermost, x fastest.  The same enumeration, read as
 * exponent tuples, lists the monomials spanning P_k or Q_k.
 * ------------------------------------------------------------------------- */
static int ref_lattice(int cell, int k, int L[][3])
{
    int d = cell_dim(cell), n = 0;
    int lmax = (d == 3) ? k : 0;
    for (int l = 0; l <= lmax; l++)
        for (int j = 0; j <= k; j++)
            for (int i = 0; i <= k; i++) {
                if (is_simplex(cell) && i + j + l > k) continue;
                L[n][0] = i; L[n][1] = j; L[n][2] = l;
                n++;
            }
    return n;
}

int or_ref_lattice(int cell, int k, int *nb, int *lattice /* [nb][3] */)
{
    int L[OR_MAXNB][3];
    if (!valid_cell(cell, k)) return OR_EINVAL;
    int n = ref_lattice(cell, k, L);
    *nb = n;
    if (lattice) memcpy(lattice, L, sizeof(int) * 3 * n);
    return OR_OK;
}

/* ---------------------------------------------------------------------------
 * Lagrange basis by Vandermonde inversion.
 *   V[i][j] = m_j(xi_i), m_j(xi) = t_0^E[j][0] t_1^E[j][1] t_2^E[j][2],
 *   t = sc (xi - ctr) centred on the reference cell (a change of polynomial
 *   basis only: the span is still P_k or Q_k, and it keeps V well conditioned);
 *   C = V^{-1}  so that  phi_a(xi) = sum_j C[j][a] m_j(xi).
 * ------------------------------------------------------------------------- */
typedef struct {
    int cell, k, d, nb;
    int E[OR_MAXNB][3];          /* monomial exponents */
    double C[OR_MAXNB][OR_MAXNB];/* C[j][a] */
    double ctr, sc;              /* monomials in t = sc (xi - ctr), for conditioning */
} basis_t;

static double ipow(double x, int e)
{
    double r = 1.0;
    for (int i = 0; i < e; i++) r *= x;
    return r;
}

/* Solve A X = B (n x n, nrhs columns) by LU with partial pivoting and
 * iterative refinement; residuals in long double. Returns 0 on success. */
static int solve_refined(int n, const double *A, double *X, const double *B, int nrhs)
{
    double *LU = malloc(sizeof(double) * n * n);
    int *piv = malloc(sizeof(int) * n);
    double *R = malloc(sizeof(double) * n * nrhs);
    if (!LU || !piv || !R) { free(LU); free(piv); free(R); return -1; }
    memcpy(LU, A, sizeof(double) * n * n);
    for (int c = 0; c < n; c++) {
        int p = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(LU[r * n + c]) > fabs(LU[p * n + c])) p = r;
        if (LU[p * n + c] == 0.0) { free(LU); free(piv); free(R); return -1; }
        piv[c] = p;
        if (p != c)
            for (int j = 0; j < n; j++) {
                double t = LU[c * n + j]; LU[c * n + j] = LU[p * n + j]; LU[p * n + j] = t;
            }
        for (int r = c + 1; r < n; r++) {
            double f = LU[r * n + c] / LU[c * n + c];
            LU[r * n + c] = f;
            for (int j = c + 1; j < n; j++) LU[r * n + j] -= f * LU[c * n + j];
        }
    }
    /* X = 0, R = B; then repeat: solve LU dX = R, X += dX, R = B - A X */
    memset(X, 0, sizeof(double) * n * nrhs);
    memcpy(R, B, sizeof(double) * n * nrhs);
    for (int it = 0; it < 4; it++) {
        for (int col = 0; col < nrhs; col++) {
            double *y = malloc(sizeof(double) * n);
            if (!y) { free(LU); free(piv); free(R); return -1; }
            for (int i = 0; i < n; i++) y[i] = R[i * nrhs + col];
            for (int c = 0; c < n; c++) {           /* apply row swaps */
                int p = piv[c];
                if (p != c) { double t = y[c]; y[c] = y[p]; y[p] = t; }
            }
            for (int i = 0; i < n; i++)              /* forward, unit L */
                for (int j = 0; j < i; j++) y[i] -= LU[i * n + j] * y[j];
            for (int i = n - 1; i >= 0; i--) {       /* backward, U */
                for (int j = i + 1; j < n; j++) y[i] -= LU[i * n + j] * y[j];
                y[i] /= LU[i * n + i];
            }
            for (int i = 0; i < n; i++) X[i * nrhs + col] += y[i];
            free(y);
        }
        for (int i = 0; i < n; i++)
            for (int col = 0; col < nrhs; col++) {
                long double s = B[i * nrhs + col];
                for (int j = 0; j < n; j++) s -= (long double)A[i * n + j] * (long double)X[j * nrhs + col];
                R[i * nrhs + col] = (double)s;
            }
    }
    free(LU); free(piv); free(R);
    return 0;
}

static int basis_init(basis_t *bs, int cell, int k)
{
    int L[OR_MAXNB][3];
    bs->cell = cell; bs->k = k; bs->d = cell_dim(cell);
    bs->nb = ref_lattice(cell, k, L);
    memcpy(bs->E, L, sizeof(L));
    int n = bs->nb;
    bs->ctr = is_simplex(cell) ? 1.0 / (bs->d + 1) : 0.5;
    bs->sc = 2.0;
    double *V = malloc(sizeof(double) * n * n), *I = calloc((size_t)n * n, sizeof(double));
    double *X = malloc(sizeof(double) * n * n);
    if (!V || !I || !X) { free(V); free(I); free(X); return -1; }
    for (int i = 0; i < n; i++) {
        double t[3];
        for (int m = 0; m < 3; m++) t[m] = bs->sc * ((double)L[i][m] / k - bs->ctr);
        for (int j = 0; j < n; j++)
            V[i * n + j] = ipow(t[0], bs->E[j][0]) * ipow(t[1], bs->E[j][1]) * ipow(t[2], bs->E[j][2]);
        I[i * n + i] = 1.0;
    }
    int rc = solve_refined(n, V, X, I, n);
    if (rc == 0)
        for (int j = 0; j < n; j++)
            for (int a = 0; a < n; a++) bs->C[j][a] = X[j * n + a];
    free(V); free(I); free(X);
    return rc;
}

/* phi[a] and dphi[a][m] (reference derivatives) at reference point x */
static void basis_eval(const basis_t *bs, const double x[3], double *phi, double dphi[][3])
{
    int n = bs->nb;
    double mv[OR_MAXNB], dm[OR_MAXNB][3], tx[3];
    for (int m = 0; m < 3; m++) tx[m] = bs->sc * (x[m] - bs->ctr);
    for (int j = 0; j < n; j++) {
        const int *e = bs->E[j];
        mv[j] = ipow(tx[0], e[0]) * ipow(tx[1], e[1]) * ipow(tx[2], e[2]);
        for (int m = 0; m < 3; m++) {
            if (e[m] == 0) { dm[j][m] = 0.0; continue; }
            double t = bs->sc * e[m] * ipow(tx[m], e[m] - 1);   /* d/dxi = sc d/dt */
            for (int q = 0; q < 3; q++)
                if (q != m) t *= ipow(tx[q], e[q]);
            dm[j][m] = t;
        }
    }
    for (int a = 0; a < n; a++) {
        double s = 0.0, g[3] = { 0.0, 0.0, 0.0 };
        for (int j = 0; j < n; j++) {
            s += bs->C[j][a] * mv[j];
            for (int m = 0; m < 3; m++) g[m] += bs->C[j][a] * dm[j][m];
        }
        if (phi) phi[a] = s;
        if (dphi) for (int m = 0; m < 3; m++) dphi[a][m] = g[m];
    }
}

int or_basis_eval(int cell, int k, int npts, const double *x /* [npts][3] */,
                  double *phi /* [npts][nb] */, double *dphi /* [npts][nb][3] */)
{
    basis_t *bs = malloc(sizeof(basis_t));
    if (!valid_cell(cell, k) || !bs) { free(bs); return OR_EINVAL; }
    if (basis_init(bs, cell, k)) { free(bs); return OR_EINVAL; }
    for (int p = 0; p < npts; p++)
        basis_eval(bs, x + 3 * p, phi ? phi + (size_t)p * bs->nb : NULL,
                   dphi ? (double (*)[3])(dphi + (size_t)p * bs->nb * 3) : NULL);
    free(bs);
    return OR_OK;
}

/* ---------------------------------------------------------------------------
 * Quadrature.
 * ------------------------------------------------------------------------- */
/* Gauss-Legendre nodes/weights on [0,1]: Newton iteration on the Legendre
 * polynomial P_n (three-term recurrence), weights 2/((1-t^2) P_n'(t)^2). */
int or_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1 || n > 32) return OR_EINVAL;
    for (int i = 0; i < n; i++) {
        double t = cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = t;
            for (int j = 2; j <= n; j++) {
                double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
                p0 = p1; p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-17) break;
        }
        {   /* derivative at the converged root */
            double p0 = 1.0, p1 = t;
            for (int j = 2; j <= n; j++) {
                double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
                p0 = p1; p1 = p2;
            }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
        }
        x[i] = 0.5 * (t + 1.0);
        w[i] = 1.0 / ((1.0 - t * t) * dp * dp);   /* (2/((1-t^2)P'^2)) / 2 */
    }
    return OR_OK;
}

/* Quadrature on the reference cell, n points per direction.
 * Tensor: product rule on [0,1]^d.  Simplex: collapsed coordinates
 *   triangle: xi = (s, (1-s) t),                 weight (1-s)
 *   tet:      xi = (s, (1-s) t, (1-s)(1-t) r),   weight (1-s)^2 (1-t)            */
static int ref_quadrature(int cell, int n, double X[][3], double *W)
{
    double g[32], gw[32];
    or_gauss_legendre(n, g, gw);
    int d = cell_dim(cell), nq = 0;
    int n3 = (d == 3) ? n : 1;
    for (int c = 0; c < n3; c++)
        for (int b = 0; b < n; b++)
            for (int a = 0; a < n; a++) {
                double s = g[a], t = g[b], r = (d == 3) ? g[c] : 0.0;
                double w = gw[a] * gw[b] * ((d == 3) ? gw[c] : 1.0);
                if (!is_simplex(cell)) {
                    X[nq][0] = s; X[nq][1] = t; X[nq][2] = r;
                } else if (d == 2) {
                    X[nq][0] = s; X[nq][1] = (1.0 - s) * t; X[nq][2] = 0.0;
                    w *= (1.0 - s);
                } else {
                    X[nq][0] = s; X[nq][1] = (1.0 - s) * t; X[nq][2] = (1.0 - s) * (1.0 - t) * r;
                    w *= (1.0 - s) * (1.0 - s) * (1.0 - t);
                }
                W[nq] = w;
                nq++;
            }
    return nq;
}

int or_ref_quadrature(int cell, int n, int *nq, double *x /* [n^d][3] */, double *w)
{
    double X[OR_MAXQ * 8][3], W[OR_MAXQ * 8];
    if (cell < OR_TRI || cell > OR_HEX || n < 1 || n > 8) return OR_EINVAL;
    int q = ref_quadrature(cell, n, X, W);
    *nq = q;
    memcpy(x, X, sizeof(double) * 3 * q);
    memcpy(w, W, sizeof(double) * q);
    return OR_OK;
}

/* ---------------------------------------------------------------------------
 * Element matrix K_e^0 = int B^T D B with E = 1.
 * ------------------------------------------------------------------------- */
typedef struct {
    int cell, k, d, nb, nv, nq;
    basis_t fe;        /* order-k displacement basis */
    basis_t geo;       /* order-1 geometric basis */
    double X[OR_MAXQ][3], W[OR_MAXQ];
    double dphi[OR_MAXQ][OR_MAXNB][3];   /* reference gradients at quad points */
    double dgeo[OR_MAXQ][8][3];
    double D[6][6];
} elem_ctx;

static void elasticity_D(int d, double nu, int plane_strain, double D[6][6])
{
    memset(D, 0, sizeof(double) * 36);
    double mu = 1.0 / (2.0 * (1.0 + nu));
    if (d == 3 || plane_strain) {
        double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
        if (d == 3) {
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) D[i][j] = lam + (i == j ? 2.0 * mu : 0.0);
            D[3][3] = D[4][4] = D[5][5] = mu;
        } else {
            D[0][0] = D[1][1] = lam + 2.0 * mu;
            D[0][1] = D[1][0] = lam;
            D[2][2] = mu;
        }
    } else {          /* plane stress */
        double f = 1.0 / (1.0 - nu * nu);
        D[0][0] = D[1][1] = f;
        D[0][1] = D[1][0] = f * nu;
        D[2][2] = f * (1.0 - nu) / 2.0;
    }
}

static int elem_ctx_init(elem_ctx *c, int cell, int k, double nu, int plane_strain)
{
    c->cell = cell; c->k = k; c->d = cell_dim(cell);
    c->nv = n_cell_vertices(cell);
    if (basis_init(&c->fe, cell, k) || basis_init(&c->geo, cell, 1)) return -1;
    c->nb = c->fe.nb;
    c->nq = ref_quadrature(cell, k + 1, c->X, c->W);
    for (int q = 0; q < c->nq; q++) {
        basis_eval(&c->fe, c->X[q], NULL, c->dphi[q]);
        basis_eval(&c->geo, c->X[q], NULL, c->dgeo[q]);
    }
    elasticity_D(c->d, nu, plane_strain, c->D);
    return 0;
}

/* Inverse and determinant of a d x d matrix (cofactors). */
static double inv_det(int d, const double J[3][3], double G[3][3])
{
    if (d == 2) {
        double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        G[0][0] = J[1][1] / det; G[0][1] = -J[0][1] / det;
        G[1][0] = -J[1][0] / det; G[1][1] = J[0][0] / det;
        return det;
    }
    double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    G[0][0] = c00 / det;
    G[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    G[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    G[1][0] = c01 / det;
    G[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    G[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    G[2][0] = c02 / det;
    G[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    G[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    return det;
}

/* xv: vertex coordinates of the cell, [nv][d], in reference vertex order.
 * Ke: [ldof][ldof], local dof = d*a + i. Returns 0, or -1 on a degenerate cell. */
static int elem_matrix(const elem_ctx *c, const double *xv, double *Ke)
{
    int d = c->d, nb = c->nb, ldof = d * nb, ns = (d == 2) ? 3 : 6;
    memset(Ke, 0, sizeof(double) * ldof * ldof);
    double B[6][OR_MAXLDOF], DB[6][OR_MAXLDOF];
    for (int q = 0; q < c->nq; q++) {
        /* J = sum_v x_v (grad N_v)^T, formed from the edge vectors x_v - x_0:
         * the vertex basis sums to one, so its gradients sum to zero and J is
         * the same; with vertex 0 as origin its rounding is relative to the
         * cell's size instead of the cell's distance from the origin. */
        double J[3][3] = { { 0 } }, G[3][3];
        for (int v = 1; v < c->nv; v++)
            for (int i = 0; i < d; i++)
                for (int m = 0; m < d; m++) J[i][m] += (xv[v * d + i] - xv[i]) * c->dgeo[q][v][m];
        double det = inv_det(d, J, G);
        if (!(fabs(det) > 0.0) || !isfinite(det)) return -1;
        /* physical gradients: dphi/dx_i = sum_m G[m][i] dphi/dxi_m */
        double gx[OR_MAXNB][3];
        for (int a = 0; a < nb; a++)
            for (int i = 0; i < d; i++) {
                double s = 0.0;
                for (int m = 0; m < d; m++) s += G[m][i] * c->dphi[q][a][m];
                gx[a][i] = s;
            }
        memset(B, 0, sizeof(B));
        for (int a = 0; a < nb; a++) {
            if (d == 2) {
                B[0][2 * a] = gx[a][0];
                B[1][2 * a + 1] = gx[a][1];
                B[2][2 * a] = gx[a][1];  B[2][2 * a + 1] = gx[a][0];
            } else {
                B[0][3 * a] = gx[a][0];
                B[1][3 * a + 1] = gx[a][1];
                B[2][3 * a + 2] = gx[a][2];
                B[3][3 * a + 1] = gx[a][2]; B[3][3 * a + 2] = gx[a][1];   /* yz */
                B[4][3 * a] = gx[a][2];     B[4][3 * a + 2] = gx[a][0];   /* xz */
                B[5][3 * a] = gx[a][1];     B[5][3 * a + 1] = gx[a][0];   /* xy */
            }
        }
        for (int r = 0; r < ns; r++)
            for (int col = 0; col < ldof; col++) {
                double s = 0.0;
                for (int t = 0; t < ns; t++) s += c->D[r][t] * B[t][col];
                DB[r][col] = s;
            }
        double wq = c->W[q] * fabs(det);
        for (int r = 0; r < ldof; r++)
            for (int col = 0; col < ldof; col++) {
                double s = 0.0;
                for (int t = 0; t < ns; t++) s += B[t][r] * DB[t][col];
                Ke[r * ldof + col] += wq * s;
            }
    }
    return 0;
}

int or_element_matrix(int cell, int k, const double *xv, double nu, int plane_strain, double *Ke)
{
    if (!valid_cell(cell, k)) return OR_EINVAL;
    elem_ctx *c = malloc(sizeof(elem_ctx));
    if (!c) return OR_ENOMEM;
    if (elem_ctx_init(c, cell, k, nu, plane_strain)) { free(c); return OR_EINVAL; }
    int rc = elem_matrix(c, xv, Ke) ? OR_EINVAL : OR_OK;
    free(c);
    return rc;
}

/* ---------------------------------------------------------------------------
 * Global node numbering.
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t key[4];   /* sorted global vertex ids of the entity, padded with -1 */
    int64_t slot;     /* index into cell_node: e*nb + a */
    int32_t idx;      /* position of the node inside the entity */
} ent_rec;

static int cmp_key(const void *pa, const void *pb)
{
    const ent_rec *a = pa, *b = pb;
    for (int i = 0; i < 4; i++) {
        if (a->key[i] < b->key[i]) return -1;
        if (a->key[i] > b->key[i]) return 1;
    }
    return (a->slot < b->slot) ? -1 : (a->slot > b->slot);
}

static void sort4(int32_t *v, int n)
{
    for (int i = 1; i < n; i++)
        for (int j = i; j > 0 && v[j - 1] > v[j]; j--) {
            int32_t t = v[j]; v[j] = v[j - 1]; v[j - 1] = t;
        }
}

/* Fills cell_node [NC][nb]; returns NN in *nn_out. */
int or_number(int cell, int k, int64_t nv_total, int64_t nc, const int32_t *cv,
              int32_t *cell_node, int64_t *nn_out)
{
    if (!valid_cell(cell, k) || nc < 0) return OR_EINVAL;
    int L[OR_MAXNB][3];
    int nb = ref_lattice(cell, k, L), d = cell_dim(cell), nvc = n_cell_vertices(cell);
    int nedge_nodes = k - 1;
    int nface_nodes = is_simplex(cell) ? (k - 1) * (k - 2) / 2 : (k - 1) * (k - 1);
    int nint;
    if (cell == OR_TRI) nint = (k - 1) * (k - 2) / 2;
    else if (cell == OR_TET) nint = (k - 1) * (k - 2) * (k - 3) / 6;
    else if (cell == OR_QUAD) nint = (k - 1) * (k - 1);
    else nint = (k - 1) * (k - 1) * (k - 1);

    /* classify local nodes once (topology of the reference lattice) */
    int kind[OR_MAXNB];        /* 0 vertex, 1 edge, 2 face, 3 interior */
    int lverts[OR_MAXNB][8], nlv[OR_MAXNB], int_idx[OR_MAXNB];
    int ni = 0;
    for (int a = 0; a < nb; a++) {
        int n = 0;
        if (is_simplex(cell)) {
            int lam[4];
            lam[0] = k - L[a][0] - L[a][1] - L[a][2];
            for (int m = 0; m < d; m++) lam[m + 1] = L[a][m];
            for (int v = 0; v <= d; v++)
                if (lam[v] > 0) lverts[a][n++] = v;
        } else {
            /* corners matching the fixed coordinates, free axes take both values */
            for (int v = 0; v < nvc; v++) {
                int ok = 1;
                for (int m = 0; m < d; m++) {
                    int bit = (v >> m) & 1;
                    if (L[a][m] == 0 && bit != 0) ok = 0;
                    if (L[a][m] == k && bit != 1) ok = 0;
                }
                if (ok) lverts[a][n++] = v;
            }
        }
        nlv[a] = n;
        int edim;              /* dimension of the entity */
        if (is_simplex(cell)) edim = n - 1;
        else { edim = 0; while ((1 << edim) < n) edim++; }
        if (edim == 0) kind[a] = 0;
        else if (edim == d) kind[a] = 3;
        else if (edim == 1) kind[a] = 1;
        else kind[a] = 2;
        int_idx[a] = (kind[a] == 3) ? ni++ : -1;
    }
    if (ni != nint) return OR_EINVAL;

    int64_t nrec_e = 0, nrec_f = 0;
    for (int a = 0; a < nb; a++) {
        if (kind[a] == 1) nrec_e++;
        if (kind[a] == 2) nrec_f++;
    }
    ent_rec *er = malloc(sizeof(ent_rec) * (size_t)(nrec_e * nc + 1));
    ent_rec *fr = malloc(sizeof(ent_rec) * (size_t)(nrec_f * nc + 1));
    if (!er || !fr) { free(er); free(fr); return OR_ENOMEM; }
    int64_t ne = 0, nf = 0;
    for (int64_t e = 0; e < nc; e++) {
        const int32_t *g = cv + e * nvc;
        for (int a = 0; a < nb; a++) {
            int64_t slot = e * nb + a;
            if (kind[a] == 0) { cell_node[slot] = g[lverts[a][0]]; continue; }
            if (kind[a] == 3) continue;
            ent_rec r;
            r.key[0] = r.key[1] = r.key[2] = r.key[3] = -1;
            for (int t = 0; t < nlv[a]; t++) r.key[t] = g[lverts[a][t]];
            sort4(r.key, nlv[a]);
            r.slot = slot;
            if (kind[a] == 1) {
                if (is_simplex(cell)) {
                    /* barycentric weight of the larger-id vertex */
                    int va = lverts[a][0], vb = lverts[a][1];
                    int vmax = (g[va] > g[vb]) ? va : vb;
                    int lam = (vmax == 0) ? k - L[a][0] - L[a][1] - L[a][2] : L[a][vmax - 1];
                    r.idx = lam - 1;
                } else {
                    int m = 0;
                    while (L[a][m] == 0 || L[a][m] == k) m++;      /* free axis */
                    int c0 = -1, c1 = -1;
                    for (int t = 0; t < 2; t++) {
                        int v = lverts[a][t];
                        if ((v >> m) & 1) c1 = v; else c0 = v;
                    }
                    int tpos = (g[c0] < g[c1]) ? L[a][m] : k - L[a][m];
                    r.idx = tpos - 1;
                }
                er[ne++] = r;
            } else {
                if (is_simplex(cell)) {
                    r.idx = 0;   /* orders <= 3 carry at most one node per face */
                } else {
                    int m1 = -1, m2 = -1;
                    for (int m = 0; m < d; m++)
                        if (L[a][m] != 0 && L[a][m] != k) { if (m1 < 0) m1 = m; else m2 = m; }
                    int o = lverts[a][0];
                    for (int t = 1; t < 4; t++)
                        if (g[lverts[a][t]] < g[o]) o = lverts[a][t];
                    int p1 = o ^ (1 << m1), p2 = o ^ (1 << m2);
                    /* distance from o's side along each free axis */
                    int s1 = ((o >> m1) & 1) ? k - L[a][m1] : L[a][m1];
                    int s2 = ((o >> m2) & 1) ? k - L[a][m2] : L[a][m2];
                    int s, t;
                    if (g[p1] < g[p2]) { s = s1; t = s2; } else { s = s2; t = s1; }
                    r.idx = (s - 1) + (k - 1) * (t - 1);
                }
                fr[nf++] = r;
            }
        }
    }
    int64_t off = nv_total;
    qsort(er, (size_t)ne, sizeof(ent_rec), cmp_key);
    int64_t id = -1;
    for (int64_t i = 0; i < ne; i++) {
        if (i == 0 || memcmp(er[i].key, er[i - 1].key, sizeof(er[i].key))) id++;
        cell_node[er[i].slot] = (int32_t)(off + id * nedge_nodes + er[i].idx);
    }
    off += (id + 1) * nedge_nodes;
    qsort(fr, (size_t)nf, sizeof(ent_rec), cmp_key);
    id = -1;
    for (int64_t i = 0; i < nf; i++) {
        if (i == 0 || memcmp(fr[i].key, fr[i - 1].key, sizeof(fr[i].key))) id++;
        cell_node[fr[i].slot] = (int32_t)(off + id * nface_nodes + fr[i].idx);
    }
    if (nface_nodes > 0) off += (id + 1) * nface_nodes;
    for (int64_t e = 0; e < nc; e++)
        for (int a = 0; a < nb; a++)
            if (kind[a] == 3) cell_node[e * nb + a] = (int32_t)(off + e * nint + int_idx[a]);
    off += nc * nint;
    free(er); free(fr);
    *nn_out = off;
    return OR_OK;
}

/* Node positions: x(node) = sum_v N_v(xi_a) x_v for every cell and local node. */
int or_node_coords(int cell, int k, int64_t nc, const int32_t *cv, const double *coords,
                   const int32_t *cell_node, int64_t nn, double *xn /* [nn][d] */)
{
    if (!valid_cell(cell, k)) return OR_EINVAL;
    basis_t *geo = malloc(sizeof(basis_t));
    if (!geo) return OR_ENOMEM;
    if (basis_init(geo, cell, 1)) { free(geo); return OR_EINVAL; }
    int L[OR_MAXNB][3];
    int nb = ref_lattice(cell, k, L), d = cell_dim(cell), nvc = n_cell_vertices(cell);
    double N[OR_MAXNB][8];
    for (int a = 0; a < nb; a++) {
        double x[3] = { (double)L[a][0] / k, (double)L[a][1] / k, (double)L[a][2] / k };
        double phi[8];
        basis_eval(geo, x, phi, NULL);
        for (int v = 0; v < nvc; v++) N[a][v] = phi[v];
    }
    for (int64_t i = 0; i < nn * d; i++) xn[i] = NAN;
    for (int64_t e = 0; e < nc; e++)
        for (int a = 0; a < nb; a++) {
            int64_t n = cell_node[e * nb + a];
            for (int i = 0; i < d; i++) {
                double s = 0.0;
                for (int v = 0; v < nvc; v++) s += N[a][v] * coords[(int64_t)cv[e * nvc + v] * d + i];
                xn[n * d + i] = s;
            }
        }
    free(geo);
    return OR_OK;
}

/* ---------------------------------------------------------------------------
 * SIMP (Sec. 2.1) and the assembly (Sec. 2.2).
 * ------------------------------------------------------------------------- */
static double simp_E(double rho, double E0, double Emin, double p)
{
    return Emin + pow(rho, p) * (E0 - Emin);
}
static double simp_dE(double rho, double E0, double Emin, double p)
{
    return p * pow(rho, p - 1.0) * (E0 - Emin);
}

typedef struct {
    int64_t row;     /* selected-row index */
    int64_t col;
    int64_t seq;     /* generation order: element-major, then a, i, b, j */
    double val;
} trip;

static int cmp_trip(const void *pa, const void *pb)
{
    const trip *a = pa, *b = pb;
    if (a->row != b->row) return a->row < b->row ? -1 : 1;
    if (a->col != b->col) return a->col < b->col ? -1 : 1;
    return (a->seq < b->seq) ? -1 : (a->seq > b->seq);
}

static void cell_coords(const elem_ctx *c, const double *coords, const int32_t *cv, int64_t e, double *xv)
{
    for (int v = 0; v < c->nv; v++)
        for (int i = 0; i < c->d; i++)
            xv[v * c->d + i] = coords[(int64_t)cv[e * c->nv + v] * c->d + i];
}

/*
 * Assemble the rows sel[0..nsel) of K(rho) (nsel < 0: every row, in order).
 * absval != 0 sums |E_e K_e^0[a][b]| instead: the scale against which a
 * computed entry's rounding error is judged.
 * Outputs are malloc'ed here and released with or_free():
 *   rowptr [nrows+1] int64, cols [nnz] int32, vals [nnz] double.
 * Also returns ndof, and NN through nn_out (both may be NULL).
 */
int or_assemble_rows(int cell, int k, int64_t nv_total, const double *coords,
                     int64_t nc, const int32_t *cv,
                     double E0, double Emin, double nu, double p, int plane_strain,
                     const double *rho, int64_t nsel, const int64_t *sel, int absval,
                     int64_t *nnz_out, int64_t **rowptr_out, int32_t **cols_out,
                     double **vals_out, int64_t *ndof_out)
{
    if (!valid_cell(cell, k)) return OR_EINVAL;
    elem_ctx *c = malloc(sizeof(elem_ctx));
    if (!c) return OR_ENOMEM;
    if (elem_ctx_init(c, cell, k, nu, plane_strain)) { free(c); return OR_EINVAL; }
    int d = c->d, nb = c->nb, ldof = d * nb;
    int32_t *cn = malloc(sizeof(int32_t) * (size_t)(nc * nb + 1));
    int64_t nn = 0;
    if (!cn) { free(c); return OR_ENOMEM; }
    int rc = or_number(cell, k, nv_total, nc, cv, cn, &nn);
    if (rc) { free(c); free(cn); return rc; }
    int64_t ndof = d * nn;
    int64_t nrows = (nsel < 0) ? ndof : nsel;
    int64_t *rowsel = malloc(sizeof(int64_t) * (size_t)(ndof + 1));
    if (!rowsel) { free(c); free(cn); return OR_ENOMEM; }
    for (int64_t r = 0; r < ndof; r++) rowsel[r] = (nsel < 0) ? r : -1;
    for (int64_t s = 0; s < nsel; s++) {
        if (sel[s] < 0 || sel[s] >= ndof) { free(c); free(cn); free(rowsel); return OR_EINVAL; }
        rowsel[sel[s]] = s;
    }
    /* count triplets */
    int64_t nt = 0;
    for (int64_t e = 0; e < nc; e++)
        for (int a = 0; a < nb; a++)
            for (int i = 0; i < d; i++)
                if (rowsel[d * (int64_t)cn[e * nb + a] + i] >= 0) nt += ldof;
    trip *T = malloc(sizeof(trip) * (size_t)(nt + 1));
    double *Ke = malloc(sizeof(double) * ldof * ldof);
    double xv[8 * 3];
    if (!T || !Ke) { free(c); free(cn); free(rowsel); free(T); free(Ke); return OR_ENOMEM; }
    int64_t t = 0, seq = 0;
    for (int64_t e = 0; e < nc; e++) {
        int need = 0;
        for (int a = 0; a < nb && !need; a++)
            for (int i = 0; i < d; i++)
                if (rowsel[d * (int64_t)cn[e * nb + a] + i] >= 0) need = 1;
        if (!need) continue;
        cell_coords(c, coords, cv, e, xv);
        if (elem_matrix(c, xv, Ke)) { rc = OR_EINVAL; break; }
        double Ee = simp_E(rho[e], E0, Emin, p);
        for (int a = 0; a < nb; a++)
            for (int i = 0; i < d; i++) {
                int64_t r = rowsel[d * (int64_t)cn[e * nb + a] + i];
                if (r < 0) continue;
                for (int b = 0; b < nb; b++)
                    for (int j = 0; j < d; j++) {
                        T[t].row = r;
                        T[t].col = d * (int64_t)cn[e * nb + b] + j;
                        T[t].seq = seq++;
                        T[t].val = Ee * Ke[(d * a + i) * ldof + d * b + j];
                        if (absval) T[t].val = fabs(T[t].val);
                        t++;
                    }
            }
    }
    if (rc) { free(c); free(cn); free(rowsel); free(T); free(Ke); return rc; }
    qsort(T, (size_t)t, sizeof(trip), cmp_trip);
    int64_t nnz = 0;
    for (int64_t i = 0; i < t; i++)
        if (i == 0 || T[i].row != T[i - 1].row || T[i].col != T[i - 1].col) nnz++;
    int64_t *rowptr = calloc((size_t)(nrows + 1), sizeof(int64_t));
    int32_t *cols = malloc(sizeof(int32_t) * (size_t)(nnz + 1));
    double *vals = malloc(sizeof(double) * (size_t)(nnz + 1));
    if (!rowptr || !cols || !vals) {
        free(c); free(cn); free(rowsel); free(T); free(Ke); free(rowptr); free(cols); free(vals);
        return OR_ENOMEM;
    }
    int64_t s = -1;
    for (int64_t i = 0; i < t; i++) {
        if (i == 0 || T[i].row != T[i - 1].row || T[i].col != T[i - 1].col) {
            s++;
            cols[s] = (int32_t)T[i].col;
            vals[s] = T[i].val;
            rowptr[T[i].row + 1]++;
        } else {
            vals[s] += T[i].val;      /* left to right: ascending element */
        }
    }
    for (int64_t r = 0; r < nrows; r++) rowptr[r + 1] += rowptr[r];
    *nnz_out = nnz; *rowptr_out = rowptr; *cols_out = cols; *vals_out = vals;
    if (ndof_out) *ndof_out = ndof;
    free(c); free(cn); free(rowsel); free(T); free(Ke);
    return OR_OK;
}

void or_free(void *ptr) { free(ptr); }

/*
 * Element sensitivities on the cells sel[0..nsel) (nsel < 0: every cell):
 *   s_e  = u_e^T K_e^0 u_e                      (strain-energy density form)
 *   dc_e = -E'(rho_e) s_e
 * and, when every cell is selected, c = sum_e E(rho_e) s_e in element order.
 * s_out and sabs_out (sum_ab |u_a K_ab u_b|, the rounding-error scale of s_e)
 * may be NULL.
 */
int or_sensitivity(int cell, int k, int64_t nv_total, const double *coords,
                   int64_t nc, const int32_t *cv,
                   double E0, double Emin, double nu, double p, int plane_strain,
                   const double *rho, const double *u, int64_t nsel, const int64_t *sel,
                   double *dc, double *s_out, double *sabs_out, double *c_out)
{
    if (!valid_cell(cell, k)) return OR_EINVAL;
    elem_ctx *c = malloc(sizeof(elem_ctx));
    if (!c) return OR_ENOMEM;
    if (elem_ctx_init(c, cell, k, nu, plane_strain)) { free(c); return OR_EINVAL; }
    int d = c->d, nb = c->nb, ldof = d * nb;
    int32_t *cn = malloc(sizeof(int32_t) * (size_t)(nc * nb + 1));
    double *Ke = malloc(sizeof(double) * ldof * ldof);
    int64_t nn = 0;
    if (!cn || !Ke) { free(c); free(cn); free(Ke); return OR_ENOMEM; }
    int rc = or_number(cell, k, nv_total, nc, cv, cn, &nn);
    if (rc) { free(c); free(cn); free(Ke); return rc; }
    int64_t ncell = (nsel < 0) ? nc : nsel;
    double ctot = 0.0, ue[OR_MAXLDOF], xv[8 * 3];
    for (int64_t q = 0; q < ncell; q++) {
        int64_t e = (nsel < 0) ? q : sel[q];
        if (e < 0 || e >= nc) { rc = OR_EINVAL; break; }
        cell_coords(c, coords, cv, e, xv);
        if (elem_matrix(c, xv, Ke)) { rc = OR_EINVAL; break; }
        for (int a = 0; a < nb; a++)
            for (int i = 0; i < d; i++) ue[d * a + i] = u[d * (int64_t)cn[e * nb + a] + i];
        double se = 0.0, sa = 0.0;
        for (int r = 0; r < ldof; r++) {
            double kr = 0.0;
            for (int col = 0; col < ldof; col++) {
                kr += Ke[r * ldof + col] * ue[col];
                sa += fabs(ue[r] * Ke[r * ldof + col] * ue[col]);
            }
            se += ue[r] * kr;
        }
        if (sabs_out) sabs_out[q] = sa;
        dc[q] = -simp_dE(rho[e], E0, Emin, p) * se;
        if (s_out) s_out[q] = se;
        ctot += simp_E(rho[e], E0, Emin, p) * se;
    }
    if (c_out) *c_out = (nsel < 0) ? ctot : NAN;
    free(c); free(cn); free(Ke);
    return rc;
}

/*
 * Backward of f(rho) = u^T K(rho) u at fixed u, scaled by the incoming
 * gradient g:  grad_rho_e = g E'(rho_e) u_e^T K_e^0 u_e,  grad_u = 2 g K(rho) u
 * (grad_u may be NULL).  The u-gradient uses the full CSR assembly above.
 */
int or_compliance_vjp(int cell, int k, int64_t nv_total, const double *coords,
                      int64_t nc, const int32_t *cv,
                      double E0, double Emin, double nu, double p, int plane_strain,
                      const double *rho, const double *u, double g,
                      double *grad_rho, double *grad_u)
{
    double *s = malloc(sizeof(double) * (size_t)(nc + 1));
    double *dc = malloc(sizeof(double) * (size_t)(nc + 1));
    if (!s || !dc) { free(s); free(dc); return OR_ENOMEM; }
    int rc = or_sensitivity(cell, k, nv_total, coords, nc, cv, E0, Emin, nu, p, plane_strain,
                            rho, u, -1, NULL, dc, s, NULL, NULL);
    if (rc) { free(s); free(dc); return rc; }
    for (int64_t e = 0; e < nc; e++) grad_rho[e] = g * simp_dE(rho[e], E0, Emin, p) * s[e];
    free(s); free(dc);
    if (!grad_u) return OR_OK;
    int64_t nnz = 0, ndof = 0, *rp = NULL;
    int32_t *ci = NULL;
    double *v = NULL;
    rc = or_assemble_rows(cell, k, nv_total, coords, nc, cv, E0, Emin, nu, p, plane_strain,
                          rho, -1, NULL, 0, &nnz, &rp, &ci, &v, &ndof);
    if (rc) return rc;
    for (int64_t r = 0; r < ndof; r++) {
        double acc = 0.0;
        for (int64_t q = rp[r]; q < rp[r + 1]; q++) acc += v[q] * u[ci[q]];
        grad_u[r] = 2.0 * g * acc;
    }
    free(rp); free(ci); free(v);
    return OR_OK;
}
