/*
 * soptx_opt.h -- the steps of a SIMP iteration after the sensitivities
 * (Sec. 2.3-2.4 of the paper): the sensitivity and density filters with the
 * density filter's chain rule, the Heaviside projection, and the optimality-
 * criteria update of the densities with the volume multiplier found by
 * bisection (Algorithm 1).  Element data are per cell, device float64.
 */
#ifndef SOPTX_OPT_H
#define SOPTX_OPT_H

#include <stdint.h>

#include "soptx.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct soptx_filter_s *soptx_filter;

/*
 * The filter weights H_ij = max(0, rmin - |c_i - c_j|) over cells whose
 * centroids lie closer than rmin (Sec. 2.4), kept on the device as a CSR
 * matrix (rows sorted by column; H is symmetric).
 *   centroids : host float64 [n_cells][dim];  volumes : host float64 [n_cells]
 * Built on the host with a uniform grid of bucket size rmin.  Errors: EINVAL
 * (dim not 2 or 3, rmin <= 0, non-finite input), ENOMEM, ECUDA.
 */
soptx_status soptx_filter_create(int dim, int64_t n_cells, const double *centroids, const double *volumes,
                                 double rmin, void *stream, soptx_filter *out);
soptx_status soptx_filter_info(soptx_filter f, int64_t *n_cells, int64_t *nnz);

/* Sensitivity filter: out_i = sum_j H_ij rho_j dc_j / (max(1e-3, rho_i) sum_j H_ij). */
soptx_status soptx_filter_sensitivity(soptx_filter f, const double *d_rho, const double *d_dc, double *d_out,
                                      void *stream);

/* Density filter: out_i = sum_j H_ij v_j x_j / sum_j H_ij v_j. */
soptx_status soptx_filter_density(soptx_filter f, const double *d_x, double *d_out, void *stream);

/* Chain rule of the density filter: out_j = sum_i (H_ij v_j / sum_k H_ik v_k) g_i,
 * g = d psi / d(filtered density), out = d psi / d x. */
soptx_status soptx_filter_density_grad(soptx_filter f, const double *d_g, double *d_out, void *stream);

soptx_status soptx_filter_destroy(soptx_filter f);

/*
 * Heaviside projection: out_i = 1 - exp(-beta x_i) + x_i exp(-beta); with
 * d_dout non-NULL also d out_i / d x_i = beta exp(-beta x_i) + exp(-beta).
 */
soptx_status soptx_heaviside(int64_t n, double beta, const double *d_x, double *d_out, double *d_dout,
                             void *stream);

typedef struct {
    double volfrac;        /* target: sum_e v_e rho_e <= volfrac sum_e v_e            */
    double move;           /* move limit m                                              */
    double eta;            /* damping exponent eta in (0, 1]                            */
    double l_lo, l_hi;     /* initial bracket of the multiplier (e.g. 0 and 1e9)        */
    double tol;            /* bisection stops when (l_hi - l_lo) / (l_hi + l_lo) <= tol */
} soptx_oc_opts;

/*
 * Optimality-criteria update (Sec. 2.3, Algorithm 1): with B_e = -dc_e / (lambda dv_e),
 *   rho_new = clamp(rho_e B_e^eta, max(0, rho_e - m), min(1, rho_e + m)),
 * lambda found by bisection on the volume constraint (at most 100 steps), the
 * bracket moved on the device between steps; its sums run in a fixed order.
 *   d_rho, d_dc, d_dv, d_vol : device float64 [n] (densities, objective and
 *   volume sensitivities, cell volumes);  d_out [n] the new densities;
 *   d_stats : device float64 [3] or NULL: max |rho_new - rho|, lambda, volume fraction.
 * Allocates n + O(1000) doubles of scratch for the call and returns after the
 * stream has finished with it.
 */
soptx_status soptx_oc_update(int64_t n, const double *d_rho, const double *d_dc, const double *d_dv,
                             const double *d_vol, const soptx_oc_opts *opts, double *d_out, double *d_stats,
                             void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SOPTX_OPT_H */
