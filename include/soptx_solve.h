/*
 * soptx_solve.h -- the step after assembly in each SIMP iteration (Sec. 2.2,
 * the discrete problem K(rho) u = F): the product of the assembled K with a
 * vector and the equilibrium solve under Dirichlet constraints, on the CSR
 * values that soptx_assemble_K wrote into the mesh's pattern.
 */
#ifndef SOPTX_SOLVE_H
#define SOPTX_SOLVE_H

#include <stdint.h>

#include "soptx.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * y = K x with K the mesh's CSR pattern and the values d_vals.
 *   d_vals : device float64 [nnz] (e.g. the output of soptx_assemble_K)
 *   d_x    : device float64 [ndof];  d_y : device float64 [ndof], overwritten
 * Rows are summed in a fixed order (bitwise reproducible).  Async on stream.
 * Errors: EINVAL for NULL pointers, ECUDA for a failed launch.
 */
soptx_status soptx_spmv(soptx_mesh mesh, const double *d_vals, const double *d_x, double *d_y, void *stream);

typedef struct {
    double rtol;           /* stop when ||r_free|| <= rtol * ||f_free - K_fd u_d|| (> 0)       */
    int32_t max_iter;      /* iteration cap (>= 1)                                             */
    int32_t check_every;   /* the residual is read back to the host every this many steps (>= 1) */
    int32_t warm_start;    /* nonzero: start from the free entries of d_u instead of 0         */
} soptx_cg_opts;

typedef struct {
    int32_t iterations;    /* CG steps taken                                                   */
    int32_t converged;     /* 1 when the residual test was met                                 */
    double rel_residual;   /* ||r_free|| / ||f_free - K_fd u_d|| at the last check             */
} soptx_cg_result;

/*
 * K u = f on the free dofs, u fixed where d_fixed[dof] != 0 (Dirichlet):
 * Jacobi-preconditioned conjugate gradients started from u = 0 on the free
 * dofs (or from the free entries of d_u with warm_start, e.g. the previous
 * design's displacements in an optimisation loop); the residual is measured
 * against the right-hand side f - K u_D on the free rows.
 *   d_vals  : device float64 [nnz], the assembled K
 *   d_fixed : device uint8 [ndof], nonzero marks a constrained dof
 *   d_f     : device float64 [ndof], the load (ignored on constrained dofs)
 *   d_u     : device float64 [ndof]; on entry the prescribed values on the
 *             constrained dofs (and the initial guess elsewhere with
 *             warm_start, else ignored), on exit the solution
 * Runs on `stream` and returns when done: the host reads the residual back
 * every opts->check_every steps.  The first call on a mesh allocates its CG
 * vectors (5 ndof doubles), kept until soptx_mesh_destroy.  Sums are taken in
 * a fixed order, so the iterates are bitwise reproducible.  Calls on one mesh
 * must not overlap.
 * Errors: EINVAL (bad arguments), ENOMEM, ECUDA; a zero diagonal on a free dof
 * (a free dof no element touches) makes the preconditioner undefined: EINVAL.
 */
soptx_status soptx_solve_cg(soptx_mesh mesh, const double *d_vals, const uint8_t *d_fixed, const double *d_f,
                            double *d_u, const soptx_cg_opts *opts, void *stream, soptx_cg_result *res);

#ifdef __cplusplus
}
#endif

#endif /* SOPTX_SOLVE_H */
