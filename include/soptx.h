/*
 * soptx.h -- C ABI of the GB300 (sm_103a) SIMP stiffness-assembly library.
 *
 * The library computes, on one GPU, the per-iteration hot path of density-based
 * topology optimisation with the modified SIMP model (SOPTX, arXiv 2505.02438):
 *
 *   E(rho_e)  = Emin + rho_e^p (E0 - Emin)                       (Sec. 2.1)
 *   K(rho)    = sum_e E(rho_e) K_e^0   into a fixed CSR pattern   (Sec. 2.2)
 *   dc_e      = -p rho_e^(p-1) (E0 - Emin) u_e^T K_e^0 u_e        (Appendix D)
 *   c         = sum_e E(rho_e) u_e^T K_e^0 u_e  (= u^T K(rho) u)
 *
 * where K_e^0 is the linear-elasticity element matrix at unit Young's modulus
 * (Sec. 2.2).  Following the paper's fast / symbolic-fast assembly (Sec. 3.2.2,
 * Sec. 5.5), the element-independent part (exact reference-cell integrals of
 * basis-gradient products) is computed once per mesh and contracted with each
 * element's Jacobian; everything that does not depend on rho is kept resident
 * on the device between calls.
 *
 * Conventions shared by every call:
 *  - Pointers named d_* are DEVICE pointers owned by the caller (contiguous,
 *    dtype as declared).  Pointers without the prefix are host pointers.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Every call except soptx_mesh_create / soptx_mesh_destroy only
 *    enqueues work on `stream` and returns without synchronising.
 *  - A mesh owns a small device scratch area, so calls on ONE mesh must be
 *    ordered on the device (same stream, or explicit events); calls on
 *    different meshes may overlap freely.
 *  - No call aborts, traps or prints.  On failure the call returns a non-zero
 *    soptx_status and soptx_last_error() describes it (thread-local).
 *  - Degrees of freedom are node-interleaved: dof = dim * node + component.
 *  - Cells: dim 2 = SOPTX_TRI / SOPTX_QUAD, dim 3 = SOPTX_TET / SOPTX_HEX.
 *    Vertex order inside a cell: simplices list the vertex at the reference
 *    origin first, then the vertices at the unit vectors e_1..e_d (either
 *    orientation is accepted; |det J| is used); quads and hexes list their
 *    corners lexicographically on the unit square / cube, x fastest.  Quads
 *    and hexes may be general bilinear / trilinear cells: parallelograms and
 *    parallelepipeds take the exact reference-integral contraction, any other
 *    cell the (order+1)^d-point Gauss rule with the Jacobian of the geometry
 *    map at every point (computed once, at mesh creation).  A cell whose
 *    Jacobian changes sign or vanishes at a corner is rejected.
 *  - Lagrange order 1..3.  Higher-order nodes are numbered after the vertices:
 *    edge nodes (edges sorted by (min vertex id, max vertex id), the order-1
 *    nodes of an edge running from the min-id vertex to the max-id vertex),
 *    then face nodes of 3D cells (faces sorted by their sorted vertex ids; on a
 *    quad face the nodes run in the frame of its smallest vertex o, first axis
 *    toward the smaller-id neighbour of o), then interior nodes cell by cell.
 *  - The CSR pattern is the full symmetric structural pattern over all dofs
 *    (no boundary-condition elimination), column indices sorted ascending per
 *    row; entries that cancel to zero are kept.
 */
#ifndef SOPTX_H
#define SOPTX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SOPTX_OK = 0,
    SOPTX_EINVAL = 1,     /* an argument is invalid (see soptx_last_error)   */
    SOPTX_ENOMEM = 2,     /* a device or host allocation failed              */
    SOPTX_ECUDA = 3,      /* a CUDA runtime call failed                      */
    SOPTX_EBUSY = 4,      /* server: no slot and the queue is full           */
    SOPTX_ETIMEOUT = 5,   /* server: a bounded wait ran out                  */
    SOPTX_ENOTFOUND = 6,  /* server: unknown ticket                          */
    SOPTX_EINTERNAL = 7   /* a device-side consistency check failed          */
} soptx_status;

typedef enum { SOPTX_TRI = 0, SOPTX_TET = 1, SOPTX_QUAD = 2, SOPTX_HEX = 3 } soptx_cell;

/* Precision of the element matrices K_e^0.  The CSR accumulation, the
 * sensitivities and c are FP64-accurate in both modes (Sec. 2.2 is stated in
 * exact arithmetic; the paper fixes no precision). */
typedef enum { SOPTX_ELEM_FP64 = 0, SOPTX_ELEM_FP32 = 1 } soptx_elem_prec;

/* Modified SIMP material (Sec. 2.1, Sec. 3.2.1): E0 solid modulus, Emin void
 * modulus (the paper uses 1e-9 E0), nu Poisson ratio, p penalisation.  In 2D,
 * plane_strain = 0 selects plane stress (unit thickness). */
typedef struct {
    double E0, Emin, nu, p;
    int32_t plane_strain;
} soptx_material;

typedef struct soptx_mesh_s *soptx_mesh;

/* Which device path a mesh was given (soptx_mesh_path). */
typedef enum {
    SOPTX_PATH_LATTICE = 0,   /* order-1 box lattice: implicit maps, one K^0;
                                 in 3D only while the used entries of K^0 span
                                 at most 2^24 (else the uniform path)          */
    SOPTX_PATH_UNIFORM = 1,   /* every cell has the same Jacobian: one K^0     */
    SOPTX_PATH_CACHED = 2     /* per-cell K_e^0 cached on the device           */
} soptx_path;

/*
 * Build a device-resident mesh (Sec. 3.2.2 "fast matrix assembly": everything
 * independent of rho is computed here, once).
 *   dim, cell, order : 2/3, cell type, Lagrange order 1..3
 *   coords           : host, float64 [n_vertices][dim]
 *   cell_vertices    : host, int32 [n_cells][nv] (nv = 3, 4, 4, 8 for
 *                      TRI, TET, QUAD, HEX), ids in [0, n_vertices)
 *   mat              : host, material; nu in (-1, 0.5), p >= 1, E0 > Emin >= 0
 *   prec             : element-matrix precision
 *   stream           : stream for the setup copies and kernels
 *   out              : receives the mesh handle
 * Allocates device memory (reported by soptx_mesh_device_bytes) and
 * synchronises `stream`.  Errors: EINVAL (bad sizes, ids, a degenerate or
 * inverted cell, ndof >= 2^31), ENOMEM, ECUDA.  n_cells = 0 is allowed.
 */
soptx_status soptx_mesh_create(int dim, soptx_cell cell, int order,
                               int64_t n_vertices, const double *coords,
                               int64_t n_cells, const int32_t *cell_vertices,
                               const soptx_material *mat, soptx_elem_prec prec,
                               void *stream, soptx_mesh *out);

/* Sizes: ndof = dim * n_nodes, nnz of the CSR pattern, n_cells, local dofs per
 * cell.  Any output pointer may be NULL. */
soptx_status soptx_mesh_info(soptx_mesh mesh, int64_t *ndof, int64_t *nnz,
                             int64_t *n_cells, int32_t *ldof);

/* Borrowed device pointers, valid until soptx_mesh_destroy:
 * d_indptr int64 [ndof+1], d_indices int32 [nnz]. */
soptx_status soptx_mesh_pattern(soptx_mesh mesh, const int64_t **d_indptr,
                                const int32_t **d_indices);

/* Borrowed device pointer to the cell -> node map, int32 [n_cells][nb]
 * (nb = ldof / dim); dof of (cell e, local node a, component i) is
 * dim * map[e][a] + i.  The local node order is the library's own. */
soptx_status soptx_mesh_cell_nodes(soptx_mesh mesh, const int32_t **d_cell_nodes, int32_t *nb);

/* Copy the pattern / cell -> node map into caller-owned device buffers
 * (d_indptr int64 [ndof+1], d_indices int32 [nnz], d_cell_nodes int32
 * [n_cells][nb]); enqueued on `stream`.  Either pattern pointer may be NULL. */
soptx_status soptx_mesh_copy_pattern(soptx_mesh mesh, int64_t *d_indptr, int32_t *d_indices, void *stream);
soptx_status soptx_mesh_copy_cell_nodes(soptx_mesh mesh, int32_t *d_cell_nodes, void *stream);

/* Device path chosen for the mesh and the device bytes the mesh holds. */
soptx_status soptx_mesh_path(soptx_mesh mesh, soptx_path *path);

/*
 * The kernels that serve the mesh's per-call work.
 *   *assembly    : 0 box lattice (k_lattice_assemble2/3), 1 row gather of
 *                  element matrices (cached, or one shared matrix), 2
 *                  per-call contraction of the reference integrals in FP32
 *                  (FP32 element matrices of affine cells: k_contract_pairs
 *                  in 2D, k_contract_rows in 3D), 3 node pairs over the
 *                  cached FP64 element matrices (2D affine cells:
 *                  k_contract_pairs reading each pair's blocks once)
 *   *sensitivity : 0 box lattice (Walsh sectors), 1 fused into the row
 *                  gather, 2 strain energy at quadrature points
 *                  (k_strain_energy: affine cells)
 * Either pointer may be NULL.
 */
soptx_status soptx_mesh_routes(soptx_mesh mesh, int32_t *assembly, int32_t *sensitivity);
soptx_status soptx_mesh_device_bytes(soptx_mesh mesh, int64_t *bytes);

/*
 * K(rho) = sum_e E(rho_e) K_e^0 into the mesh's CSR pattern (Sec. 2.2).
 *   d_rho  : device float64 [n_cells], element densities (any real values;
 *            the SIMP power is evaluated as given)
 *   d_vals : device float64 [nnz], overwritten with the CSR values
 * No atomics: every value is formed in a fixed order, so the result is
 * bitwise reproducible run to run, and it is within 1e-12 of the sum of the
 * absolute element contributions of the exact value (FP64 element matrices).
 * The order depends on the path: on a general mesh each value is the sum of
 * its element contributions in ascending element order (float-pair
 * accumulation); on a box lattice it is the reference block entry times a
 * signed sum of the (at most 2^d) moduli of the cells the two nodes share,
 * formed by per-axis sums and differences.
 */
soptx_status soptx_assemble_K(soptx_mesh mesh, const double *d_rho, double *d_vals, void *stream);

/*
 * Element compliance sensitivities (Appendix D; Sec. 2.2):
 *   d_dc[e] = -p rho_e^(p-1) (E0 - Emin) u_e^T K_e^0 u_e
 *   *d_c    = sum_e E(rho_e) u_e^T K_e^0 u_e   (skipped when d_c is NULL)
 *   d_u    : device float64 [ndof]
 *   d_dc   : device float64 [n_cells]
 *   d_c    : device float64 [1] or NULL; summed in a fixed order.
 */
soptx_status soptx_sensitivity(soptx_mesh mesh, const double *d_rho, const double *d_u,
                               double *d_dc, double *d_c, void *stream);

/* One pass that produces both K(rho) and the sensitivities (the per-iteration
 * step); same arguments and results as the two calls above: K and dc bitwise,
 * c the same fixed-order sum of block partials (on 2D meshes of affine cells
 * other than box lattices over one block per SM, so its last bits may differ
 * from the separate call's when the mesh has more cells than the SMs' blocks
 * hold).  On a 2D box lattice the sensitivities run on a second, mesh-owned
 * stream beside the assembly; on other 2D meshes of affine cells they run
 * first on that stream (created at the highest stream priority), one block per
 * SM, beside the assembly on `stream`; on 3D meshes of affine cells the
 * assembly runs on that stream beside the sensitivities on `stream` (the
 * stream and two events are made by the first such call); everything is
 * ordered on `stream` when the call returns. */
soptx_status soptx_assemble_and_sensitivity(soptx_mesh mesh, const double *d_rho,
                                            const double *d_u, double *d_vals,
                                            double *d_dc, double *d_c, void *stream);

/*
 * The one-call step (Sec. 2.2, Appendix D) for a group of n distinct meshes,
 * one launch serving many small ones: per k the arguments and results of
 * soptx_assemble_and_sensitivity(meshes[k], d_rho[k], d_u[k], d_vals[k],
 * d_dc[k], d_c[k], stream).  Box lattices of up to 4096 cells in 2D (Q4 up
 * to 64 x 64) and 1024 in 3D (hex Q1, e.g. 16 x 8 x 8) share one kernel launch per 32 meshes of
 * a dimension, a cluster of 8 CTAs each (the moduli, then the assembly and the
 * sensitivities); the other meshes get the ordinary call on the same stream.
 * K, dc and c are bitwise the values of the ordinary call (the same
 * arithmetic, c summed over the same blocks in the same order).
 *   n      : number of meshes (0 does nothing)
 *   arrays : host arrays of n entries (device pointers inside); d_c[k] may be
 *            NULL, the others as in soptx_assemble_and_sensitivity
 * Errors: SOPTX_EINVAL (a NULL array or entry, a mesh listed twice, n < 0)
 * before anything is launched; SOPTX_ECUDA from a launch.  No mesh of the
 * group may have work in flight on another stream.
 */
soptx_status soptx_assemble_and_sensitivity_group(int32_t n, const soptx_mesh *meshes,
                                                  const double *const *d_rho,
                                                  const double *const *d_u,
                                                  double *const *d_vals, double *const *d_dc,
                                                  double *const *d_c, void *stream);

/*
 * The per-iteration step from host memory: the results of
 * soptx_assemble_and_sensitivity (Sec. 2.2 and Appendix D) with rho and u
 * read from, and dc and c written to, host buffers.
 *   h_rho : host float64 [n_cells]; h_u : host float64 [ndof]
 *   d_vals: device float64 [nnz], overwritten with the CSR values of K(rho)
 *   h_dc  : host float64 [n_cells]; h_c : host float64 [1] or NULL.  When
 *           h_c == h_dc + n_cells, dc and c come back in one copy.
 * Asynchronous on `stream`: h_rho and h_u must stay unchanged, and h_dc and
 * *h_c may be read, only once the stream has completed; page-locked host
 * buffers (cudaHostAlloc, torch pin_memory) keep the copies asynchronous.
 * On a box lattice the sensitivities, which need rho and u but not K, run on a
 * second stream behind u's copy while the moduli and the assembly run on
 * `stream`; everything is ordered on `stream` when the call returns.  The
 * first call allocates the device staging (8 (2 n_cells + ndof + 1) bytes, in
 * soptx_mesh_device_bytes), that stream and two events, kept with the mesh;
 * calls on one mesh must therefore not overlap.  Results are bitwise those of
 * the device-pointer calls.
 */
soptx_status soptx_step_host(soptx_mesh mesh, const double *h_rho, const double *h_u, double *d_vals,
                             double *h_dc, double *h_c, void *stream);

/*
 * Backward of f(rho, u) = u^T K(rho) u (the compliance written as a function
 * of an independent u) scaled by the incoming gradient g = *d_gout:
 *   d_grad_rho[e] = g p rho_e^(p-1) (E0 - Emin) u_e^T K_e^0 u_e   (= -g dc_e)
 *   d_grad_u      = 2 g K(rho) u          (skipped when d_grad_u is NULL)
 * d_gout is a device float64 [1]; d_grad_rho [n_cells]; d_grad_u [ndof].
 * The u-gradient is the product with K(rho) assembled into a mesh-owned
 * scratch of 8 nnz bytes, made by the first call with d_grad_u (counted in
 * soptx_mesh_device_bytes); if that memory cannot be allocated it is formed
 * matrix-free from the element matrices instead (same result within the
 * tolerance, about an order of magnitude slower).
 */
soptx_status soptx_compliance_vjp(soptx_mesh mesh, const double *d_rho, const double *d_u,
                                  const double *d_gout, double *d_grad_rho, double *d_grad_u,
                                  void *stream);

/*
 * Allocation-free sensitivities on a box lattice.  The paper has no
 * counterpart to this call: it exists for callers that must not allocate
 * device memory -- code running under another framework's memory pool or
 * allocator hooks, or in a process whose GPU memory is reserved up front --
 * and therefore cannot create a mesh either (soptx_mesh_create allocates).
 *
 * The lattice is described by its sizes alone: cells_per_axis[dim] cells of
 * edge lengths cell_size[dim] (host arrays), vertices, cells and corners in
 * lexicographic order with x fastest, dofs node-interleaved -- the same layout
 * and results as a mesh that soptx_mesh_create puts on its box-lattice path.
 *   d_rho [n_cells], d_u [ndof], d_dc [n_cells]: device float64, caller-owned;
 *   d_c: device float64 [1] or NULL.
 * Computes d_dc[e] = -E'(rho_e) u_e^T K^0 u_e and *d_c = sum_e E(rho_e) u_e^T K^0 u_e.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine.  Its only
 * scratch, one partial sum of c per 1024 cells, is a fixed 64 KiB __device__
 * array inside the library that every GPU loading the library keeps until the
 * process exits; hence the limit: n_cells <= 8,388,608, larger lattices return
 * SOPTX_EINVAL.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture.  The address is kept for the life of the process:
 * do not call this entry point on a device after a cudaDeviceReset of that
 * device.  All calls share the array, so calls that overlap on the device race
 * on it; every call overwrites the slots it uses.
 */
soptx_status soptx_lattice_sensitivity_noalloc(int dim, const int32_t *cells_per_axis,
                                               const double *cell_size, const soptx_material *mat,
                                               const double *d_rho, const double *d_u, double *d_dc,
                                               double *d_c, void *stream);

/* Frees the mesh's device memory (synchronises the device first). */
soptx_status soptx_mesh_destroy(soptx_mesh mesh);

/*
 * Host-only planning (no device work, usable without a GPU): runs the same
 * validation, numbering and pattern construction as soptx_mesh_create and
 * returns the sizes and, for non-NULL host buffers, the results:
 *   indptr int64 [ndof+1], indices int32 [nnz], cell_nodes int32 [n_cells][nb],
 *   *path the device path a mesh would take (a 3D box lattice whose boxes are
 *   so elongated that K^0 spans more than 2^24 is planned as the lattice but
 *   built on the uniform path).  Call once with NULL buffers to
 *   learn ndof / nnz, then again with buffers of those sizes.
 */
soptx_status soptx_host_plan(int dim, soptx_cell cell, int order, int64_t n_vertices,
                             const double *coords, int64_t n_cells, const int32_t *cell_vertices,
                             int64_t *ndof, int64_t *nnz, int32_t *nb, soptx_path *path,
                             int64_t *indptr, int32_t *indices, int32_t *cell_nodes);

/*
 * Host-only inspection (no device work, usable without a GPU) of the node-pair
 * schedule by which the pair kernel forms K(rho) = sum_e E(rho_e) K_e^0
 * (Sec. 2.2) on 2D affine meshes and uniform meshes.  Built exactly as
 * soptx_mesh_create builds it for a mesh; the mesh arguments are those of
 * soptx_host_plan.
 *
 * A pair is two nodes a, b that share a cell (or a = b).  In 2D K is
 * symmetric, so each unordered pair appears once, owned by whichever node
 * comes first in the processing order (nodes by first cell, then id), and its
 * block is written into row block (a, b) and, transposed, into (b, a); in 3D
 * every ordered pair appears, each node writing its own row blocks.  Pairs come
 * in tiles of 32 (one per lane of a warp); lanes past a window's last pair are
 * empty (count 0).  Per pair (int32 / uint32 arrays of n_tiles * 32 entries):
 *   pair_block[t*32+l]   the CSR value index of entry (d a, d b) of block (a, b), divided by d;
 *   pair_block_t[t*32+l] the same for block (b, a) (2D; 3D: equal to pair_block);
 *   pair_meta[t*32+l]    cell count | (row length of a's rows) << 10 | (of b's rows) << 21.
 * tile_offsets (uint32 [n_tiles + 1]): tile t's records are rows
 * tile_offsets[t] .. tile_offsets[t+1] - 1 of 32 records each, record (k, l) at
 * 32 k + l, the pair's k-th cell in ascending order (k below its count; the
 * remaining slots are 0):
 *   record_cell int32 [n_records]  the cell;
 *   record_pair uint16 [n_records] the pair's local nodes in that cell, as
 *                                  a_loc << 8 | b_loc when local_pair_bytes is
 *                                  nonzero (the FP64 forms), else a_loc nb + b_loc.
 * n_records = 32 * tile_offsets[n_tiles].  *n_tiles = -1 (and *n_records = 0)
 * when the mesh is past the tables' limits (a node in more than 1023 cells,
 * more than 255 nodes per cell, rows of more than 2047 values, value indices
 * past 2^32 d): such meshes are assembled by the row gather.  Call once with
 * NULL buffers for the sizes, then again with buffers of those sizes.
 * Errors: those of soptx_host_plan.
 */
soptx_status soptx_host_pair_tables(int dim, soptx_cell cell, int order, int64_t n_vertices,
                                    const double *coords, int64_t n_cells, const int32_t *cell_vertices,
                                    int32_t local_pair_bytes, int64_t *n_tiles, int64_t *n_records,
                                    uint32_t *tile_offsets, uint32_t *pair_block, uint32_t *pair_block_t,
                                    uint32_t *pair_meta, int32_t *record_cell, uint16_t *record_pair);

/*
 * Host-only inspection (no device work, usable without a GPU) of the
 * node-owner schedule by which 3D meshes with FP32 element matrices form
 * K(rho) = sum_e E(rho_e) K_e^0 (Sec. 2.2): a group of nb lanes owns the d rows
 * of one node and walks the node's cells as a chain.  Built exactly as
 * soptx_mesh_create builds it; the mesh arguments are those of soptx_host_plan.
 *   node_records int32 [n_nodes][4], in processing order (cell count
 *     descending, then node id): the node's first row block offset (low and
 *     high 32-bit words; the value index of its entry (d n, .) is d^2 times
 *     it), its first incidence q0, and cell count << 16 | degree (the number
 *     of column blocks in its rows).
 *   chain_cell int32 [n_incidences], chain_local uint8 [n_incidences]: for
 *     each node, at q0 .. q0 + count - 1, its cells in chain order (the first
 *     is its lowest cell; then the unvisited cell holding the most of the
 *     nodes the lanes hold, lowest id on ties) and its local index there.
 *   lane_records uint16 [n_incidences][nb]: per chain position and lane, the
 *     column block p (bits 0-8, its position in the node's rows), the lane's
 *     local node b in that cell (bits 9-13; a lane keeps its node when the
 *     next cell holds it, the other nodes go to the free lanes in local
 *     order), and whether this is the first (bit 14) or the last (bit 15)
 *     (position, lane) of the chain that meets block p.
 * *n_nodes = -1 (and *n_incidences = 0) for a 2D mesh or one past the
 * schedule's limits (other than 4, 8, 10, 20 or 27 nodes per cell, more than
 * 512 column blocks per row, 65536 or more cells at a node, or accumulators
 * past shared memory): such meshes are assembled otherwise.  *nb is set
 * whenever the call succeeds.  Call once with NULL buffers for the sizes, then
 * again with buffers of those sizes.  Errors: those of soptx_host_plan.
 */
soptx_status soptx_host_row_tables(int dim, soptx_cell cell, int order, int64_t n_vertices,
                                   const double *coords, int64_t n_cells, const int32_t *cell_vertices,
                                   int64_t *n_nodes, int64_t *n_incidences, int32_t *nb,
                                   int32_t *node_records, int32_t *chain_cell, uint8_t *chain_local,
                                   uint16_t *lane_records);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char *soptx_last_error(void);

/* Library version string. */
const char *soptx_version(void);

/*
 * Diagnostic (no counterpart in the paper): the current device's throughput of
 * FP32 and FP64 fused multiply-adds and of f32 -> f64 conversions, from
 * all-SM microkernels timed with CUDA events (best of five launches).  The
 * ratio ffma / dfma is why this library forms FP64-accurate element
 * arithmetic in float pairs on the FP32 pipes.  Synchronises the device;
 * allocates and frees a small buffer.  Errors: EINVAL (NULL), ENOMEM, ECUDA.
 */
typedef struct {
    double ffma_per_s, dfma_per_s, f2f64_per_s;
    int32_t sms;
} soptx_pipe_rates;
soptx_status soptx_measure_pipe_rates(soptx_pipe_rates *out);

/* Test hook for failure handling: the n-th device allocation from now on
 * (n >= 1) fails as if the device were out of memory; n <= 0 disables. */
void soptx_debug_fail_alloc_after(int64_t n);

/* Test hook for the lattice path: while enabled (nonzero), meshes created
 * from now on skip the Walsh-sector split of the box element, so their
 * sensitivities take the general gather kernels (the route a box whose
 * element matrix does not split would take). */
void soptx_debug_lattice_no_sectors(int32_t enable);

#ifdef __cplusplus
}
#endif

#endif /* SOPTX_H */
