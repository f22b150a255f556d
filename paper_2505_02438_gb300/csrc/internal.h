// Internal declarations shared by the host setup, the kernels and the ABI.
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/soptx.h"

namespace soptx {

constexpr int kMaxNb = 64;       // hex Q3
constexpr int kMaxLdof = 192;

inline int cell_dim(int cell) { return (cell == SOPTX_TRI || cell == SOPTX_QUAD) ? 2 : 3; }
inline bool is_simplex(int cell) { return cell == SOPTX_TRI || cell == SOPTX_TET; }
inline int cell_nverts(int cell) { return cell == SOPTX_TRI ? 3 : (cell == SOPTX_HEX ? 8 : 4); }

// ---------------------------------------------------------------- errors
void set_error(const std::string &msg);
struct Status {
    soptx_status code = SOPTX_OK;
};
#define SOPTX_FAIL(code, msg)            \
    do {                                 \
        ::soptx::set_error(msg);         \
        return (code);                   \
    } while (0)

// Device allocation with the failure-injection test hook.
cudaError_t dev_alloc(void **p, size_t bytes);

// ---------------------------------------------------------------- reference element
// Local nodes of the library's own reference element and the exact integrals
// M[k][l][a][b] = int_ref d_k phi_a d_l phi_b (rational arithmetic, rounded once).
struct RefElement {
    int cell = 0, order = 1, dim = 2, nb = 0;
    // Lattice coordinates of each local node (multiples of 1/order).  Simplices
    // carry barycentric indices lam[0..dim] (lam[0] = order - sum of the rest).
    std::vector<std::array<int, 4>> lat;
    std::vector<double> M;   // [dim][dim][nb][nb]
};
bool build_ref_element(int cell, int order, RefElement &ref, std::string &err);

// Gauss-Legendre rule of the reference square / cube, (order + 1) points per
// direction, with the reference gradients of the order-k basis and of the
// vertex (order-1) basis at the points: the standard numerical assembly of
// general (non-affine) bilinear / trilinear cells.
struct RefQuad {
    int nq = 0, nvc = 0;
    std::vector<double> w;      // [nq]
    std::vector<double> dphi;   // [nq][nb][dim]
    std::vector<double> dgeo;   // [nq][nvc][dim]
};
void build_tensor_quadrature(const RefElement &ref, RefQuad &q);
// its 1D factors: Gauss weights [n] and the basis values / derivatives [n][n]
void tensor_1d_factors(int order, std::vector<double> &w, std::vector<double> &val, std::vector<double> &der);
// Quadrature of the reference simplex exact for degree 2 (order - 1), with the
// reference gradients of the basis at its points (dgeo left empty).
void build_simplex_quadrature(const RefElement &ref, RefQuad &q);

// ---------------------------------------------------------------- host mesh setup
struct HostMesh {
    int dim = 0, cell = 0, order = 0, nb = 0, ldof = 0, nvc = 0;
    int64_t nv = 0, nc = 0, nn = 0, ndof = 0, nnz = 0, ninc = 0;
    std::vector<int32_t> cell_node;     // [nc][nb]
    std::vector<int64_t> node_off;      // [nn+1] prefix of node degrees
    std::vector<int32_t> nbr;           // [node_off[nn]] sorted neighbour nodes
    std::vector<int32_t> inc_ptr;       // [nn+1]
    std::vector<int32_t> inc;           // [ninc] e * nb + a, ascending e per node
    std::vector<int32_t> inc_e;         // [ninc] e
    std::vector<uint8_t> inc_a;         // [ninc] a
    std::vector<uint16_t> pos;          // [ninc][nb] column block of node b in row n
    std::vector<double> geo;            // [nc][dim*dim + 1]: G = J^-1 (row-major), |det J|
    bool uniform = false;               // every cell has the same Jacobian
    bool nonaffine = false;             // some tensor cell is not a parallelogram / parallelepiped
    std::vector<double> xcell;          // [nc][nvc][dim] corner coordinates (non-affine meshes)
    bool lattice = false;               // order-1 box lattice in canonical numbering
    int lat_n[3] = {1, 1, 1};           // cells per axis
    std::vector<float2> sectors;        // [2^d][d][d] Walsh-sector blocks of K^0 (empty: no split)
    int lat_kshift = 0;                 // the kappa pairs hold kappa 2^-lat_kshift
    int max_deg = 0;
};

bool setup_host_mesh(int dim, int cell, int order, int64_t nv, const double *coords, int64_t nc,
                     const int32_t *cv, const RefElement &ref, HostMesh &hm, std::string &err);
void build_csr(const HostMesh &hm, std::vector<int64_t> &indptr, std::vector<int32_t> &indices);

// ---------------------------------------------------------------- device mesh
struct DeviceMesh {
    int64_t *indptr = nullptr;     // [ndof+1]
    int32_t *indices = nullptr;    // [nnz]
    int32_t *cell_node = nullptr;  // [nc][nb]
    int64_t *node_off = nullptr;   // [nn+1]
    int32_t *inc_ptr = nullptr;    // [nn+1]
    int32_t *inc = nullptr;        // [ninc]
    int32_t *inc_e = nullptr;      // [ninc] cell of each incidence
    uint8_t *inc_a = nullptr;      // [ninc] local node of each incidence
    uint16_t *pos = nullptr;       // [ninc][nb]
    double *geo = nullptr;         // [nc][dim*dim+1]
    double *M = nullptr;           // reference integrals [dim][dim][nb][nb]
    double *xcell = nullptr;       // non-affine meshes: corner coordinates [nc][nvc][dim]
    double *qw = nullptr;          //   quadrature weights [nq]
    double *qdphi = nullptr;       //   basis gradients at the points [nq][nb][dim]
    double *qdgeo = nullptr;       //   vertex-basis gradients at the points [nq][nvc][dim]
    int nq = 0;
    void *K = nullptr;             // uniform: [ldof][ldof]; cached: [nc][ldof][ldof]
    double *scratch = nullptr;     // partial sums
    int64_t scratch_len = 0;
    unsigned *counter = nullptr;   // last-block ticket of the grid sums (zero between calls)
    // order-1 box lattice path
    float2 *Edf = nullptr;         // [nc] element moduli as float pairs
    float2 *kappa = nullptr;       // [3^d][d][d] reference blocks as float pairs
    double *K0 = nullptr;          // [ldof][ldof] unit-modulus matrix in FP64
    float2 *sectors = nullptr;     // [2^d][d][d] Walsh-sector blocks of K^0 (nullptr: no split)
    unsigned *lat_bad = nullptr;   // generation of the last call that met out-of-range moduli
    // general path
    float2 *udf = nullptr;         // [ndof] u as float pairs (general path; lattice: one-call step)
    double *part = nullptr;        // [nc][nb] per-(cell, node) partials of u_e^T K_e^0 u_e
    // meshes of affine cells: strain-energy sensitivities (contract.cu)
    bool strain = false;           // the sensitivities take k_strain_energy
    float2 *sgeo = nullptr;        //   [nc, or 1 when uniform][d*d + 1] G and |det J| as float pairs
    float2 *sq = nullptr;          //   quadrature: weights [snq], reference gradients [snq][nb][d]
    int snq = 0;
    float2 *ssf = nullptr;         //   hexahedra of order 2, 3: 1D weights, basis values and derivatives,
                                   //   local nodes' lattice indices (k_strain_hex_sf)
    // FP32 element matrices of affine cells: assembled by contraction per call
    bool contract = false;         // the assembly takes k_contract_pairs (2D) or k_contract_rows (3D)
    float4 *cgeo = nullptr;        //   [nc][2 or 3] G and |det J| in FP32
    float *Mf = nullptr;           //   [nb][nb][4 or 12] reference integrals in FP32
    // node pairs in tiles of 32 (2D: {a, b} with b = a or b after a; 3D: every
    // ordered pair); also for the cached FP64 element matrices of 2D affine meshes
    // (pcached) and the one element matrix of a uniform mesh (puniform)
    bool pcached = false;
    bool puniform = false;         //   the pair kernel over the one element matrix of a uniform mesh
    int64_t ptiles = 0;            //   tiles
    uint32_t *ptoff = nullptr;     //   [8 chunks + 16] first record of each tile / 32
    uint32_t *pia = nullptr;       //   [256 chunks] value index of block (a, b) / d
    uint32_t *pib = nullptr;       //   [256 chunks] value index of block (b, a) / d (3D: = pia)
    uint32_t *pmeta = nullptr;     //   [256 chunks] cells | a's row length << 10 | b's << 21
    int32_t *pre = nullptr;        //   per record: the cell (ascending per pair)
    uint16_t *prm = nullptr;       //   per record: a_loc nb + b_loc (pcached, puniform: a_loc << 8 | b_loc)
    float4 *pblk = nullptr;        //   pcached: per record its 2 x 2 block of K_e^0 (2 float4s)
    // 3D: each node's cells as a chain, walked by the node's group of lanes
    int4 *cnrec = nullptr;         //   [nn] nodes by incident-cell count, largest first: row block
                                   //   offset (2 ints), first incidence, cells << 16 | degree
    int32_t *cinc_e = nullptr;     //   [ninc] each node's cells in the contraction's chain order
    uint8_t *cinc_a = nullptr;     //   [ninc] the node's local index in those cells
    uint16_t *crec = nullptr;      //   [ninc][nb] per lane: block p, local node b << 9, first/last flags
    unsigned *cticket = nullptr;   //   [2] work counter and finished warps or CTAs (zero between calls)
    // equilibrium solve (allocated by the first soptx_solve_cg)
    double *cg = nullptr;          // r z p q diag [ndof], scalars, partials, counters
    cudaGraphExec_t cg_exec = nullptr; // the CG iterations between two checks, as a graph
    cudaStream_t cg_cap = nullptr;     // its capture stream
    const void *cg_key[4] = {};        // vals, fixed, u and the iteration count it was made for
    // K(rho) for the backward's u-gradient (made by the first soptx_compliance_vjp with d_grad_u)
    double *kvals = nullptr;
    // the step from host buffers (made by the first soptx_step_host)
    double *stage = nullptr;           // rho [nc], u [ndof], dc [nc], c [1] on the device
    cudaStream_t side = nullptr;       // second stream: u's copy, the sensitivities, dc and c back
    cudaEvent_t ev[2] = {};            // rho on the device (and all work before it), side stream done
};

struct Material {
    double E0, Emin, nu, p;
    double dE;          // E0 - Emin
    double lam, mu;     // Lame constants at E = 1 (plane stress: lam*)
    int p_int;          // p when p is a small positive integer, else 0
};

}  // namespace soptx

struct soptx_mesh_s {
    soptx::HostMesh h;
    soptx::DeviceMesh d;
    soptx::Material mat;
    soptx_material user_mat;
    int prec = SOPTX_ELEM_FP64;
    soptx_path path = SOPTX_PATH_CACHED;
    int64_t device_bytes = 0;
    mutable uint32_t lattice_gen = 0;   // calls of the 3D lattice assembly (marks the out-of-range flag)
};

namespace soptx {
// ---------------------------------------------------------------- launchers (kernels.cu)
cudaError_t launch_element_matrices(const soptx_mesh_s &m, int64_t n_elems, cudaStream_t st);
cudaError_t launch_assemble(const soptx_mesh_s &m, const double *rho, double *vals, cudaStream_t st);
cudaError_t launch_sensitivity(const soptx_mesh_s &m, const double *rho, const double *u, double *dc,
                               double *c, double scale, const double *gscale, cudaStream_t st);
cudaError_t launch_Ku(const soptx_mesh_s &m, const double *rho, const double *u, const double *gout,
                      double *out, cudaStream_t st);
cudaError_t launch_scaled_product(const soptx_mesh_s &m, const double *vals, const double *u, const double *gout,
                                  double *out, cudaStream_t st);
int64_t sensitivity_scratch_len(const soptx_mesh_s &m);
cudaError_t launch_lattice_assemble(const soptx_mesh_s &m, const double *rho, double *vals, cudaStream_t st);
bool lattice_kappa_shift(int dim, const std::vector<double> &K0, int &shift);
void build_lattice_kappa(int dim, const std::vector<double> &K0, int shift, std::vector<float2> &kappa);
bool build_lattice_sectors(int dim, const std::vector<double> &K0, double zero_tol, std::vector<float2> &B);
cudaError_t launch_lattice_sensitivity(const soptx_mesh_s &m, const double *rho, const double *u, double *out,
                                       double *c, const double *gscale, cudaStream_t st);
int lattice_sens_grid(int64_t nc);
cudaError_t launch_lattice_step(const soptx_mesh_s &m, const double *rho, const double *u, double *vals, double *dc,
                                double *c, cudaStream_t st, const double *gscale = nullptr);
// Grouped one-call steps of small 2D and 3D box lattices (a cluster of 8 CTAs each, one launch
// per 32 meshes of a dimension); the meshes must be distinct and lattice_groupable.
bool lattice_groupable(const soptx_mesh_s &m);
cudaError_t launch_lattice_group(const soptx_mesh_s *const *ms, const double *const *rho, const double *const *u,
                                 double *const *vals, double *const *dc, double *const *c, int n, cudaStream_t st);
cudaError_t launch_gather(const soptx_mesh_s &m, const double *rho, const double *u, double *vals, double *dc,
                          double *c, const double *gscale, cudaStream_t st);
int gather_finalize_grid(int64_t nc);
cudaError_t launch_prep(const soptx_mesh_s &m, const double *rho, const double *u, cudaStream_t st);
// contract.cu
bool contract_fits(int dim, int nb, int max_deg);
bool pairs_fit(int dim, int nb, int max_deg);
cudaError_t launch_contract_assemble(const soptx_mesh_s &m, const double *rho, double *vals, cudaStream_t st);
cudaError_t launch_pair_blocks(const soptx_mesh_s &m, int64_t nrec, cudaStream_t st);
// max_grid > 0 caps the blocks (the kernel loops over the cells): beside a
// persistent assembly, a block per SM leaves it the rest of the GPU
cudaError_t launch_strain_sensitivity(const soptx_mesh_s &m, const double *rho, const double *u, double *out,
                                      double *c, const double *gscale, cudaStream_t st, int max_grid = 0);
cudaError_t launch_step(const soptx_mesh_s &m, const double *rho, const double *u, double *vals, double *dc,
                        double *c, cudaStream_t st, const double *gscale = nullptr);
__global__ void k_reduce_partials(int n, const double *__restrict__ partial, double *__restrict__ c);
}  // namespace soptx
