"""Shared test helpers: small meshes and oracle comparisons."""
import numpy as np

import oracle
from paper_2505_02438_gb300 import workloads as W

# FP64 form: |K_gpu - K_ref| <= TOL64 * sum_e |E_e K_e^0[a,b]| per CSR entry,
# |dc_gpu - dc_ref| <= TOL64 * |E'_e| sum_ab |u_a K_ab u_b| per cell.
TOL64 = 1e-12
# FP32 element matrices (FP64 accumulation): the element entries carry a
# relative error of a few FP32 ulps (2^-24 ~ 6e-8) from the contraction.
TOL32 = 2e-6


def relabel(coords, cells, seed):
    perm = np.random.default_rng(seed).permutation(len(coords))
    out = np.empty_like(coords)
    out[perm] = coords
    return out, perm[cells].astype(np.int32)


def small_cases():
    """(name, cell, order, coords, cells) covering every cell type and order,
    several tiles and ragged tails."""
    g = lambda s: np.random.default_rng(s)
    cases = []
    c, cl = W.structured_quad(60, 20)
    cases.append(("q4_60x20_lattice", "quad", 1, c, cl))
    c, cl = W.structured_hex(13, 5, 4)
    cases.append(("hex_q1_13x5x4_lattice", "hex", 1, c, cl))
    c, cl = relabel(*W.structured_hex(6, 3, 2), 3)
    cases.append(("hex_q1_relabelled_uniform", "hex", 1, c, cl))
    c, cl = W.structured_quad(7, 5)
    cases.append(("quad_q2_7x5", "quad", 2, c, cl))
    c, cl = W.structured_quad(5, 3)
    cases.append(("quad_q3_5x3", "quad", 3, c, cl))
    c, cl = W.structured_hex(4, 3, 2)
    cases.append(("hex_q2_4x3x2", "hex", 2, c, cl))
    c, cl = W.structured_hex(2, 2, 1)
    cases.append(("hex_q3_2x2x1", "hex", 3, c, cl))
    # general (non-affine) bilinear / trilinear cells: Gauss quadrature per cell
    for k in (1, 2, 3):
        c, cl = W.quad_grid(9, 6, 0.2, g(20 + k))
        cases.append(("quad_q%d_9x6_distorted" % k, "quad", k, c, cl))
    for k, sh in ((1, (5, 4, 3)), (2, (3, 3, 2)), (3, (2, 2, 2))):
        c, cl = W.hex_grid(*sh, 0.15, g(30 + k))
        cases.append(("hex_q%d_%dx%dx%d_distorted" % ((k,) + sh), "hex", k, c, cl))
    for k in (1, 2, 3):
        c, cl = W.triangle_grid(17, 9, 0.2, g(k))
        cases.append(("tri_p%d_17x9_jitter" % k, "tri", k, c, cl))
    for k in (1, 2, 3):
        c, cl = W.kuhn_tets(5, 3, 2, 0.15, g(10 + k))
        cases.append(("tet_p%d_5x3x2_jitter" % k, "tet", k, c, cl))
    return cases


def oracle_csr(cell, k, coords, cells, mat, rho, rows=None):
    rp, ci, v, ndof = oracle.assemble(cell, k, coords, cells, mat, rho, rows=rows)
    _, _, va, _ = oracle.assemble(cell, k, coords, cells, mat, rho, rows=rows, absval=True)
    return rp, ci, v, va, ndof


def _oracle_rows_job(job):
    """One worker of oracle_full_parallel: the oracle's rows [r0, r1), their
    values and the per-entry scale (sum of |contributions|)."""
    cell, k, coords, cells, mat, rho, r0, r1 = job
    rows = np.arange(r0, r1, dtype=np.int64)
    rp, ci, v, ndof = oracle.assemble(cell, k, coords, cells, mat, rho, rows=rows)
    _, _, va, _ = oracle.assemble(cell, k, coords, cells, mat, rho, rows=rows, absval=True)
    return rp, ci, v, va, ndof


def _oracle_sens_job(job):
    cell, k, coords, cells, mat, rho, u, e0, e1 = job
    sel = np.arange(e0, e1, dtype=np.int64)
    dc, s, _, sa = oracle.sensitivity(cell, k, coords, cells, mat, rho, u, sel=sel, with_abs=True)
    return dc, s, sa


def _pool_size():
    import os
    n = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    return max(1, min(16, n))


def oracle_full_parallel(cell, k, coords, cells, mat, rho, u, ndof):
    """The oracle's whole CSR matrix (rowptr, cols, vals, |contribution| sums)
    and every cell's (dc, s, sum_ab |u_a K_ab u_b|), computed by the oracle
    unchanged over contiguous row and cell ranges in a spawned process pool
    (spawn: safe in a process that has used the GPU)."""
    import multiprocessing as mp
    n = _pool_size()
    rb = np.linspace(0, ndof, 4 * n + 1).astype(np.int64)
    cb = np.linspace(0, len(cells), 2 * n + 1).astype(np.int64)
    rjobs = [(cell, k, coords, cells, mat, rho, int(a), int(b)) for a, b in zip(rb[:-1], rb[1:]) if b > a]
    cjobs = [(cell, k, coords, cells, mat, rho, u, int(a), int(b)) for a, b in zip(cb[:-1], cb[1:]) if b > a]
    with mp.get_context("spawn").Pool(n) as pool:
        rparts = pool.map(_oracle_rows_job, rjobs)
        cparts = pool.map(_oracle_sens_job, cjobs)
    assert all(p[4] == ndof for p in rparts)
    rowptr = [np.zeros(1, np.int64)]
    base = 0
    for rp, _, _, _, _ in rparts:
        rowptr.append(rp[1:] + base)
        base += rp[-1]
    rowptr = np.concatenate(rowptr)
    cols = np.concatenate([p[1] for p in rparts])
    vals = np.concatenate([p[2] for p in rparts])
    va = np.concatenate([p[3] for p in rparts])
    dc = np.concatenate([p[0] for p in cparts])
    s = np.concatenate([p[1] for p in cparts])
    sa = np.concatenate([p[2] for p in cparts])
    return rowptr, cols, vals, va, dc, s, sa
