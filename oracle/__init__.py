"""Ctypes binding of the plain FP64 CPU oracle in ``oracle.c``.

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module; the library under ``paper_2505_02438_gb300`` never does.  The oracle
shares no code with the CUDA path.

Every function takes plain numpy arrays:
  coords  float64 [NV, d]   vertex coordinates
  cells   int32   [NC, nv]  vertex ids per cell, in reference vertex order
                            (simplex: origin first, then the unit-vector
                            vertices; tensor cells: lexicographic, x fastest)
  mat     (E0, Emin, nu, p, plane_strain)
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_liboracle.so")

CELL = {"tri": 0, "tet": 1, "quad": 2, "hex": 3}
DIM = {"tri": 2, "tet": 3, "quad": 2, "hex": 3}
NVERT = {"tri": 3, "tet": 4, "quad": 4, "hex": 8}

_lib = None


def build(force=False):
    """Compile oracle.c into _liboracle.so beside it (plain gcc, no OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        i32, i64, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.or_ref_lattice.argtypes = [i32, i32, P, P]
        lib.or_basis_eval.argtypes = [i32, i32, i32, P, P, P]
        lib.or_gauss_legendre.argtypes = [i32, P, P]
        lib.or_ref_quadrature.argtypes = [i32, i32, P, P, P]
        lib.or_element_matrix.argtypes = [i32, i32, P, dbl, i32, P]
        lib.or_number.argtypes = [i32, i32, i64, i64, P, P, P]
        lib.or_node_coords.argtypes = [i32, i32, i64, P, P, P, i64, P]
        lib.or_assemble_rows.argtypes = [i32, i32, i64, P, i64, P, dbl, dbl, dbl, dbl, i32,
                                         P, i64, P, i32, P, P, P, P, P]
        lib.or_sensitivity.argtypes = [i32, i32, i64, P, i64, P, dbl, dbl, dbl, dbl, i32,
                                       P, P, i64, P, P, P, P, P]
        lib.or_compliance_vjp.argtypes = [i32, i32, i64, P, i64, P, dbl, dbl, dbl, dbl, i32,
                                          P, P, dbl, P, P]
        lib.or_free.argtypes = [P]
        for f in ("or_ref_lattice", "or_basis_eval", "or_gauss_legendre", "or_ref_quadrature",
                  "or_element_matrix", "or_number", "or_node_coords", "or_assemble_rows",
                  "or_sensitivity", "or_compliance_vjp"):
            getattr(lib, f).restype = ctypes.c_int
        lib.or_free.restype = None
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))


def ref_lattice(cell, k):
    lat = np.zeros((64, 3), np.int32)
    nb = ctypes.c_int(0)
    _check(_L().or_ref_lattice(CELL[cell], k, ctypes.byref(nb), _p(lat)), "ref_lattice")
    return lat[: nb.value].copy()


def basis_eval(cell, k, x):
    x = np.ascontiguousarray(np.atleast_2d(x), np.float64)
    if x.shape[1] < 3:
        x = np.hstack([x, np.zeros((x.shape[0], 3 - x.shape[1]))])
    nb = len(ref_lattice(cell, k))
    phi = np.zeros((len(x), nb))
    dphi = np.zeros((len(x), nb, 3))
    _check(_L().or_basis_eval(CELL[cell], k, len(x), _p(x), _p(phi), _p(dphi)), "basis_eval")
    return phi, dphi[:, :, : DIM[cell]]


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    _check(_L().or_gauss_legendre(n, _p(x), _p(w)), "gauss_legendre")
    return x, w


def ref_quadrature(cell, n):
    x = np.zeros((n ** 3, 3))
    w = np.zeros(n ** 3)
    nq = ctypes.c_int(0)
    _check(_L().or_ref_quadrature(CELL[cell], n, ctypes.byref(nq), _p(x), _p(w)), "ref_quadrature")
    return x[: nq.value, : DIM[cell]].copy(), w[: nq.value].copy()


def element_matrix(cell, k, xv, nu, plane_strain=False):
    """K_e^0 (unit modulus) of one cell with vertex coordinates xv [nv, d]."""
    xv = np.ascontiguousarray(xv, np.float64)
    nb = len(ref_lattice(cell, k))
    ldof = DIM[cell] * nb
    Ke = np.zeros((ldof, ldof))
    _check(_L().or_element_matrix(CELL[cell], k, _p(xv), float(nu), int(plane_strain), _p(Ke)),
           "element_matrix")
    return Ke


def number(cell, k, nv, cells):
    """Global Lagrange node of every (cell, local node): (cell_node [NC, nb], NN)."""
    cells = np.ascontiguousarray(cells, np.int32)
    nb = len(ref_lattice(cell, k))
    cn = np.zeros((len(cells), nb), np.int32)
    nn = ctypes.c_int64(0)
    _check(_L().or_number(CELL[cell], k, int(nv), len(cells), _p(cells), _p(cn), ctypes.byref(nn)),
           "number")
    return cn, nn.value


def node_coords(cell, k, coords, cells):
    coords = np.ascontiguousarray(coords, np.float64)
    cells = np.ascontiguousarray(cells, np.int32)
    cn, nn = number(cell, k, len(coords), cells)
    xn = np.zeros((nn, DIM[cell]))
    _check(_L().or_node_coords(CELL[cell], k, len(cells), _p(cells), _p(coords), _p(cn), nn, _p(xn)),
           "node_coords")
    return xn


def assemble(cell, k, coords, cells, mat, rho, rows=None, absval=False):
    """K(rho) in CSR.  rows=None: every row; else only the listed dof rows, in
    that order.  absval=True sums |E_e K_e^0[a,b]| instead (the per-entry
    rounding scale).  Returns (rowptr int64, cols int32, vals float64, ndof)."""
    lib = _L()
    coords = np.ascontiguousarray(coords, np.float64)
    cells = np.ascontiguousarray(cells, np.int32)
    rho = np.ascontiguousarray(rho, np.float64)
    E0, Emin, nu, p, ps = mat
    if rows is None:
        nsel, sel = -1, None
    else:
        sel = np.ascontiguousarray(rows, np.int64)
        nsel = len(sel)
    nnz = ctypes.c_int64(0)
    ndof = ctypes.c_int64(0)
    rp = ctypes.POINTER(ctypes.c_int64)()
    ci = ctypes.POINTER(ctypes.c_int32)()
    vv = ctypes.POINTER(ctypes.c_double)()
    rc = lib.or_assemble_rows(CELL[cell], k, len(coords), _p(coords), len(cells), _p(cells),
                              E0, Emin, nu, p, int(ps), _p(rho), nsel,
                              _p(sel) if sel is not None else None, int(bool(absval)),
                              ctypes.byref(nnz), ctypes.byref(rp), ctypes.byref(ci),
                              ctypes.byref(vv), ctypes.byref(ndof))
    _check(rc, "assemble")
    nrows = ndof.value if rows is None else nsel
    rowptr = np.ctypeslib.as_array(rp, shape=(nrows + 1,)).copy()
    cols = np.ctypeslib.as_array(ci, shape=(max(nnz.value, 1),))[: nnz.value].copy()
    vals = np.ctypeslib.as_array(vv, shape=(max(nnz.value, 1),))[: nnz.value].copy()
    for ptr in (rp, ci, vv):
        lib.or_free(ctypes.cast(ptr, ctypes.c_void_p))
    return rowptr, cols, vals, ndof.value


def sensitivity(cell, k, coords, cells, mat, rho, u, sel=None, with_abs=False):
    """(dc, s, c): dc_e = -E'(rho_e) s_e, s_e = u_e^T K_e^0 u_e, c = sum_e E_e s_e
    (c is NaN when only a subset of cells is selected).  with_abs=True appends
    sabs_e = sum_ab |u_a K_ab u_b| (the rounding scale of s_e)."""
    coords = np.ascontiguousarray(coords, np.float64)
    cells = np.ascontiguousarray(cells, np.int32)
    rho = np.ascontiguousarray(rho, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    E0, Emin, nu, p, ps = mat
    if sel is None:
        n, nsel, selp = len(cells), -1, None
    else:
        sel = np.ascontiguousarray(sel, np.int64)
        n, nsel, selp = len(sel), len(sel), _p(sel)
    dc = np.zeros(n)
    s = np.zeros(n)
    sa = np.zeros(n)
    c = ctypes.c_double(0.0)
    _check(_L().or_sensitivity(CELL[cell], k, len(coords), _p(coords), len(cells), _p(cells),
                               E0, Emin, nu, p, int(ps), _p(rho), _p(u), nsel, selp,
                               _p(dc), _p(s), _p(sa), ctypes.byref(c)), "sensitivity")
    if with_abs:
        return dc, s, c.value, sa
    return dc, s, c.value


def compliance_vjp(cell, k, coords, cells, mat, rho, u, g, want_u=True):
    coords = np.ascontiguousarray(coords, np.float64)
    cells = np.ascontiguousarray(cells, np.int32)
    rho = np.ascontiguousarray(rho, np.float64)
    u = np.ascontiguousarray(u, np.float64)
    E0, Emin, nu, p, ps = mat
    gr = np.zeros(len(cells))
    gu = np.zeros(len(u)) if want_u else None
    _check(_L().or_compliance_vjp(CELL[cell], k, len(coords), _p(coords), len(cells), _p(cells),
                                  E0, Emin, nu, p, int(ps), _p(rho), _p(u), float(g), _p(gr),
                                  _p(gu) if want_u else None), "compliance_vjp")
    return gr, gu


def spmv(rowptr, cols, vals, x):
    """y = K x for a CSR matrix, row by row in column order (plain loops over
    numpy slices)."""
    x = np.asarray(x, np.float64)
    y = np.zeros(len(rowptr) - 1)
    for r in range(len(y)):
        sl = slice(rowptr[r], rowptr[r + 1])
        y[r] = np.dot(vals[sl], x[cols[sl]])
    return y


def solve_dirichlet(rowptr, cols, vals, fixed, f, u_fixed):
    """The discrete equilibrium K u = f (Sec. 2.2) with Dirichlet constraints:
    u = u_fixed on the constrained dofs, K_ff u_f = f_f - K_fd u_d on the free
    ones, solved directly (scipy's sparse LU as the library routine).
    Returns u [ndof]."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    n = len(rowptr) - 1
    K = sp.csr_matrix((vals, cols, rowptr), shape=(n, n))
    fixed = np.asarray(fixed, bool)
    free = ~fixed
    u = np.zeros(n)
    u[fixed] = np.asarray(u_fixed, np.float64)[fixed]
    rhs = np.asarray(f, np.float64)[free] - K[free][:, fixed] @ u[fixed]
    u[free] = spla.spsolve(K[free][:, free].tocsc(), rhs)
    return u


# ---------------------------------------------------------------- after the sensitivities (Sec. 2.3-2.4)

def filter_weights(centroids, rmin):
    """H_ij = max(0, rmin - |c_i - c_j|) (Sec. 2.4), by brute force over all
    pairs, row by row; returns a scipy CSR matrix."""
    import scipy.sparse as sp
    c = np.asarray(centroids, np.float64)
    rows, cols, vals = [], [], []
    for i in range(len(c)):
        dist = np.sqrt(((c - c[i]) ** 2).sum(axis=1))
        j = np.nonzero(dist < rmin)[0]
        rows.append(np.full(len(j), i))
        cols.append(j)
        vals.append(rmin - dist[j])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(len(c), len(c)))


def sensitivity_filter(H, rho, dc, gamma=1e-3):
    """Sigmund's filter (Sec. 2.4): sum_j H_ij rho_j dc_j / (max(gamma, rho_i) sum_j H_ij)."""
    return (H @ (rho * dc)) / (np.maximum(gamma, rho) * np.asarray(H.sum(axis=1)).ravel())


def density_filter(H, vol, x):
    """Density filter (Sec. 2.4): sum_j H_ij v_j x_j / sum_j H_ij v_j."""
    return (H @ (vol * x)) / (H @ vol)


def density_filter_grad(H, vol, g):
    """The density filter's chain rule (Sec. 2.4):
    d psi / d x_j = sum_i H_ij v_j / (sum_k H_ik v_k) d psi / d rho~_i."""
    return vol * (H.T @ (g / (H @ vol)))


def heaviside(x, beta):
    """Heaviside projection and its derivative (Sec. 2.4)."""
    t = np.exp(-beta * x)
    return 1.0 - t + x * np.exp(-beta), beta * t + np.exp(-beta)


def oc_update(rho, dc, dv, vol, volfrac, move=0.2, eta=0.5, l_lo=0.0, l_hi=1e9, tol=1e-3):
    """Optimality criteria (Sec. 2.3, Algorithm 1): rho_e B_e^eta clamped to
    the move limits, B_e = -dc_e / (lambda dv_e), lambda by bisection on the
    volume until (l_hi - l_lo) / (l_hi + l_lo) <= tol; rho_e B_e^eta is
    evaluated as q_e lambda^-eta with q_e = rho_e (max(0, -dc_e) / dv_e)^eta.
    Returns (rho_new, lambda)."""
    rho = np.asarray(rho, np.float64)
    q = rho * np.power(np.maximum(0.0, -np.asarray(dc)) / np.asarray(dv), eta)
    lo_b, hi_b = np.maximum(0.0, rho - move), np.minimum(1.0, rho + move)
    target = volfrac * np.sum(vol)
    lo, hi, lmid = l_lo, l_hi, 0.5 * (l_lo + l_hi)
    for _ in range(100):
        if not (hi - lo) / (hi + lo) > tol:
            break
        lmid = 0.5 * (hi + lo)
        x = np.minimum(hi_b, np.maximum(lo_b, q * lmid ** (-eta)))
        if np.dot(vol, x) > target:
            lo = lmid
        else:
            hi = lmid
    return np.minimum(hi_b, np.maximum(lo_b, q * lmid ** (-eta))), lmid


def oc_loop(cell, k, coords, cells, mat, fixed, f, rmin, volfrac, vol, centroids, max_iter=200, tol=1e-2,
            move=0.2, eta=0.5, callback=None):
    """Compliance minimisation by Algorithm 1 (Sec. 2.3) with the sensitivity
    filter (Sec. 2.4), every step plain: K(rho) and u by the oracle's assembly
    and direct constrained solve, dc and c by the oracle's sensitivity, the
    filter and the OC update above; stops when max |rho_new - rho| <= tol.
    Returns (rho, history [(c, change)])."""
    H = filter_weights(centroids, rmin)
    x = np.full(len(cells), float(volfrac))
    hist = []
    for it in range(max_iter):
        rp, ci, v, ndof = assemble(cell, k, coords, cells, mat, x)
        u = solve_dirichlet(rp, ci, v, fixed, f, np.zeros(ndof))
        dc, s, c = sensitivity(cell, k, coords, cells, mat, x, u)
        xnew, lam = oc_update(x, sensitivity_filter(H, x, dc), vol, vol, volfrac, move, eta)
        change = float(np.abs(xnew - x).max())
        hist.append((float(c), change))
        if callback:
            callback(it, hist[-1])
        x = xnew
        if change <= tol:
            break
    return x, hist
