"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the
mathematics, not by the oracle itself (CPU only).

Each test names what fixes the expected value: a closed form, an invariant,
a special case that reduces to a textbook formula or a library routine, brute
force on a tiny mesh, or a count the paper prints.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2505_02438_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

REF_VERTS = {
    "tri": np.array([[0, 0], [1, 0], [0, 1]], float),
    "tet": np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float),
    "quad": np.array([[0, 0], [1, 0], [0, 1], [1, 1]], float),
    "hex": np.array([[i, j, l] for l in (0, 1) for j in (0, 1) for i in (0, 1)], float),
}
CELLS_ORDERS = [(c, k) for c in ("tri", "tet", "quad", "hex") for k in (1, 2, 3)]


def geo_map(cell, xv, xi):
    """Textbook geometric map of a reference point: affine for simplices,
    multilinear (tensor product of (1 - t, t)) for quads / hexes."""
    xi = np.asarray(xi, float)
    if cell in ("tri", "tet"):
        return xv[0] + sum(xi[m] * (xv[m + 1] - xv[0]) for m in range(len(xv) - 1))
    d = xv.shape[1]
    x = np.zeros(d)
    for v in range(len(xv)):
        w = 1.0
        for m in range(d):
            w *= xi[m] if (v >> m) & 1 else 1.0 - xi[m]
        x += w * xv[v]
    return x


def local_node_positions(cell, k, xv):
    lat = oracle.ref_lattice(cell, k)
    return np.array([geo_map(cell, xv, l[: xv.shape[1]] / k) for l in lat])


def affine_cell(cell, rng):
    """A random, well-shaped affine cell (parallelogram / parallelepiped for
    tensor cells)."""
    d = W.DIM[cell]
    while True:
        A = np.eye(d) + 0.3 * rng.standard_normal((d, d))
        if np.linalg.det(A) > 0.3:
            break
    x0 = rng.standard_normal(d)
    return np.array([x0 + A @ r for r in REF_VERTS[cell]])


def rigid_modes(pos):
    n, d = pos.shape
    modes = []
    for i in range(d):
        t = np.zeros((n, d))
        t[:, i] = 1.0
        modes.append(t.ravel())
    if d == 2:
        modes.append(np.stack([-pos[:, 1], pos[:, 0]], 1).ravel())
    else:
        for w in np.eye(3):
            modes.append(np.cross(w, pos).ravel())
    return np.array(modes)


# ---------------------------------------------------------------- quadrature

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8])
def test_gauss_legendre_matches_numpy_and_is_exact(n):
    x, w = oracle.gauss_legendre(n)
    t, v = np.polynomial.legendre.leggauss(n)      # library routine on [-1, 1]
    np.testing.assert_allclose(np.sort(x), np.sort((t + 1) / 2), rtol=0, atol=1e-15)
    np.testing.assert_allclose(w[np.argsort(x)], (v / 2)[np.argsort(t)], rtol=1e-14)
    for m in range(2 * n):
        assert abs(np.dot(w, x ** m) - 1.0 / (m + 1)) < 1e-15


@pytest.mark.parametrize("cell,n", [("tri", 2), ("tri", 3), ("tri", 4), ("tet", 2), ("tet", 3), ("tet", 4)])
def test_simplex_quadrature_monomials(cell, n):
    """int_T xi^alpha = alpha! / (|alpha| + d)!  (Dirichlet integral)."""
    x, w = oracle.ref_quadrature(cell, n)
    d = W.DIM[cell]
    top = 2 * n - 2 if d == 2 else 2 * n - 3
    for alpha in itertools.product(range(top + 1), repeat=d):
        if sum(alpha) > top:
            continue
        exact = np.prod([math.factorial(a) for a in alpha]) / math.factorial(sum(alpha) + d)
        got = np.dot(w, np.prod(x ** np.array(alpha), axis=1))
        assert abs(got - exact) < 1e-15, (alpha, got, exact)


# ---------------------------------------------------------------- basis

@pytest.mark.parametrize("cell,k", CELLS_ORDERS)
def test_basis_is_nodal_and_reproduces_polynomials(cell, k):
    lat = oracle.ref_lattice(cell, k)
    d = W.DIM[cell]
    nb = {"tri": (k + 1) * (k + 2) // 2, "tet": (k + 1) * (k + 2) * (k + 3) // 6,
          "quad": (k + 1) ** 2, "hex": (k + 1) ** 3}[cell]
    assert len(lat) == nb
    xi = lat[:, :d] / k
    phi, _ = oracle.basis_eval(cell, k, xi)
    np.testing.assert_allclose(phi, np.eye(nb), atol=1e-13)
    rng = np.random.default_rng(7)
    pts = rng.uniform(0, 1, (20, d))
    if cell in ("tri", "tet"):
        pts = pts / (1.0 + pts.sum(1, keepdims=True))
    phi, dphi = oracle.basis_eval(cell, k, pts)
    np.testing.assert_allclose(phi.sum(1), 1.0, atol=1e-13)
    np.testing.assert_allclose(dphi.sum(1), 0.0, atol=1e-12)
    # reproduces every monomial of total degree <= k (contained in P_k and Q_k)
    for alpha in itertools.product(range(k + 1), repeat=d):
        if sum(alpha) > k:
            continue
        nodal = np.prod(xi ** np.array(alpha), axis=1)
        exact = np.prod(pts ** np.array(alpha), axis=1)
        np.testing.assert_allclose(phi @ nodal, exact, atol=1e-12)


def test_p2_triangle_basis_textbook():
    """P2 triangle: vertex functions l(2l - 1), edge functions 4 l_i l_j."""
    pts = np.array([[0.2, 0.3], [0.1, 0.7], [0.45, 0.05]])
    phi, _ = oracle.basis_eval("tri", 2, pts)
    lat = oracle.ref_lattice("tri", 2)
    for q, (x, y) in enumerate(pts):
        lam = np.array([1 - x - y, x, y])
        for a, L in enumerate(lat):
            bc = np.array([2 - L[0] - L[1], L[0], L[1]])     # barycentric lattice index
            nz = np.nonzero(bc)[0]
            if len(nz) == 1:
                v = nz[0]
                want = lam[v] * (2 * lam[v] - 1)
            else:
                want = 4 * lam[nz[0]] * lam[nz[1]]
            assert abs(phi[q, a] - want) < 1e-14


# ---------------------------------------------------------------- element matrices

def test_q4_unit_square_closed_form():
    """Bilinear square, plane stress: exact symbolic integration of B^T D B
    with textbook shape functions, and the two first-row entries known in
    closed form, (1/2 - nu/6)/(1 - nu^2) and (1/8 + nu/8)/(1 - nu^2)."""
    sp = pytest.importorskip("sympy")
    x, y, nu = sp.symbols("x y nu")
    N = [(1 - x) * (1 - y), x * (1 - y), (1 - x) * y, x * y]
    B = sp.zeros(3, 8)
    for a, Na in enumerate(N):
        B[0, 2 * a] = sp.diff(Na, x)
        B[1, 2 * a + 1] = sp.diff(Na, y)
        B[2, 2 * a] = sp.diff(Na, y)
        B[2, 2 * a + 1] = sp.diff(Na, x)
    D = sp.Matrix([[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu) / 2]]) / (1 - nu ** 2)
    K = sp.integrate(sp.integrate(B.T * D * B, (x, 0, 1)), (y, 0, 1))
    assert sp.simplify(K[0, 0] - (sp.Rational(1, 2) - nu / 6) / (1 - nu ** 2)) == 0
    assert sp.simplify(K[0, 1] - (sp.Rational(1, 8) + nu / 8) / (1 - nu ** 2)) == 0
    for nv in (0.3, 0.0, 0.45):
        want = np.array(K.subs(nu, nv).evalf(30), dtype=float)
        got = oracle.element_matrix("quad", 1, REF_VERTS["quad"], nv)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("cell", ["tri", "tet"])
@pytest.mark.parametrize("plane_strain", [0, 1])
def test_p1_simplex_constant_strain(cell, plane_strain):
    """P1 simplices: K = |T| B^T D B with constant barycentric gradients."""
    rng = np.random.default_rng(11)
    d = W.DIM[cell]
    nu = 0.3
    for _ in range(5):
        xv = affine_cell(cell, rng)
        M = np.hstack([np.ones((d + 1, 1)), xv])       # rows [1, x_v]
        grads = np.linalg.inv(M)[1:, :].T              # [v, d]: grad of lambda_v
        vol = abs(np.linalg.det(M)) / math.factorial(d)
        ns = 3 if d == 2 else 6
        B = np.zeros((ns, d * (d + 1)))
        for a in range(d + 1):
            g = grads[a]
            if d == 2:
                B[0, 2 * a], B[1, 2 * a + 1] = g[0], g[1]
                B[2, 2 * a], B[2, 2 * a + 1] = g[1], g[0]
            else:
                B[0, 3 * a], B[1, 3 * a + 1], B[2, 3 * a + 2] = g
                B[3, 3 * a + 1], B[3, 3 * a + 2] = g[2], g[1]
                B[4, 3 * a], B[4, 3 * a + 2] = g[2], g[0]
                B[5, 3 * a], B[5, 3 * a + 1] = g[1], g[0]
        lam = nu / ((1 + nu) * (1 - 2 * nu))
        mu = 1 / (2 * (1 + nu))
        if d == 3:
            D = np.diag([2 * mu] * 3 + [mu] * 3)
            D[:3, :3] += lam
        elif plane_strain:
            D = np.array([[lam + 2 * mu, lam, 0], [lam, lam + 2 * mu, 0], [0, 0, mu]])
        else:
            D = np.array([[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu) / 2]]) / (1 - nu ** 2)
        want = vol * B.T @ D @ B
        got = oracle.element_matrix(cell, 1, xv, nu, plane_strain)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max())


@pytest.mark.parametrize("cell,k", CELLS_ORDERS)
def test_element_matrix_symmetric_psd_rigid_null_space(cell, k):
    rng = np.random.default_rng(100 + 7 * k)
    d = W.DIM[cell]
    nrig = 3 if d == 2 else 6
    for _ in range(3):
        xv = affine_cell(cell, rng)
        K = oracle.element_matrix(cell, k, xv, 0.3)
        scale = np.abs(K).max()
        np.testing.assert_allclose(K, K.T, atol=1e-14 * scale)
        ev = np.linalg.eigvalsh(K)
        assert ev[0] > -1e-12 * scale
        assert np.sum(ev < 1e-10 * scale) == nrig       # rank = ldof - rigid modes
        R = rigid_modes(local_node_positions(cell, k, xv))
        assert np.abs(K @ R.T).max() < 1e-12 * scale * max(1.0, np.abs(R).max())


@pytest.mark.parametrize("cell,k", [(c, k) for c in ("quad", "hex") for k in (1, 2, 3)])
def test_distorted_tensor_cell_symmetric_psd_rigid_null_space(cell, k):
    """General (non-affine) bilinear / trilinear cells: K_e^0 is still
    symmetric PSD with exactly the rigid-body null space (a rigid motion has
    zero strain at every quadrature point), and moving the corners changes it
    (it is not the parallelogram's matrix)."""
    rng = np.random.default_rng(300 + k)
    d = W.DIM[cell]
    nrig = 3 if d == 2 else 6
    for _ in range(2):
        xa = affine_cell(cell, rng)
        xv = xa + 0.12 * rng.standard_normal(xa.shape)
        K = oracle.element_matrix(cell, k, xv, 0.3)
        scale = np.abs(K).max()
        np.testing.assert_allclose(K, K.T, atol=1e-14 * scale)
        ev = np.linalg.eigvalsh(K)
        assert ev[0] > -1e-12 * scale
        assert np.sum(ev < 1e-10 * scale) == nrig
        R = rigid_modes(local_node_positions(cell, k, xv))
        assert np.abs(K @ R.T).max() < 1e-12 * scale * max(1.0, np.abs(R).max())
        assert np.abs(K - oracle.element_matrix(cell, k, xa, 0.3)).max() > 1e-3 * scale


@pytest.mark.parametrize("cell,k", [("tri", 2), ("tet", 2), ("quad", 2), ("hex", 1), ("tri", 3)])
def test_element_matrix_scaling_and_rotation(cell, k):
    rng = np.random.default_rng(5)
    d = W.DIM[cell]
    xv = affine_cell(cell, rng)
    K = oracle.element_matrix(cell, k, xv, 0.3)
    s = 2.5
    Ks = oracle.element_matrix(cell, k, s * xv, 0.3)
    np.testing.assert_allclose(Ks, K * (s if d == 3 else 1.0), atol=1e-12 * np.abs(K).max())
    Q, _ = np.linalg.qr(rng.standard_normal((d, d)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    Kr = oracle.element_matrix(cell, k, xv @ Q.T, 0.3)
    nb = K.shape[0] // d
    Rb = np.kron(np.eye(nb), Q)
    np.testing.assert_allclose(Kr, Rb @ K @ Rb.T, atol=1e-12 * np.abs(K).max())


@pytest.mark.parametrize("cell,k", [("quad", 1), ("hex", 1), ("tri", 3), ("tet", 2), ("quad", 2), ("hex", 2)])
def test_element_matrix_translation_invariance(cell, k):
    """K_e^0 depends on a cell's shape, not on where it sits: a cell moved far
    from the origin (here by about 1e3 to 2e4 edge lengths, as on the largest
    meshes) has the matrix of the same cell at the origin, to a few rounding
    errors of its entries, including entries that cancel (the Q4 coupling
    (nu - (1 - nu) / 2) / (4 (1 - nu^2)))."""
    rng = np.random.default_rng(9)
    d = W.DIM[cell]
    # vertices on a dyadic grid and integer shifts: the moved cell is exactly the same shape
    xv = np.round(affine_cell(cell, rng) * 2.0 ** 20) / 2.0 ** 20
    K = oracle.element_matrix(cell, k, xv, 0.3)
    for shift in (1e3, 2e4):
        t = np.round(shift * (1.0 + rng.uniform(size=d))) * np.where(rng.uniform(size=d) < 0.5, -1.0, 1.0)
        assert np.array_equal((xv + t) - t, xv)
        Kt = oracle.element_matrix(cell, k, xv + t, 0.3)
        assert np.all(np.abs(Kt - K) <= 2e-15 * np.abs(K).max() + 8e-16 * np.abs(K)), (shift, np.abs(Kt - K).max())


# ---------------------------------------------------------------- numbering

def small_mesh(cell, jitter=0.0, seed=0):
    g = np.random.default_rng(seed)
    if cell == "tri":
        return W.triangle_grid(3, 2, jitter, g)
    if cell == "tet":
        return W.kuhn_tets(2, 2, 1, jitter, g)
    if cell == "quad":
        return W.structured_quad(3, 2)
    return W.structured_hex(2, 2, 1)


def expected_nn(cell, k, shape):
    if cell in ("quad", "tri"):
        return (k * shape[0] + 1) * (k * shape[1] + 1)
    return (k * shape[0] + 1) * (k * shape[1] + 1) * (k * shape[2] + 1)


def relabel_vertices(coords, cells, seed):
    """Same mesh, vertex ids randomly permuted (so an edge's min-id vertex is
    not always its lower-left end)."""
    perm = np.random.default_rng(seed).permutation(len(coords))   # old -> new
    new_coords = np.empty_like(coords)
    new_coords[perm] = coords
    return new_coords, perm[cells].astype(np.int32)


@pytest.mark.parametrize("relabel", [False, True])
@pytest.mark.parametrize("cell,k", CELLS_ORDERS)
def test_numbering_conforming_and_convention(cell, k, relabel):
    """Every cell places a shared global node at the same point; distinct nodes
    sit at distinct points; the ordering follows the stated convention."""
    coords, cells = small_mesh(cell, jitter=0.1, seed=3)
    if relabel:
        coords, cells = relabel_vertices(coords, cells, 17)
    shape = {"tri": (3, 2), "tet": (2, 2, 1), "quad": (3, 2), "hex": (2, 2, 1)}[cell]
    cn, nn = oracle.number(cell, k, len(coords), cells)
    if cell != "tet" or k < 3:
        # lattice-filling element families: NN = (k n + 1)^d
        assert nn == expected_nn(cell, k, shape)
    d = W.DIM[cell]
    pos = np.full((nn, d), np.nan)
    for e, cv in enumerate(cells):
        P = local_node_positions(cell, k, coords[cv])
        for a, n in enumerate(cn[e]):
            if np.isnan(pos[n, 0]):
                pos[n] = P[a]
            else:
                assert np.abs(pos[n] - P[a]).max() < 1e-12
    assert not np.isnan(pos).any()
    key = np.round(pos, 9)
    assert len(np.unique(key, axis=0)) == nn
    np.testing.assert_allclose(pos[: len(coords)], coords, atol=1e-14)
    # edges: sorted by (min, max), nodes from the min vertex toward the max one
    nvc = W.NVERT[cell]
    edges = set()
    for cv in cells:
        for a, b in itertools.combinations(range(nvc), 2):
            if cell in ("quad", "hex") and bin(a ^ b).count("1") != 1:
                continue
            edges.add((min(cv[a], cv[b]), max(cv[a], cv[b])))
    edges = sorted(edges)
    for t, (v0, v1) in enumerate(edges):
        for s in range(k - 1):
            n = len(coords) + t * (k - 1) + s
            want = coords[v0] + (s + 1) / k * (coords[v1] - coords[v0])
            np.testing.assert_allclose(pos[n], want, atol=1e-12)
    off = len(coords) + len(edges) * (k - 1)
    if cell == "tet" and k == 3:
        faces = sorted({tuple(sorted(f)) for cv in cells for f in itertools.combinations(cv, 3)})
        for t, f in enumerate(faces):
            np.testing.assert_allclose(pos[off + t], coords[list(f)].mean(0), atol=1e-12)
        off += len(faces)
    if cell == "hex" and k >= 2:
        faces = set()
        for cv in cells:
            for m in range(3):
                for side in (0, 1):
                    f = [cv[v] for v in range(8) if ((v >> m) & 1) == side]
                    faces.add(tuple(sorted(f)))
        faces = sorted(faces)
        nf = (k - 1) ** 2
        for t, f in enumerate(faces):
            if k == 2:
                np.testing.assert_allclose(pos[off + t], coords[list(f)].mean(0), atol=1e-12)
        off += len(faces) * nf
    ni = {"tri": (k - 1) * (k - 2) // 2, "tet": (k - 1) * (k - 2) * (k - 3) // 6,
          "quad": (k - 1) ** 2, "hex": (k - 1) ** 3}[cell]
    assert nn == off + len(cells) * ni
    if cell == "tri" and k == 3:
        for e, cv in enumerate(cells):
            np.testing.assert_allclose(pos[off + e], coords[cv].mean(0), atol=1e-12)


@pytest.mark.parametrize("relabel", [False, True])
def test_hex_q3_face_frame(relabel):
    """Q3 hex faces: 4 nodes in the frame of the face's smallest vertex o,
    first axis toward the smaller of o's two face neighbours."""
    coords, cells = W.structured_hex(1, 1, 2)
    if relabel:
        coords, cells = relabel_vertices(coords, cells, 5)
    cn, nn = oracle.number("hex", 3, len(coords), cells)
    pos = np.full((nn, 3), np.nan)
    for e, cv in enumerate(cells):
        for a, n in enumerate(cn[e]):
            pos[n] = local_node_positions("hex", 3, coords[cv])[a]
    edges = set()
    for cv in cells:
        for a, b in itertools.combinations(range(8), 2):
            if bin(a ^ b).count("1") == 1:
                edges.add((min(cv[a], cv[b]), max(cv[a], cv[b])))
    off = len(coords) + 2 * len(edges)
    faces = set()
    for cv in cells:
        for m in range(3):
            for side in (0, 1):
                faces.add(tuple(sorted(cv[v] for v in range(8) if ((v >> m) & 1) == side)))
    for t, f in enumerate(sorted(faces)):
        o = f[0]
        nbrs = [v for v in f[1:] if np.isclose(np.abs(coords[v] - coords[o]).sum(), 1.0)]
        p, q = sorted(nbrs)
        for tt in range(2):
            for s in range(2):
                want = coords[o] + (s + 1) / 3 * (coords[p] - coords[o]) + (tt + 1) / 3 * (coords[q] - coords[o])
                np.testing.assert_allclose(pos[off + 4 * t + s + 2 * tt], want, atol=1e-12)


def test_paper_printed_counts():
    """Sec. 5.5 and Sec. 5.7 print dof and density counts for two hex meshes."""
    with open(os.path.join(GOLDEN, "paper_counts.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        coords, cells = W.structured_hex(*case["shape"])
        cn, nn = oracle.number("hex", case["order"], len(coords), cells)
        assert 3 * nn == case["ndof"], case["cite"]
        assert len(cells) == case["n_cells"], case["cite"]


def test_workload_counts():
    """P2 on the Kuhn split fills the half lattice; P3 triangles fill the
    third lattice (closed forms of the conforming Lagrange spaces)."""
    coords, cells = W.kuhn_tets(6, 2, 2)
    cn, nn = oracle.number("tet", 2, len(coords), cells)
    assert nn == 13 * 5 * 5 and len(cells) == 6 * 24
    coords, cells = W.triangle_grid(8, 4)
    cn, nn = oracle.number("tri", 3, len(coords), cells)
    assert nn == 25 * 13 and len(cells) == 64


# ---------------------------------------------------------------- assembly

def dense_brute_force(cell, k, coords, cells, mat, rho):
    """Explicit loops: dense K(rho) = sum_e E(rho_e) K_e^0 scattered by dof."""
    E0, Emin, nu, p, ps = mat
    cn, nn = oracle.number(cell, k, len(coords), cells)
    d = W.DIM[cell]
    K = np.zeros((d * nn, d * nn))
    struct = np.zeros((d * nn, d * nn), bool)
    for e, cv in enumerate(cells):
        Ke = oracle.element_matrix(cell, k, coords[cv], nu, ps)
        Ee = Emin + rho[e] ** p * (E0 - Emin)
        nb = len(cn[e])
        for a in range(nb):
            for i in range(d):
                for b in range(nb):
                    for j in range(d):
                        r, c = d * cn[e, a] + i, d * cn[e, b] + j
                        K[r, c] += Ee * Ke[d * a + i, d * b + j]
                        struct[r, c] = True
    return K, struct


@pytest.mark.parametrize("cell,k", [("tri", 1), ("tri", 3), ("tet", 2), ("quad", 1), ("quad", 2), ("hex", 1), ("tet", 3)])
@pytest.mark.parametrize("nel", [1, 2, 4])
def test_csr_matches_dense_brute_force(cell, k, nel):
    coords, cells = small_mesh(cell, jitter=0.1, seed=nel)
    cells = cells[:nel]
    used = np.unique(cells)
    remap = -np.ones(len(coords), np.int64)
    remap[used] = np.arange(len(used))
    coords, cells = coords[used], remap[cells].astype(np.int32)
    rho = np.random.default_rng(nel).uniform(0.001, 1, len(cells))
    mat = (1.0, 1e-9, 0.3, 3.0, 0)
    Kd, struct = dense_brute_force(cell, k, coords, cells, mat, rho)
    rp, ci, v, ndof = oracle.assemble(cell, k, coords, cells, mat, rho)
    assert ndof == len(Kd)
    Kc = np.zeros_like(Kd)
    sc = np.zeros_like(struct)
    for r in range(ndof):
        cols = ci[rp[r]:rp[r + 1]]
        assert np.all(np.diff(cols) > 0)            # sorted, unique
        Kc[r, cols] = v[rp[r]:rp[r + 1]]
        sc[r, cols] = True
    assert np.array_equal(sc, struct)               # every structural pair, zeros included
    np.testing.assert_allclose(Kc, Kd, rtol=0, atol=1e-15 * np.abs(Kd).max())


def test_row_selection_matches_full():
    wl = W.jittered_tri(5, 3, order=3)
    rp, ci, v, ndof = oracle.assemble(wl.cell, 3, wl.coords, wl.cells, wl.mat, wl.rho)
    rows = np.array([ndof - 1, 0, 17, 5, 17 + 1])
    rp2, ci2, v2, _ = oracle.assemble(wl.cell, 3, wl.coords, wl.cells, wl.mat, wl.rho, rows=rows)
    for s, r in enumerate(rows):
        assert np.array_equal(ci2[rp2[s]:rp2[s + 1]], ci[rp[r]:rp[r + 1]])
        assert np.array_equal(v2[rp2[s]:rp2[s + 1]], v[rp[r]:rp[r + 1]])


# ---------------------------------------------------------------- patch test / exact energy

PATCH = [("tri", 1, 0.2), ("tri", 2, 0.2), ("tri", 3, 0.2), ("tet", 1, 0.15), ("tet", 2, 0.15),
         ("tet", 3, 0.15), ("quad", 1, 0.0), ("quad", 2, 0.0), ("quad", 3, 0.0), ("hex", 1, 0.0),
         ("hex", 2, 0.0)]
# general (non-affine) bilinear / trilinear cells: the (k+1)-point Gauss rule
# integrates the nodal forces of a constant stress exactly (the integrand
# adj(J)^T grad phi is a polynomial of degree <= k + 1 per direction), so
# the patch test holds on distorted meshes too
PATCH_DISTORTED = [("quad", 1, 0.2), ("quad", 2, 0.2), ("quad", 3, 0.2), ("hex", 1, 0.15), ("hex", 2, 0.15)]


def patch_mesh(cell, jitter):
    g = np.random.default_rng(21)
    if cell == "tri":
        return W.triangle_grid(4, 3, jitter, g), (4, 3)
    if cell == "tet":
        return W.kuhn_tets(3, 2, 2, jitter, g), (3, 2, 2)
    if cell == "quad":
        return W.quad_grid(4, 3, jitter, g), (4, 3)
    return W.hex_grid(3, 3, 3, jitter, g), (3, 3, 3)


@pytest.mark.parametrize("cell,k,jit", PATCH + PATCH_DISTORTED)
def test_patch_test_affine_field(cell, k, jit):
    """rho = 1, u = interpolant of an affine field: (K u)_i = 0 at every dof
    whose node is not on the boundary (constant stress, no body force)."""
    (coords, cells), shape = patch_mesh(cell, jit)
    d = W.DIM[cell]
    xn = oracle.node_coords(cell, k, coords, cells)
    A = np.random.default_rng(1).standard_normal((d, d))
    b = np.random.default_rng(2).standard_normal(d)
    u = (xn @ A.T + b).ravel()
    rho = np.ones(len(cells))
    rp, ci, v, ndof = oracle.assemble(cell, k, coords, cells, (1.0, 0.0, 0.3, 3.0, 0), rho)
    Ku = np.array([np.dot(v[rp[r]:rp[r + 1]], u[ci[rp[r]:rp[r + 1]]]) for r in range(ndof)])
    inner = np.all((xn > 1e-9) & (xn < np.array(shape) - 1e-9), axis=1)
    assert inner.sum() > 0
    assert np.abs(Ku.reshape(-1, d)[inner]).max() < 1e-11 * np.abs(v).max() * np.abs(u).max()


def exact_energy_2d(ux, uy, nx, ny, nu):
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    ex, ey = sp.diff(ux(x, y), x), sp.diff(uy(x, y), y)
    g = sp.diff(ux(x, y), y) + sp.diff(uy(x, y), x)
    D = sp.Matrix([[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu) / 2]]) / (1 - nu ** 2)
    eps = sp.Matrix([ex, ey, g])
    dens = (eps.T * D * eps)[0, 0]
    return float(sp.integrate(sp.integrate(sp.expand(dens), (x, 0, nx)), (y, 0, ny)))


def exact_energy_3d(uf, shape, nu):
    sp = pytest.importorskip("sympy")
    X = sp.symbols("x y z")
    u = uf(*X)
    grad = [[sp.diff(u[i], X[j]) for j in range(3)] for i in range(3)]
    eps = sp.Matrix([grad[0][0], grad[1][1], grad[2][2], grad[1][2] + grad[2][1],
                     grad[0][2] + grad[2][0], grad[0][1] + grad[1][0]])
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1 / (2 * (1 + nu))
    D = sp.zeros(6, 6)
    for i in range(3):
        for j in range(3):
            D[i, j] = lam + (2 * mu if i == j else 0)
        D[i + 3, i + 3] = mu
    dens = sp.expand((eps.T * D * eps)[0, 0])
    r = dens
    for m in range(3):
        r = sp.integrate(r, (X[m], 0, shape[m]))
    return float(r)


@pytest.mark.parametrize("cell,k,jit", [c for c in PATCH if c[1] >= 2])
def test_polynomial_field_energy_is_exact(cell, k, jit):
    """u = interpolant of a degree-k polynomial field (reproduced exactly by
    the element space on affine cells): u^T K(1) u = int sigma(u):eps(u)."""
    sp = pytest.importorskip("sympy")
    (coords, cells), shape = patch_mesh(cell, jit)
    nu = sp.Rational(3, 10)
    xn = oracle.node_coords(cell, k, coords, cells)
    if W.DIM[cell] == 2:
        if k == 2:
            ux = lambda x, y: x * x / 5 - x * y / 7 + y / 3
            uy = lambda x, y: x * y / 4 + y * y / 9 - x / 2
        else:
            ux = lambda x, y: x ** 3 / 30 - x * y * y / 17 + x * y / 5
            uy = lambda x, y: y ** 3 / 25 + x * x * y / 13 - y / 2
        want = exact_energy_2d(ux, uy, shape[0], shape[1], nu)
        u = np.stack([[float(ux(a, b)) for a, b in xn], [float(uy(a, b)) for a, b in xn]], 1).ravel()
    else:
        if k == 2:
            uf = lambda x, y, z: (x * y / 5 + z * z / 7, y * z / 3 - x * x / 11, x * z / 4 + y / 2)
        else:
            uf = lambda x, y, z: (x * y * z / 9 + x ** 3 / 40, y ** 3 / 30 - x * z / 7, z ** 3 / 35 + x * x * y / 20)
        want = exact_energy_3d(uf, shape, nu)
        u = np.array([[float(c) for c in uf(*pt)] for pt in xn]).ravel()
    rho = np.ones(len(cells))
    rp, ci, v, ndof = oracle.assemble(cell, k, coords, cells, (1.0, 0.0, 0.3, 3.0, 0), rho)
    Ku = np.array([np.dot(v[rp[r]:rp[r + 1]], u[ci[rp[r]:rp[r + 1]]]) for r in range(ndof)])
    assert abs(u @ Ku - want) < 1e-11 * abs(want)
    dc, s, c = oracle.sensitivity(cell, k, coords, cells, (1.0, 0.0, 0.3, 3.0, 0), rho, u)
    assert abs(c - want) < 1e-11 * abs(want)


# ---------------------------------------------------------------- sensitivity

@pytest.mark.parametrize("cell,k", [("quad", 1), ("tri", 3), ("tet", 2), ("hex", 1)])
def test_sensitivity_consistency_and_euler_identity(cell, k):
    """c = u^T (K u) through the CSR; with Emin = 0, E(rho) = rho^p E0 is
    homogeneous of degree p, so sum_e rho_e dc_e = -p c."""
    coords, cells = small_mesh(cell, jitter=0.1, seed=9)
    g = np.random.default_rng(4)
    rho = g.uniform(0.001, 1, len(cells))
    for mat in ((1.0, 1e-9, 0.3, 3.0, 0), (1.0, 0.0, 0.3, 3.0, 0), (2.0, 0.0, 0.25, 2.5, 1)):
        rp, ci, v, ndof = oracle.assemble(cell, k, coords, cells, mat, rho)
        u = g.standard_normal(ndof)
        Ku = np.array([np.dot(v[rp[r]:rp[r + 1]], u[ci[rp[r]:rp[r + 1]]]) for r in range(ndof)])
        dc, s, c = oracle.sensitivity(cell, k, coords, cells, mat, rho, u)
        assert abs(c - u @ Ku) < 1e-12 * np.abs(u).max() ** 2 * np.abs(v).sum()
        E0, Emin, nu, p, ps = mat
        dE = p * rho ** (p - 1) * (E0 - Emin)
        np.testing.assert_allclose(dc, -dE * s, rtol=1e-15)
        if Emin == 0.0:
            assert abs(np.dot(rho, dc) + p * c) < 1e-12 * np.abs(rho * dc).sum()
        # subset selection returns the same numbers
        sel = np.array([len(cells) - 1, 0, 2])
        dcs, ss, cs = oracle.sensitivity(cell, k, coords, cells, mat, rho, u, sel=sel)
        np.testing.assert_array_equal(dcs, dc[sel])
        assert math.isnan(cs)


def _cell_volumes(cell, coords, cells):
    """|e| from the vertices alone: simplices by the determinant of their edge
    vectors, parallelograms / parallelepipeds (corners lexicographic, x
    fastest) by that of the edges from corner 0."""
    x = coords[cells]
    if cell == "tri":
        return np.abs(np.linalg.det(np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]], 1))) / 2
    if cell == "tet":
        return np.abs(np.linalg.det(np.stack([x[:, m] - x[:, 0] for m in (1, 2, 3)], 1))) / 6
    if cell == "quad":
        # the polygon 0, 1, 3, 2 (shoelace): a bilinear cell has straight edges
        p = x[:, [0, 1, 3, 2]]
        q = np.roll(p, -1, axis=1)
        return np.abs(np.sum(p[..., 0] * q[..., 1] - q[..., 0] * p[..., 1], axis=1)) / 2
    return np.abs(np.linalg.det(np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 4] - x[:, 0]], 1)))


@pytest.mark.parametrize("cell,k,general", [
    ("tri", 1, False), ("tri", 2, False), ("tri", 3, False), ("tet", 1, False), ("tet", 2, False),
    ("tet", 3, False), ("quad", 1, False), ("quad", 2, False), ("quad", 3, False), ("hex", 1, False),
    ("hex", 2, False), ("hex", 3, False), ("quad", 1, True), ("quad", 2, True), ("quad", 3, True)])
def test_sensitivity_of_an_affine_field_cell_by_cell(cell, k, general):
    """u = A x + b is reproduced by every element space (on general
    quadrilaterals too: x and y are in the span of the bilinear map), so its
    strain eps = (A + A^T) / 2 is constant and each cell's s_e = u_e^T K_e^0 u_e
    equals |e| (lam (tr eps)^2 + 2 mu eps:eps) at unit modulus -- cell by cell,
    with |e| from the vertices and lam, mu from the plane-stress /
    plane-strain / 3D formulas."""
    g = np.random.default_rng(17)
    d = W.DIM[cell]
    if cell in ("tri", "tet"):
        coords, cells = small_mesh(cell, jitter=0.15, seed=3)
    elif general:
        coords, cells = W.quad_grid(4, 3, 0.2, g)
    else:
        coords, cells = small_mesh(cell)
        B = np.eye(d) + 0.3 * g.uniform(-1, 1, (d, d))   # parallelograms / parallelepipeds
        coords = coords @ B.T
    xn = oracle.node_coords(cell, k, coords, cells)
    A, b = g.standard_normal((d, d)), g.standard_normal(d)
    u = (xn @ A.T + b).ravel()
    eps = (A + A.T) / 2
    rho = g.uniform(0.1, 1.0, len(cells))
    vol = _cell_volumes(cell, coords, cells)
    assert np.all(vol > 0)
    for nu, ps in ((0.3, 0), (0.25, 1)):
        if d == 3 or ps:
            lam = nu / ((1 + nu) * (1 - 2 * nu))
        else:
            lam = nu / (1 - nu * nu)
        mu = 1 / (2 * (1 + nu))
        want = vol * (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps))
        dc, s, c = oracle.sensitivity(cell, k, coords, cells, (1.0, 1e-9, nu, 3.0, ps), rho, u)
        np.testing.assert_allclose(s, want, rtol=1e-11, atol=1e-12 * want.max())
        E = 1e-9 + rho ** 3 * (1.0 - 1e-9)
        assert abs(c - np.dot(E, want)) < 1e-11 * np.dot(E, want)


def test_compliance_vjp_central_differences():
    """f(rho) = u^T K(rho) u is cubic in each rho_e (p = 3), so the central
    difference error is exactly (E0 - Emin) s_e h^2 plus rounding."""
    wl = W.jittered_tet(2, 2, 1, order=2)
    rp, ci, v, ndof = oracle.assemble(wl.cell, 2, wl.coords, wl.cells, wl.mat, wl.rho)
    u = wl.displacement(ndof)
    g = 1.7
    gr, gu = oracle.compliance_vjp(wl.cell, 2, wl.coords, wl.cells, wl.mat, wl.rho, u, g)

    def f(rho):
        _, _, c = oracle.sensitivity(wl.cell, 2, wl.coords, wl.cells, wl.mat, rho, u)
        return c

    h = 1e-6
    f0 = f(wl.rho)
    _, s, _ = oracle.sensitivity(wl.cell, 2, wl.coords, wl.cells, wl.mat, wl.rho, u)
    for e in range(0, len(wl.cells), 5):
        rp_, rm_ = wl.rho.copy(), wl.rho.copy()
        rp_[e] += h
        rm_[e] -= h
        fd = g * (f(rp_) - f(rm_)) / (2 * h)
        tol = g * ((wl.E0 - wl.Emin) * s[e] * h * h + 8 * np.finfo(float).eps * abs(f0) / h) + 1e-8 * abs(gr[e])
        assert abs(fd - gr[e]) <= tol
    Ku = np.array([np.dot(v[rp[r]:rp[r + 1]], u[ci[rp[r]:rp[r + 1]]]) for r in range(ndof)])
    np.testing.assert_allclose(gu, 2 * g * Ku, rtol=1e-13, atol=1e-13 * np.abs(gu).max())


# ---------------------------------------------------------------- the step after assembly (NEXT row f1)

@pytest.mark.parametrize("cell,k,jit", [("quad", 2, 0.2), ("hex", 1, 0.15), ("tet", 2, 0.15), ("tri", 3, 0.2)])
def test_dirichlet_solve_reproduces_affine_field(cell, k, jit):
    """Patch test of the constrained solve: a homogeneous body (one density
    for every cell), u = an affine field on every boundary dof, no load; the
    discrete solution is that field at every dof (it lies in the element space
    and its constant stress is in equilibrium)."""
    (coords, cells), shape = patch_mesh(cell, jit)
    d = W.DIM[cell]
    xn = oracle.node_coords(cell, k, coords, cells)
    A = np.random.default_rng(3).standard_normal((d, d))
    b = np.random.default_rng(4).standard_normal(d)
    ulin = (xn @ A.T + b).ravel()
    rho = np.full(len(cells), 0.6)
    rp, ci, v, ndof = oracle.assemble(cell, k, coords, cells, (1.0, 1e-9, 0.3, 3.0, 0), rho)
    bnd = ~np.all((xn > 1e-9) & (xn < np.array(shape) - 1e-9), axis=1)
    fixed = np.repeat(bnd, d)
    u = oracle.solve_dirichlet(rp, ci, v, fixed, np.zeros(ndof), ulin)
    assert (~fixed).sum() > 0
    assert np.abs(u - ulin).max() < 1e-10 * np.abs(ulin).max()


def test_spmv_matches_dense_product():
    """The oracle's CSR product against a dense matrix-vector product."""
    coords, cells = W.kuhn_tets(2, 2, 1, 0.1, np.random.default_rng(0))
    rp, ci, v, ndof = oracle.assemble("tet", 2, coords, cells, (1.0, 1e-9, 0.3, 3.0, 0), np.full(len(cells), 0.7))
    K = np.zeros((ndof, ndof))
    for r in range(ndof):
        K[r, ci[rp[r]:rp[r + 1]]] = v[rp[r]:rp[r + 1]]
    x = np.random.default_rng(1).standard_normal(ndof)
    np.testing.assert_allclose(oracle.spmv(rp, ci, v, x), K @ x, rtol=0, atol=1e-13 * np.abs(K).sum(1).max())


# ---------------------------------------------------------------- filters and the OC update (NEXT rows f2, f3)

def _centroids(cell, coords, cells):
    return np.asarray(coords)[np.asarray(cells)].mean(axis=1)


def test_filter_weights_symmetric_with_rmin_diagonal():
    coords, cells = W.kuhn_tets(4, 3, 2, 0.15, np.random.default_rng(2))
    H = oracle.filter_weights(_centroids("tet", coords, cells), 1.3).toarray()
    np.testing.assert_allclose(H, H.T, rtol=0, atol=0)
    np.testing.assert_allclose(np.diag(H), 1.3)
    assert np.all(H >= 0.0)


def test_density_filter_keeps_constants_and_its_chain_rule_is_the_adjoint():
    """rho~ of a constant field is that constant; <g, F x> = <F^T g, x>."""
    coords, cells = W.triangle_grid(9, 6, 0.2, np.random.default_rng(3))
    cen = _centroids("tri", coords, cells)
    vol = np.random.default_rng(4).uniform(0.3, 0.6, len(cells))
    H = oracle.filter_weights(cen, 2.2)
    np.testing.assert_allclose(oracle.density_filter(H, vol, np.full(len(cells), 0.37)), 0.37, rtol=1e-15)
    g, x = np.random.default_rng(5).standard_normal((2, len(cells)))
    lhs = g @ oracle.density_filter(H, vol, x)
    rhs = oracle.density_filter_grad(H, vol, g) @ x
    assert abs(lhs - rhs) <= 1e-13 * (np.abs(g).sum() * np.abs(x).max())


def test_sensitivity_filter_constant_field():
    """With rho = 1 and dc constant the weighted average returns dc."""
    coords, cells = W.structured_quad(8, 5)
    H = oracle.filter_weights(_centroids("quad", coords, cells), 1.8)
    out = oracle.sensitivity_filter(H, np.ones(len(cells)), np.full(len(cells), -2.5))
    np.testing.assert_allclose(out, -2.5, rtol=1e-15)


def test_heaviside_derivative_and_small_beta_limit():
    x = np.linspace(0.0, 1.0, 11)
    for beta in (1.0, 8.0):
        y, dy = oracle.heaviside(x, beta)
        h = 1e-6
        fd = (oracle.heaviside(x + h, beta)[0] - oracle.heaviside(x - h, beta)[0]) / (2 * h)
        np.testing.assert_allclose(dy, fd, rtol=1e-7, atol=1e-9)
        assert abs(y[0]) < 1e-15 and abs(y[-1] - 1.0) < 1e-15
    np.testing.assert_allclose(oracle.heaviside(x, 1e-9)[0], x, atol=1e-9)


def test_oc_update_meets_volume_and_move_limits():
    g = np.random.default_rng(6)
    n = 500
    rho = g.uniform(0.05, 1.0, n)
    dc = -g.uniform(0.1, 5.0, n)
    vol = g.uniform(0.5, 1.5, n)
    new, lam = oracle.oc_update(rho, dc, vol, vol, 0.4, move=0.2, eta=0.5)
    assert np.all(new >= np.maximum(0, rho - 0.2) - 1e-15) and np.all(new <= np.minimum(1, rho + 0.2) + 1e-15)
    # the volume sits at the target to the bisection's tolerance
    tight, _ = oracle.oc_update(rho, dc, vol, vol, 0.4, tol=1e-12)
    assert abs(np.dot(vol, tight) / vol.sum() - 0.4) < 1e-9
    assert abs(np.dot(vol, new) / vol.sum() - 0.4) < 5e-3
    # cells strictly inside their bounds follow rho B^eta at the returned multiplier
    inside = (new > np.maximum(0, rho - 0.2) + 1e-12) & (new < np.minimum(1, rho + 0.2) - 1e-12)
    np.testing.assert_allclose(new[inside], rho[inside] * np.sqrt(-dc[inside] / (lam * vol[inside])), rtol=1e-13)


def test_oc_loop_reproduces_the_papers_3d_cantilever():
    """Algorithm 1 with the sensitivity filter on the paper's 3D cantilever
    (Sec. 5.4: 60x20x4 hexahedra, volume fraction 0.3, r = 1.5): the paper
    prints c = 2063.5625 after 54 iterations (Sec. 5.4-5.6); the stored
    trajectory (tests/golden/make_cantilever3d_oc.py) is this loop's."""
    with open(os.path.join(GOLDEN, "paper_cantilever3d.json")) as fh:
        paper = json.load(fh)["60x20x4"]
    with open(os.path.join(GOLDEN, "cantilever3d_60x20x4_oc.json")) as fh:
        stored = json.load(fh)
    wl, fixed, f = W.cantilever_3d_oc(60, 20, 4)
    assert 3 * len(wl.coords) == paper["dofs"] and len(wl.cells) == paper["cells"]
    x, hist = oracle.oc_loop("hex", 1, wl.coords, wl.cells, (1.0, 1e-9, 0.3, 3.0, 0), fixed, f, paper["rmin"],
                             paper["volfrac"], np.ones(len(wl.cells)), _centroids("hex", wl.coords, wl.cells))
    assert len(hist) == paper["iterations"]
    assert abs(hist[-1][0] - paper["c"]) <= 5e-5
    np.testing.assert_allclose([h[0] for h in hist], stored["c"], rtol=1e-10)
