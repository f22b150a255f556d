"""The pair kernel's schedule, built on the host (soptx_host_pair_tables), checked
without a GPU against the mesh's own CSR pattern and cell map (soptx_host_plan,
itself pinned to the oracle's numbering): every (pair, cell) contribution of
K(rho) = sum_e E(rho_e) K_e^0 (Sec. 2.2) is scheduled exactly once, with the
right local nodes and the right value offsets of both destination blocks."""
import numpy as np
import pytest

from paper_2505_02438_gb300 import build, workloads as W


@pytest.fixture(scope="module", autouse=True)
def native():
    build.build_library()


def fan(n, g):
    t = 2 * np.pi * np.arange(n) / n
    r = 1.0 + 0.1 * g.uniform(-1, 1, n)
    coords = np.vstack([[0.0, 0.0], np.stack([r * np.cos(t), r * np.sin(t)], axis=1)])
    cells = np.array([[0, 1 + k, 1 + (k + 1) % n] for k in range(n)], np.int32)
    return coords, cells


def check_tables(cell, k, coords, cells, byte_pairs):
    from paper_2505_02438_gb300.api import host_pair_tables, host_plan
    pl = host_plan(cell, k, coords, cells)
    T = host_pair_tables(cell, k, coords, cells, byte_pairs)
    assert T is not None
    d, nb = coords.shape[1], pl["nb"]
    indptr, indices, cn = pl["indptr"], pl["indices"], pl["cell_nodes"]
    nt, toff = T["n_tiles"], T["tile_offsets"].astype(np.int64)
    assert toff[0] == 0 and np.all(np.diff(toff) >= 1) and len(T["record_cell"]) == 32 * toff[-1]
    meta = T["pair_meta"].astype(np.int64)
    cnt, rla, rlb = meta & 1023, (meta >> 10) & 2047, meta >> 21
    # the cells of every node pair that shares one, from the cell map
    shared = {}
    for e, row in enumerate(cn):
        for al in range(nb):
            for bl in range(nb):
                shared.setdefault((int(row[al]), int(row[bl])), []).append(e)
    first = np.full(pl["ndof"] // d, len(cells))
    for e in range(len(cells) - 1, -1, -1):
        first[cn[e]] = e
    seen = set()
    for t in range(nt):
        ct = toff[t + 1] - toff[t]
        c = cnt[32 * t: 32 * t + 32]
        # the lanes' counts fall within a tile, the first is the tile's depth, and
        # empty lanes come last and carry nothing
        assert c[0] == ct and np.all(np.diff(c) <= 0)
        for lane in range(32):
            p = 32 * t + lane
            rec = 32 * (toff[t] + np.arange(ct)) + lane
            re, rp = T["record_cell"][rec].astype(np.int64), T["record_pair"][rec].astype(np.int64)
            n = cnt[p]
            assert np.all(re[n:] == 0) and np.all(rp[n:] == 0)
            if n == 0:
                assert meta[p] == 0 and T["pair_block"][p] == 0 and T["pair_block_t"][p] == 0
                continue
            al, bl = (rp[:n] >> 8, rp[:n] & 255) if byte_pairs else (rp[:n] // nb, rp[:n] % nb)
            a, b = cn[re[:n], al], cn[re[:n], bl]
            assert np.all(a == a[0]) and np.all(b == b[0])
            a, b = int(a[0]), int(b[0])
            # the pair's cells: all that hold both nodes, ascending
            assert list(re[:n]) == shared[(a, b)]
            key = (min(a, b), max(a, b)) if d == 2 else (a, b)
            assert key not in seen
            seen.add(key)
            # block (a, b): rows d a .. d a + d - 1 of rla values each, columns d b ..
            v = d * int(T["pair_block"][p])
            assert rla[p] == indptr[d * a + 1] - indptr[d * a] and indptr[d * a] <= v < indptr[d * a + 1]
            for i in range(d):
                assert indptr[d * a + i] == indptr[d * a] + i * rla[p]
                assert list(indices[v + i * rla[p]: v + i * rla[p] + d]) == [d * b + j for j in range(d)]
            vt = d * int(T["pair_block_t"][p])
            if d == 2:
                # the transposed destination, block (b, a); the owner a comes
                # first in the sweep (by first cell, then id)
                assert (first[a], a) <= (first[b], b)
                assert rlb[p] == indptr[d * b + 1] - indptr[d * b]
                for i in range(d):
                    assert list(indices[vt + i * rlb[p]: vt + i * rlb[p] + d]) == [d * a + j for j in range(d)]
            else:
                assert vt == v and rlb[p] == rla[p]
    # coverage: every pair that shares a cell, once
    want = {(min(a, b), max(a, b)) for (a, b) in shared} if d == 2 else set(shared)
    assert seen == want
    return T


def mk(name):
    g = np.random.default_rng(4)
    return {"tri": lambda: W.triangle_grid(7, 5, 0.2, g), "quad": lambda: W.structured_quad(5, 4),
            "hex": lambda: W.structured_hex(3, 2, 2), "tet": lambda: W.kuhn_tets(2, 2, 1, 0.1, g)}[name]()


@pytest.mark.parametrize("byte_pairs", [False, True])
@pytest.mark.parametrize("cell,k", [("tri", 1), ("tri", 2), ("tri", 3), ("quad", 2), ("quad", 3)])
def test_2d_pairs_cover_every_contribution_once(cell, k, byte_pairs):
    check_tables(cell, k, *mk(cell), byte_pairs)


@pytest.mark.parametrize("cell,k", [("hex", 2), ("hex", 3), ("tet", 2)])
def test_3d_nodes_take_their_own_blocks(cell, k):
    check_tables(cell, k, *mk(cell), True)


def test_fan_and_windows():
    """A 150-cell fan (one pair with 150 records) and a P3 mesh of more than one
    window of pairs (windows are sorted by count independently)."""
    g = np.random.default_rng(2)
    T = check_tables("tri", 3, *fan(150, g), False)
    assert T["pair_meta"].max() & 1023 == 150
    coords, cells = W.triangle_grid(16, 12, 0.2, g)
    T = check_tables("tri", 3, coords, cells, True)
    assert T["n_tiles"] * 32 > 2 * 4096


def test_past_the_limits():
    """A fan whose centre has more than 1023 neighbours' values in a row keeps
    the row gather: no tables."""
    from paper_2505_02438_gb300.api import host_pair_tables
    assert host_pair_tables("tri", 1, *fan(1100, np.random.default_rng(0))) is None
    assert host_pair_tables("tri", 1, *fan(1000, np.random.default_rng(0))) is not None
