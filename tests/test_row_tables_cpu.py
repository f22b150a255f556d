"""The 3D node-owner schedule (soptx_host_row_tables), checked without a GPU
against the mesh's own CSR pattern and cell map (soptx_host_plan): every node's
rows are met once per incident cell, each lane's record names the right column
block, and the chain follows its rules (the next cell shares the most nodes with
the lanes, a lane keeps its node, first and last meetings flagged)."""
import numpy as np
import pytest

from paper_2505_02438_gb300 import build, workloads as W


@pytest.fixture(scope="module", autouse=True)
def native():
    build.build_library()


def check_rows(cell, k, coords, cells):
    from paper_2505_02438_gb300.api import host_plan, host_row_tables
    pl = host_plan(cell, k, coords, cells)
    T = host_row_tables(cell, k, coords, cells)
    assert T is not None
    d, nb, cn = 3, pl["nb"], pl["cell_nodes"]
    indptr, indices = pl["indptr"], pl["indices"]
    nn = pl["ndof"] // d
    inc = [[] for _ in range(nn)]
    for e, row in enumerate(cn):
        for n in row:
            inc[n].append(e)
    cnt = np.array([len(x) for x in inc])
    assert np.all(cnt > 0)
    inc_ptr = np.concatenate([[0], np.cumsum(cnt)])
    node_of = {int(inc_ptr[n]): n for n in range(nn)}
    deg = (indptr[1::d][:nn] - indptr[0::d][:nn]) // d
    # processing order: every node once, cell count descending, ids ascending
    R = T["node_records"].astype(np.int64)
    order = [node_of[int(q0)] for q0 in R[:, 2]]
    assert sorted(order) == list(range(nn))
    assert order == sorted(range(nn), key=lambda n: (-cnt[n], n))
    for r, n in zip(R, order):
        assert (r[0] & 0xFFFFFFFF) | (r[1] << 32) == indptr[d * n] // (d * d)
        assert r[3] >> 16 == cnt[n] and r[3] & 0xFFFF == deg[n]
    ce, ca, rec = T["chain_cell"], T["chain_local"], T["lane_records"].astype(np.int64)
    assert len(ce) == inc_ptr[-1] and rec.shape == (len(ce), nb)
    for n in range(nn):
        q = np.arange(inc_ptr[n], inc_ptr[n + 1])
        chain = [int(e) for e in ce[q]]
        assert sorted(chain) == inc[n] and chain[0] == inc[n][0]
        assert all(cn[e][ca[i]] == n for e, i in zip(chain, q))
        row0 = indptr[d * n]
        p, b = rec[q] & 511, (rec[q] >> 9) & 31
        first, last = (rec[q] >> 14) & 1, (rec[q] >> 15) & 1
        met = set()
        for k, e in enumerate(chain):
            # the lanes hold the cell's nodes, each once, and p is the column
            # block of the lane's node in n's rows
            assert sorted(b[k]) == list(range(nb))
            for L in range(nb):
                assert indices[row0 + d * p[k, L]] == d * cn[e][b[k, L]]
            if k > 0:
                prev = set(cn[chain[k - 1]])
                # the most nodes shared with the lanes' (the previous cell's),
                # the lowest cell id on ties
                share = lambda c: len(prev & set(cn[c]))
                rest = [c for c in inc[n] if c not in chain[:k]]
                best = max(share(c) for c in rest)
                assert share(e) == best and e == min(c for c in rest if share(c) == best)
                kept = [L for L in range(nb) if cn[chain[k - 1]][b[k - 1, L]] in set(cn[e])]
                for L in kept:
                    assert cn[e][b[k, L]] == cn[chain[k - 1]][b[k - 1, L]]
                free = [L for L in range(nb) if L not in kept]
                assert list(b[k, free]) == sorted(set(range(nb)) - set(b[k, kept]))
            for L in range(nb):
                assert first[k, L] == (p[k, L] not in met)
                met.add(int(p[k, L]))
        # every column block of the node's rows is met; the last meetings mirror the first
        assert met == set(range(deg[n]))
        seen = set()
        for k in range(len(chain) - 1, -1, -1):
            for L in range(nb - 1, -1, -1):
                assert last[k, L] == (p[k, L] not in seen)
                seen.add(int(p[k, L]))
    return T


def mk(cell):
    g = np.random.default_rng(6)
    return {"tet": lambda: W.kuhn_tets(3, 2, 2, 0.1, g), "hex": lambda: W.hex_grid(3, 2, 2, 0.1, g)}[cell]()


@pytest.mark.parametrize("cell,k", [("tet", 1), ("tet", 2), ("tet", 3), ("hex", 1), ("hex", 2)])
def test_chains_follow_their_rules(cell, k):
    check_rows(cell, k, *mk(cell))


def test_relabelled_vertices():
    from helpers import relabel
    check_rows("tet", 2, *relabel(*W.kuhn_tets(2, 2, 2, 0.1, np.random.default_rng(1)), 3))


def test_no_schedule_outside_its_limits():
    """2D meshes and hexahedra of order 3 (64 nodes per cell) get none."""
    from paper_2505_02438_gb300.api import host_row_tables
    assert host_row_tables("tri", 2, *W.triangle_grid(3, 3, 0.1, np.random.default_rng(0))) is None
    assert host_row_tables("hex", 3, *W.structured_hex(2, 2, 1)) is None
