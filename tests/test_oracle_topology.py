"""Pins of the oracle's adjacency, colouring and k-rings against brute force
and independent constructions."""
import numpy as np
import pytest
import scipy.sparse as sp

import meshgen
from oracle import topology


def _box(n=4, jit=0.0):
    return meshgen.stretch_box(n, n + 1, n - 1, jitter_amount=jit, seed=3)


def test_vertex_tet_lists():
    sc = _box()
    ptr, tet, corner = topology.vertex_tets(sc.n, sc.tets)
    assert ptr[-1] == 4 * sc.T
    for v in range(sc.n):
        ts = tet[ptr[v]:ptr[v + 1]]
        assert np.all(np.diff(ts) > 0)
        assert np.all(sc.tets[ts, corner[ptr[v]:ptr[v + 1]]] == v)
    # every (tet, corner) pair appears exactly once
    pairs = set(zip(tet.tolist(), corner.tolist()))
    assert len(pairs) == 4 * sc.T


def test_neighbors_are_the_shared_tet_graph():
    sc = _box()
    ptr, idx = topology.vertex_neighbors(sc.n, sc.tets)
    # independent: adjacency from the incidence matrix product
    rows = np.repeat(np.arange(sc.T), 4)
    inc = sp.csr_matrix((np.ones(4 * sc.T), (rows, sc.tets.ravel())), shape=(sc.T, sc.n))
    A = (inc.T @ inc).tocsr()
    A.setdiag(0)
    A.eliminate_zeros()
    A.sort_indices()
    np.testing.assert_array_equal(ptr, A.indptr)
    np.testing.assert_array_equal(idx, A.indices)


def test_greedy_coloring_valid_and_first_fit():
    sc = _box(5, 0.05)
    ptr, idx = topology.vertex_neighbors(sc.n, sc.tets)
    col = topology.greedy_coloring(sc.n, ptr, idx)
    for v in range(sc.n):
        nb = idx[ptr[v]:ptr[v + 1]]
        assert np.all(col[nb] != col[v])
        lower = set(col[nb[nb < v]].tolist())
        assert all(c in lower for c in range(col[v]))   # first fit in index order


def test_eight_colors_on_kuhn_grids():
    for dims in [(8, 8, 8), (3, 5, 4)]:
        X = meshgen.grid_vertices(*dims)
        T = meshgen.kuhn_tets(*dims)
        ptr, idx = topology.vertex_neighbors(X.shape[0], T)
        assert topology.greedy_coloring(X.shape[0], ptr, idx).max() + 1 == 8


def test_k_ring_matches_adjacency_power():
    sc = _box()
    ptr, idx = topology.vertex_neighbors(sc.n, sc.tets)
    A = sp.csr_matrix((np.ones(len(idx)), idx, ptr), shape=(sc.n, sc.n)) + sp.identity(sc.n)
    for k in (1, 2, 3):
        P = A.copy()
        for _ in range(k - 1):
            P = (P @ A).tocsr()
        for v in range(0, sc.n, 7):
            ring = topology.k_ring(v, k, ptr, idx)
            np.testing.assert_array_equal(ring, np.sort(P[v].indices))


def test_interior_ring_sizes_on_kuhn_grid():
    X = meshgen.grid_vertices(8, 8, 8)
    T = meshgen.kuhn_tets(8, 8, 8)
    ptr, idx = topology.vertex_neighbors(X.shape[0], T)
    centre = 4 + 9 * (4 + 9 * 4)
    assert ptr[centre + 1] - ptr[centre] == 14
    assert len(topology.k_ring(centre, 2, ptr, idx)) == 65
    assert len(topology.k_ring(centre, 3, ptr, idx)) == 175


def test_supports_exclude_self_and_pinned():
    sc = _box()
    free = sc.pinned == 0
    topo = topology.Topology(sc.n, sc.tets, free)
    for v, S in enumerate(topo.supports(2)):
        if not free[v]:
            assert len(S) == 0
        else:
            assert v not in S and np.all(free[S]) and np.all(np.diff(S) > 0)


@pytest.mark.parametrize("dims", [(3, 4, 5), (8, 8, 8), (6, 2, 9)])
def test_lattice_colouring_is_valid_with_four_colours(dims):
    """(i + j + k) mod 4 colours every Kuhn grid: no two vertices of a tet
    alike (checked on the tets themselves, jittered or not), four colours."""
    tets = meshgen.kuhn_tets(*dims)
    col = meshgen.lattice_colors(*dims)
    c = col[tets]
    for a in range(4):
        for b in range(a + 1, 4):
            assert np.all(c[:, a] != c[:, b])
    assert set(np.unique(col)) == {0, 1, 2, 3}
    n = (dims[0] + 1) * (dims[1] + 1) * (dims[2] + 1)
    topo = topology.Topology(n, tets, np.ones(n, bool), colors=col)
    assert topo.num_colors == 4
    with pytest.raises(ValueError):
        topology.Topology(n, tets, np.ones(n, bool), colors=np.zeros(n, np.int32))
