"""Mesh adjacency, greedy colouring and k-ring supports (plain loops).

Conventions (fixed so that integer outputs can be compared bit for bit):

* vertex -> tet list: for every vertex its incident tets in ascending tet id,
  each as (tet, corner) with ``tets[tet, corner] == vertex``;
* vertex -> vertex list: the vertices sharing a tet with it, ascending,
  itself excluded (the "1-ring graph");
* block-sparse (3x3) Hessian pattern: row j holds j's 1-ring plus j itself,
  ascending;
* colouring: sequential greedy over all vertices (pinned ones included, the
  graph is pure topology) in ascending id; each vertex takes the smallest
  colour not used by an already coloured 1-ring neighbour.  Same-coloured
  vertices share no tet, so their local solves in a Gauss-Seidel sweep are
  independent (the paper's Sec. 2.2 contrasts Jacobi and Gauss-Seidel;
  colouring is the usual way to parallelise the latter);
* k-ring of i: vertices reachable from i in at most k 1-ring hops.
"""
from __future__ import annotations

from typing import List

import numpy as np


def vertex_tets(n: int, tets: np.ndarray):
    """CSR (ptr [n+1], tet [4T], corner [4T]) in ascending tet id per vertex."""
    tets = np.asarray(tets)
    lists = [[] for _ in range(n)]
    for t in range(tets.shape[0]):
        for c in range(4):
            lists[int(tets[t, c])].append((t, c))
    ptr = np.zeros(n + 1, dtype=np.int64)
    for v in range(n):
        ptr[v + 1] = ptr[v] + len(lists[v])
    tet = np.array([p[0] for L in lists for p in L], dtype=np.int64)
    corner = np.array([p[1] for L in lists for p in L], dtype=np.int64)
    return ptr, tet, corner


def vertex_neighbors(n: int, tets: np.ndarray):
    """CSR (ptr [n+1], idx) of the 1-ring graph, ascending, self excluded."""
    tets = np.asarray(tets)
    sets = [set() for _ in range(n)]
    for t in range(tets.shape[0]):
        vs = [int(v) for v in tets[t]]
        for a in vs:
            for b in vs:
                if a != b:
                    sets[a].add(b)
    ptr = np.zeros(n + 1, dtype=np.int64)
    for v in range(n):
        ptr[v + 1] = ptr[v] + len(sets[v])
    idx = np.array([b for v in range(n) for b in sorted(sets[v])], dtype=np.int64)
    return ptr, idx


def block_pattern(n: int, nbr_ptr, nbr_idx):
    """Row pattern of the 3x3-block Hessian: 1-ring plus the diagonal, ascending."""
    ptr = np.zeros(n + 1, dtype=np.int64)
    cols = []
    for v in range(n):
        row = sorted(list(nbr_idx[nbr_ptr[v]:nbr_ptr[v + 1]]) + [v])
        cols.extend(row)
        ptr[v + 1] = ptr[v] + len(row)
    return ptr, np.array(cols, dtype=np.int64)


def greedy_coloring(n: int, nbr_ptr, nbr_idx) -> np.ndarray:
    """Sequential greedy colouring in ascending vertex id (smallest free colour)."""
    color = np.full(n, -1, dtype=np.int64)
    for v in range(n):
        used = set()
        for u in nbr_idx[nbr_ptr[v]:nbr_ptr[v + 1]]:
            if color[u] >= 0:
                used.add(int(color[u]))
        c = 0
        while c in used:
            c += 1
        color[v] = c
    return color


def k_ring(v: int, k: int, nbr_ptr, nbr_idx) -> List[int]:
    """Vertices within k hops of v (v included), ascending, by breadth-first search."""
    seen = {v}
    frontier = [v]
    for _ in range(k):
        nxt = []
        for a in frontier:
            for b in nbr_idx[nbr_ptr[a]:nbr_ptr[a + 1]]:
                b = int(b)
                if b not in seen:
                    seen.add(b)
                    nxt.append(b)
        frontier = nxt
    return sorted(seen)


def supports(n: int, k: int, nbr_ptr, nbr_idx, free) -> List[np.ndarray]:
    """S_i = k-ring(i) minus i minus pinned vertices, for every vertex (pinned: empty)."""
    out = []
    for v in range(n):
        if not free[v]:
            out.append(np.zeros(0, dtype=np.int64))
            continue
        ring = [u for u in k_ring(v, k, nbr_ptr, nbr_idx) if u != v and free[u]]
        out.append(np.array(ring, dtype=np.int64))
    return out


class Topology:
    """All adjacency of one mesh, computed once."""

    def __init__(self, n: int, tets, free, colors=None):
        """``colors``: a given vertex colouring (no two vertices of a tet alike)
        in place of the greedy one; the coloured schedule only needs validity."""
        self.n = n
        self.vt_ptr, self.vt_tet, self.vt_corner = vertex_tets(n, tets)
        self.nbr_ptr, self.nbr_idx = vertex_neighbors(n, tets)
        self.bsr_ptr, self.bsr_col = block_pattern(n, self.nbr_ptr, self.nbr_idx)
        if colors is None:
            self.color = greedy_coloring(n, self.nbr_ptr, self.nbr_idx)
        else:
            self.color = np.asarray(colors, dtype=np.int64).copy()
            for v in range(n):
                if np.any(self.color[self.nbr_idx[self.nbr_ptr[v]:self.nbr_ptr[v + 1]]] == self.color[v]):
                    raise ValueError(f"vertex {v} shares its colour with a neighbour")
        self.num_colors = int(self.color.max()) + 1 if n else 0
        self.free = np.asarray(free).astype(bool)

    def color_classes(self, free_only: bool = True) -> List[np.ndarray]:
        out = []
        for c in range(self.num_colors):
            sel = self.color == c
            if free_only:
                sel = sel & self.free
            out.append(np.flatnonzero(sel))
        return out

    def supports(self, k: int) -> List[np.ndarray]:
        return supports(self.n, k, self.nbr_ptr, self.nbr_idx, self.free)
