"""Learned perturbation bases: stencil slots, network inputs and targets,
assembly of predicted bases, and the per-vertex fallback rule.

The paper builds every U_i by the patch solve of Eq. 5 (Sec. 3.1).  Nothing
learned appears in it; this module is the float64 oracle for a learned
replacement of that build on lattice meshes, in which a network (``mlp``)
maps the rest geometry of i's 2-ring and its material to U_i on the 2-ring
support S_i (k = 2), and a trial sweep decides, vertex by vertex, whether the
prediction is kept or replaced by the computed basis.

Slots.  The 2-ring of an interior vertex of the Kuhn lattice holds 64
vertices.  Their integer lattice offsets, ordered by hop count (the 14
1-ring offsets first) and then lexicographically, number the 64 slots.
``stencil()`` derives them from a generated lattice, not from a table.

Inputs of a free vertex i (float64, then bfloat16 as the GPU stores them):
  l_i   = mean over the 1-ring j of max_a |X_j[a] - X_i[a]|  (every Kuhn edge
          spans exactly one cell along its longest axis, so l_i is the cell
          size of an unjittered lattice);
  q_j   = (X_j - X_i) / l_i for every j within 2 hops (pinned ones too),
  o_j   = floor(q_j + 1/2) componentwise, the lattice offset, whose slot s
          receives channels 4s..4s+2 = 8 (q_j - o_j) and 4s+3 = +1 (free j)
          or -1 (pinned j); slots without a vertex stay zero;
  channel 256 = (log10 E - 5.5) / 1.5, channel 257 = 10 (nu - 0.4).
The basis does not change when the mesh is scaled (H_PP and H_Pi scale
alike), so dividing by l_i loses nothing; the offset o_j is implied by the
slot, so only the deviation from the lattice point is fed.

Targets: U_i[j] (3x3, rows = DOFs of j, columns = directions of i) of the
computed k = 2 basis at columns 9 s(j) .. 9 s(j) + 8 for j in S_i, zero
elsewhere.

Fallback rule (per vertex).  The computed basis is the solution of the
patch equilibrium H_PP U_i + H_Pi = 0 at rest (Eq. 5 on P = S_i).  A learned
basis leaves the residual

    rho_i = ||H_PP U_i + H_Pi||_F / ||H_Pi||_F,

and the plain update (coordinate descent, which is CC with U_i = 0) leaves
exactly rho_i = 1.  Vertex i falls back to its computed basis when its
learned basis reduces this residual no more than the plain one does,
rho_i >= tau with tau = 1 by default.  (A sweep-residual comparison is not
used: after one sweep from x0 even the exact computed bases leave a larger
||g_i|| than coordinate descent at most vertices, because CC's gain appears
over several sweeps.)
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np

from .fem import Problem
from .subspace import dofs, local_basis
from .topology import Topology, k_ring

SLOTS = 64
CHANNELS = 4
D_IN = SLOTS * CHANNELS + 2
D_OUT = SLOTS * 9
DEV_SCALE = 8.0


def stencil() -> List[Tuple[int, int, int]]:
    """The 64 lattice offsets of an interior vertex's 2-ring, by (hop, offset)."""
    import meshgen
    n = 6
    X = meshgen.grid_vertices(n, n, n, 1.0)
    tets = meshgen.kuhn_tets(n, n, n)
    topo = Topology(len(X), tets, np.ones(len(X), dtype=bool))
    c = 3 + (n + 1) * (3 + (n + 1) * 3)
    one = set(int(j) for j in topo.nbr_idx[topo.nbr_ptr[c]:topo.nbr_ptr[c + 1]])
    two = [int(j) for j in k_ring(c, 2, topo.nbr_ptr, topo.nbr_idx) if j != c]
    offs = []
    for j in two:
        o = tuple(int(round(v)) for v in (X[j] - X[c]))
        offs.append((1 if j in one else 2, o))
    offs.sort()
    return [o for _, o in offs]


def slot_table() -> Dict[Tuple[int, int, int], int]:
    return {o: s for s, o in enumerate(stencil())}


def lattice_spacing(X: np.ndarray, topo: Topology, i: int) -> float:
    nb = topo.nbr_idx[topo.nbr_ptr[i]:topo.nbr_ptr[i + 1]]
    if len(nb) == 0:
        raise ValueError(f"vertex {i} has no neighbours")
    acc = 0.0
    for j in nb:
        acc += float(np.max(np.abs(X[j] - X[i])))
    return acc / len(nb)


def offsets(X: np.ndarray, topo: Topology, i: int, table) -> List[Tuple[int, int, np.ndarray]]:
    """(j, slot, q - o) for every j within 2 hops of i, ascending j."""
    ell = lattice_spacing(X, topo, i)
    out, used = [], set()
    for j in k_ring(i, 2, topo.nbr_ptr, topo.nbr_idx):
        if j == i:
            continue
        q = (X[j] - X[i]) / ell
        o = tuple(int(v) for v in np.floor(q + 0.5))
        if o not in table:
            raise ValueError(f"vertex {j} is off the 2-ring stencil of {i}")
        s = table[o]
        if s in used:
            raise ValueError(f"two vertices share slot {s} of vertex {i}")
        used.add(s)
        out.append((j, s, q - np.array(o, dtype=np.float64)))
    return out


def material_channels(E: float, nu: float) -> Tuple[float, float]:
    return (np.log10(E) - 5.5) / 1.5, 10.0 * (nu - 0.4)


def features(problem: Problem, topo: Topology):
    """(rows, X64, Xbf): free vertices ascending, inputs [n_f, 258] in float64
    and rounded to bfloat16 (as float64)."""
    from .mlp import bf16
    table = slot_table()
    rows = np.flatnonzero(problem.free)
    F = np.zeros((len(rows), D_IN))
    cE, cnu = material_channels(problem.model.E, problem.model.nu)
    for r, i in enumerate(rows):
        for j, s, dev in offsets(problem.X, topo, int(i), table):
            F[r, CHANNELS * s:CHANNELS * s + 3] = DEV_SCALE * dev
            F[r, CHANNELS * s + 3] = 1.0 if problem.free[j] else -1.0
        F[r, SLOTS * CHANNELS] = cE
        F[r, SLOTS * CHANNELS + 1] = cnu
    return rows, F, bf16(F)


def targets(problem: Problem, topo: Topology, sup, bases) -> np.ndarray:
    """[n_f, 576]: the computed k = 2 basis of every free vertex in slot order."""
    table = slot_table()
    rows = np.flatnonzero(problem.free)
    Y = np.zeros((len(rows), D_OUT))
    for r, i in enumerate(rows):
        slot_of = {j: s for j, s, _ in offsets(problem.X, topo, int(i), table)}
        for a, j in enumerate(sup[i]):
            s = slot_of[int(j)]
            Y[r, 9 * s:9 * s + 9] = bases[i][a].reshape(9)
    return Y


def assemble(problem: Problem, topo: Topology, Y: np.ndarray):
    """(supports, bases) with U_i[j] read from the prediction row of i at the
    slot of j, on the k = 2 supports."""
    table = slot_table()
    rows = np.flatnonzero(problem.free)
    sup = topo.supports(2)
    bases = [np.zeros((0, 3, 3)) for _ in range(problem.n)]
    for r, i in enumerate(rows):
        slot_of = {j: s for j, s, _ in offsets(problem.X, topo, int(i), table)}
        bases[i] = np.stack([Y[r, 9 * slot_of[int(j)]:9 * slot_of[int(j)] + 9].reshape(3, 3)
                             for j in sup[i]]) if len(sup[i]) else np.zeros((0, 3, 3))
    return sup, bases


def basis_residual(problem: Problem, sup, bases, H=None) -> np.ndarray:
    """rho_i of every vertex at the rest Hessian (0 for pinned vertices and
    empty supports)."""
    H = problem.hessian(problem.X) if H is None else H
    rho = np.zeros(problem.n)
    for i in np.flatnonzero(problem.free):
        S = sup[i]
        if len(S) == 0:
            continue
        P, I = dofs(S), dofs([int(i)])
        Hr = H[P]
        H_Pi = Hr[:, I].toarray()
        R = Hr[:, P] @ np.asarray(bases[i]).reshape(3 * len(S), 3) + H_Pi
        rho[i] = np.linalg.norm(R) / np.linalg.norm(H_Pi)
    return rho


def fallback_set(problem: Problem, sup, bases, tau: float = 1.0, H=None):
    """(F, rho): free vertices with a non-empty support and rho_i >= tau."""
    rho = basis_residual(problem, sup, bases, H)
    F = np.array([i for i in np.flatnonzero(problem.free) if len(sup[i]) and rho[i] >= tau], dtype=np.int64)
    return F, rho


def with_fallback(problem: Problem, sup, bases, tau: float = 1.0):
    """Learned bases with the fallback set replaced by computed ones (Eq. 5 on
    the same supports at the rest Hessian).  Returns (bases, F, rho)."""
    H = problem.hessian(problem.X)
    F, rho = fallback_set(problem, sup, bases, tau, H)
    out = list(bases)
    for i in F:
        out[int(i)] = local_basis(H, int(i), sup[int(i)])
    return out, F, rho
