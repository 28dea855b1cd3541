"""Perturbation bases U_i (Sec. 2.3, Eq. 4-5; Sec. 3.1).

For coordinate i (a free vertex, 3 DOFs) and complementary free DOFs C, the
basis solves the block system of Eq. 4 with zero force on C:

    U_iC = -H_CC^{-1} H_Ci                                    (Eq. 5)

evaluated at the rest configuration (Sec. 3.1).  A basis is stored as the
support ``sup`` (ascending vertex ids) and blocks ``U[s]`` (3x3): rows are the
DOFs of vertex ``sup[s]``, columns the three perturbation directions of i.

Constructions:
* ``global_basis``        Eq. 5 with a dense solve over all of C;
* ``global_basis_inverse``  the same from the inverse Hessian W = H^{-1}:
                          block inversion gives W_Ci = U_iC W_ii, hence
                          U_iC = W_Ci W_ii^{-1};
* ``local_basis``         Eq. 5 restricted to the patch P = S_i (the k-ring of
                          i without i and without pinned vertices), with every
                          DOF outside P held fixed: U_i = -H_PP^{-1} H_Pi.
                          This is the truncated basis the sweep uses.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np

from .fem import Problem
from .topology import Topology


def dofs(vertices) -> np.ndarray:
    v = np.asarray(vertices, dtype=np.int64)
    return (3 * v[:, None] + np.arange(3)[None, :]).ravel()


def local_basis(H, i: int, S: np.ndarray) -> np.ndarray:
    """U_i on patch S: solve H_PP U = -H_Pi (dense), returned as [|S|, 3, 3]."""
    if len(S) == 0:
        return np.zeros((0, 3, 3))
    P = dofs(S)
    Hr = H[P]
    H_PP = Hr[:, P].toarray()
    H_Pi = Hr[:, dofs([i])].toarray()
    U = -np.linalg.solve(H_PP, H_Pi)
    return U.reshape(len(S), 3, 3)


def build_local_bases(problem: Problem, topo: Topology, k: int, x=None) -> Tuple[List[np.ndarray], List[np.ndarray]]:
    """(supports, bases) for every vertex (pinned vertices get empty ones).

    The Hessian is taken at ``x`` (default: the rest positions, Sec. 3.1)."""
    H = problem.hessian(problem.X if x is None else x)
    sup = topo.supports(k)
    bases = [local_basis(H, i, sup[i]) if problem.free[i] else np.zeros((0, 3, 3))
             for i in range(problem.n)]
    return sup, bases


def rebuild_bases_at(problem: Problem, sup, bases, x) -> Tuple[List[np.ndarray], int]:
    """Restarted bases (Sec. 4.4, "Subspace quality"): Eq. 5 on the same
    supports with the Hessian at the current configuration x.  Reading (the
    paper is silent on indefinite patches): a patch whose H_PP is not
    positive definite (plain Cholesky fails) keeps its current basis.
    Returns (bases, number of patches kept)."""
    H = problem.hessian(x)
    out, kept = [], 0
    for i in range(problem.n):
        S = sup[i]
        if not problem.free[i] or len(S) == 0:
            out.append(bases[i])
            continue
        P = dofs(S)
        Hr = H[P]
        H_PP = Hr[:, P].toarray()
        try:
            np.linalg.cholesky(H_PP)
        except np.linalg.LinAlgError:
            out.append(bases[i])
            kept += 1
            continue
        out.append((-np.linalg.solve(H_PP, Hr[:, dofs([i])].toarray())).reshape(len(S), 3, 3))
    return out, kept


def global_basis(problem: Problem, H, i: int) -> Tuple[np.ndarray, np.ndarray]:
    """Eq. 5 over all complementary free DOFs: (support, [|S|, 3, 3])."""
    S = np.array([j for j in range(problem.n) if problem.free[j] and j != i], dtype=np.int64)
    Hd = H.toarray() if hasattr(H, "toarray") else np.asarray(H)
    C, I = dofs(S), dofs([i])
    U = -np.linalg.solve(Hd[np.ix_(C, C)], Hd[np.ix_(C, I)])
    return S, U.reshape(len(S), 3, 3)


def global_basis_inverse(problem: Problem, H, i: int) -> Tuple[np.ndarray, np.ndarray]:
    """U_iC = W_Ci W_ii^{-1} with W the inverse of the free Hessian."""
    F = np.flatnonzero(problem.free)
    Hd = H.toarray() if hasattr(H, "toarray") else np.asarray(H)
    Fd = dofs(F)
    W = np.linalg.inv(Hd[np.ix_(Fd, Fd)])
    pos = {int(v): p for p, v in enumerate(F)}
    S = np.array([j for j in F if j != i], dtype=np.int64)
    Ci = np.concatenate([np.arange(3 * pos[int(j)], 3 * pos[int(j)] + 3) for j in S]) if len(S) else np.zeros(0, int)
    Ii = np.arange(3 * pos[i], 3 * pos[i] + 3)
    U = W[np.ix_(Ci, Ii)] @ np.linalg.inv(W[np.ix_(Ii, Ii)])
    return S, U.reshape(len(S), 3, 3)


def truncate(S_full: np.ndarray, U_full: np.ndarray, S_keep: np.ndarray) -> np.ndarray:
    """Rows of a global basis restricted to the vertices ``S_keep``."""
    pos = {int(v): p for p, v in enumerate(S_full)}
    return np.stack([U_full[pos[int(j)]] for j in S_keep]) if len(S_keep) else np.zeros((0, 3, 3))


def add_noise(bases: List[np.ndarray], sigma: float, seed: int) -> List[np.ndarray]:
    """U_noisy = U + sigma * N, N iid standard normal per entry (Sec. 4.4,
    basis-quality test; random noise as its figure caption states)."""
    import meshgen
    out, ctr = [], 0
    for U in bases:
        m = U.size
        noise = meshgen.normal(seed, np.arange(ctr, ctr + m, dtype=np.uint64)).reshape(U.shape)
        out.append(U + sigma * noise)
        ctr += m
    return out


def all_global_bases(problem: Problem, x=None):
    """Untruncated bases of Eq. 5 for every free vertex, from one dense inverse
    of the free Hessian at ``x`` (default: rest), via U_iC = W_Ci W_ii^{-1}.
    Small meshes only (dense)."""
    H = problem.hessian(problem.X if x is None else x).toarray()
    F = np.flatnonzero(problem.free)
    Fd = dofs(F)
    W = np.linalg.inv(H[np.ix_(Fd, Fd)])
    pos = {int(v): p for p, v in enumerate(F)}
    sup, bases = [], []
    for i in range(problem.n):
        if not problem.free[i]:
            sup.append(np.zeros(0, dtype=np.int64))
            bases.append(np.zeros((0, 3, 3)))
            continue
        S = np.array([j for j in F if j != i], dtype=np.int64)
        Ci = np.concatenate([np.arange(3 * pos[int(j)], 3 * pos[int(j)] + 3) for j in S]) if len(S) else np.zeros(0, int)
        Ii = np.arange(3 * pos[i], 3 * pos[i] + 3)
        sup.append(S)
        bases.append((W[np.ix_(Ci, Ii)] @ np.linalg.inv(W[np.ix_(Ii, Ii)])).reshape(len(S), 3, 3))
    return sup, bases
