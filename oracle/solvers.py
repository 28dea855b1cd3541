"""Local updates, sweeps and outer solvers (plain float64).

Local updates for a free vertex i with gradient g and Hessian H evaluated at
the current x, support S (ascending free vertices) and basis blocks U (Eq. 5,
restricted to S; U is zero elsewhere, so every sum over C reduces to S):

* coordinate descent (Eq. 3), taken as one Newton step on the vertex:
      dx_i = -H_ii^{-1} g_i
* JGS2 (Eq. 7, as printed):
      dx_i = -(H_ii + U^T H_CC U)^{-1} (g_i + U^T g_C)
* Coordinate Condensation (Eq. 9-12): with A = H_iC U, Ht = U^T H_CC U,
  b = U^T g_C,
      S  = A Ht^{-1} A^T,   gt = g_i - A Ht^{-1} b,
      dx_i = -(H_ii - S)^{-1} gt,
  and the subspace part U dalpha_i is discarded (Sec. 3.1, "Maintaining
  Locality").

Guard (the paper is silent on indefinite local systems): a 3x3 matrix counts
as SPD when its plain Cholesky pivots all exceed 1e-12 times its largest
diagonal entry (and that entry is positive).  CC falls back to the CD step
when U is empty, when Ht fails that test, or when H_ii - S fails it; JGS2
falls back when H_ii + Ht fails it.  Fallbacks are counted.

Schedules: Jacobi (Algorithm 1: g, H once per iteration, every free vertex
updated from them, then x <- x + d) and coloured Gauss-Seidel (for each colour
in turn, g and H are re-evaluated at the current x and the vertices of that
colour are updated from them; Jacobi is the one-colour case).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import Problem
from .subspace import dofs
from .topology import Topology

PIVOT_REL = 1e-12


def spd_ok(M: np.ndarray) -> bool:
    """Plain Cholesky of a small symmetric matrix: every pivot > 1e-12 * max diag."""
    d = np.max(np.diag(M))
    if not d > 0.0:
        return False
    L = np.zeros_like(M)
    m = M.shape[0]
    for c in range(m):
        piv = M[c, c] - np.dot(L[c, :c], L[c, :c])
        if not piv > PIVOT_REL * d:
            return False
        L[c, c] = np.sqrt(piv)
        for r in range(c + 1, m):
            L[r, c] = (M[r, c] - np.dot(L[r, :c], L[c, :c])) / L[c, c]
    return True


@dataclasses.dataclass
class Stats:
    fallback_empty: int = 0      # CC/JGS2 with an empty basis -> CD step
    fallback_reduced: int = 0    # Ht (CC) or H_ii + Ht (JGS2) not SPD -> CD step
    fallback_schur: int = 0      # H_ii - S not SPD -> CD step
    updates: int = 0


def local_terms(H, g: np.ndarray, i: int, S: np.ndarray, U: np.ndarray):
    """(H_ii, g_i, A, Ht, b) for vertex i; ``g`` is [n, 3], ``H`` 3n x 3n CSR."""
    I = dofs([i])
    Hi = H[I]
    H_ii = Hi[:, I].toarray()
    g_i = g[i].copy()
    if len(S) == 0:
        return H_ii, g_i, None, None, None
    P = dofs(S)
    Uf = U.reshape(3 * len(S), 3)
    A = Hi[:, P].toarray() @ Uf
    H_SS = H[P][:, P].toarray()
    Ht = Uf.T @ H_SS @ Uf
    b = Uf.T @ g[S].reshape(-1)
    return H_ii, g_i, A, Ht, b


def local_update(kind: str, H, g, i: int, S, U, stats: Optional[Stats] = None) -> np.ndarray:
    """dx_i for ``kind`` in {"cd", "jgs2", "cc"}."""
    H_ii, g_i, A, Ht, b = local_terms(H, g, i, S, U) if kind != "cd" else \
        (H[dofs([i])][:, dofs([i])].toarray(), g[i].copy(), None, None, None)
    if stats is not None:
        stats.updates += 1
    cd = -np.linalg.solve(H_ii, g_i)
    if kind == "cd":
        return cd
    if A is None:
        if stats is not None:
            stats.fallback_empty += 1
        return cd
    if kind == "jgs2":
        M = H_ii + Ht
        if not spd_ok(M):
            if stats is not None:
                stats.fallback_reduced += 1
            return cd
        return -np.linalg.solve(M, g_i + b)
    if kind != "cc":
        raise ValueError(kind)
    if not spd_ok(Ht):
        if stats is not None:
            stats.fallback_reduced += 1
        return cd
    Schur = A @ np.linalg.solve(Ht, A.T)
    gt = g_i - A @ np.linalg.solve(Ht, b)
    M = H_ii - Schur
    if not spd_ok(M):
        if stats is not None:
            stats.fallback_schur += 1
        return cd
    return -np.linalg.solve(M, gt)


def vertex_rotations(problem: Problem, topo: Topology, x: np.ndarray) -> np.ndarray:
    """Per-vertex rotations R_j [n, 3, 3] for corotated bases (Sec. 3.1,
    "Accounting for Large Deformations"; the paper estimates them from the
    displacement of each vertex's neighbourhood without giving the formula).
    Reading: fit the neighbourhood's deformation gradient by least squares,
    F_j = A_j C_j^{-1} with A_j = sum over the 1-ring l of (x_l - x_j)(X_l - X_j)^T
    and C_j = sum of (X_l - X_j)(X_l - X_j)^T, and take its orthogonal polar
    factor (scipy.linalg.polar).  This is exact for every homogeneous
    deformation (a rigid motion gives its rotation, a pure stretch the
    identity).  R_j = I when det F_j <= 0 (an inverted neighbourhood has no
    proper rotation to extract)."""
    from scipy.linalg import polar
    X = problem.X
    R = np.zeros((problem.n, 3, 3))
    for j in range(problem.n):
        nb = topo.nbr_idx[topo.nbr_ptr[j]:topo.nbr_ptr[j + 1]]
        A = np.zeros((3, 3))
        C = np.zeros((3, 3))
        for l in nb:
            A += np.outer(x[l] - x[j], X[l] - X[j])
            C += np.outer(X[l] - X[j], X[l] - X[j])
        F = A @ np.linalg.inv(C) if len(nb) else np.eye(3)
        if len(nb) == 0 or not np.linalg.det(F) > 0.0:
            R[j] = np.eye(3)
        else:
            R[j] = polar(F)[0]
    return R


def rotate_bases(sup, bases, R) -> list:
    """U_i^rot[j] = R_j U_i[j] for every support vertex j (the rotation formula of Sec. 3.1)."""
    return [np.einsum("aij,ajk->aik", R[np.asarray(S, dtype=np.int64)], U) if len(S) else U
            for S, U in zip(sup, bases)]


def sweep(problem: Problem, topo: Topology, sup, bases, x: np.ndarray, xt=None, kind: str = "cc",
          schedule: str = "colored", stats: Optional[Stats] = None, corotated: bool = False) -> np.ndarray:
    """One iteration: Jacobi (Algorithm 1) or coloured Gauss-Seidel.  Returns new x.

    With ``corotated`` the bases are rotated once per iteration, at its start,
    by the rotations of the current configuration (Sec. 3.1)."""
    x = np.array(x, dtype=np.float64, copy=True)
    if corotated:
        bases = rotate_bases(sup, bases, vertex_rotations(problem, topo, x))
    if schedule == "colored":
        groups = topo.color_classes(free_only=True)
    elif schedule == "jacobi":
        groups = [np.flatnonzero(problem.free)]
    else:
        raise ValueError(schedule)
    for group in groups:
        if len(group) == 0:
            continue
        g = problem.gradient(x, xt)
        H = problem.hessian(x)
        d = {int(i): local_update(kind, H, g, int(i), sup[i], bases[i], stats) for i in group}
        for i, di in d.items():
            x[i] += di
    return x


def jacobi_direction(problem: Problem, sup, bases, x, xt=None, kind: str = "cc",
                     stats: Optional[Stats] = None) -> np.ndarray:
    """d with d_i = local update of every free vertex from g, H at x (Algorithm 1)."""
    g = problem.gradient(x, xt)
    H = problem.hessian(x)
    d = np.zeros_like(x)
    for i in np.flatnonzero(problem.free):
        d[i] = local_update(kind, H, g, int(i), sup[i], bases[i], stats)
    return d


def backtracking(problem: Problem, x, d, xt=None, alpha0: float = 1.0, shrink: float = 0.5,
                 max_steps: int = 30, c: float = 0.0, g=None) -> float:
    """Largest alpha = alpha0 * shrink^m with E(x + alpha d) <= E(x) + c alpha g.d
    (c = 0: plain decrease, Sec. 4.4's global line search); 0 if none found."""
    E0 = problem.energy(x, xt)
    slope = 0.0 if (c == 0.0 or g is None) else float(np.sum(g * d))
    a = alpha0
    for _ in range(max_steps):
        if problem.energy(x + a * d, xt) <= E0 + c * a * slope:
            return a
        a *= shrink
    return 0.0


@dataclasses.dataclass
class History:
    energy: List[float]
    grad_norm: List[float]
    iterations: int = 0
    converged: bool = False

    @property
    def rel(self) -> List[float]:
        g0 = self.grad_norm[0] if self.grad_norm[0] > 0 else 1.0
        return [v / g0 for v in self.grad_norm]


def solve(problem: Problem, topo: Topology, sup, bases, x0, xt=None, kind: str = "cc",
          schedule: str = "colored", tol: float = 1e-6, max_iters: int = 100,
          line_search: bool = False, stats: Optional[Stats] = None, min_iters: int = 0,
          corotated: bool = False, restart_every: int = 0):
    """Iterate sweeps until ||g_free|| / ||g_free(x0)|| <= tol or max_iters.

    With ``line_search`` every iteration's updates form one global direction d
    (Jacobi: the local updates of all free vertices from g, H at x, as in
    Algorithm 1; coloured: d = sweep(x) - x) and x <- x + alpha d with alpha
    from backtracking on the energy (Sec. 4.4, "Sensitivity to basis quality").
    With ``restart_every`` = r > 0 the bases are rebuilt from the Hessian at
    the current x before iterations r, 2r, ... (restarted CC, Sec. 4.4)."""
    from .subspace import rebuild_bases_at
    x = np.array(x0, dtype=np.float64, copy=True)
    g = problem.gradient(x, xt)
    hist = History([problem.energy(x, xt)], [problem.free_gradient_norm(g)])
    g0 = hist.grad_norm[0]
    for it in range(max_iters):
        if it >= min_iters and (g0 == 0.0 or hist.grad_norm[-1] <= tol * g0):
            hist.converged = True
            break
        if restart_every > 0 and it > 0 and it % restart_every == 0:
            bases, _ = rebuild_bases_at(problem, sup, bases, x)
        if line_search:
            if schedule == "jacobi":
                B = rotate_bases(sup, bases, vertex_rotations(problem, topo, x)) if corotated else bases
                d = jacobi_direction(problem, sup, B, x, xt, kind, stats)
            else:
                d = sweep(problem, topo, sup, bases, x, xt, kind, schedule, stats, corotated) - x
            a = backtracking(problem, x, d, xt)
            x = x + a * d
        else:
            x = sweep(problem, topo, sup, bases, x, xt, kind, schedule, stats, corotated)
        g = problem.gradient(x, xt)
        hist.energy.append(problem.energy(x, xt))
        hist.grad_norm.append(problem.free_gradient_norm(g))
        hist.iterations = it + 1
    else:
        hist.converged = g0 == 0.0 or hist.grad_norm[-1] <= tol * g0
    return x, hist


def newton_direction(problem: Problem, x, xt=None) -> np.ndarray:
    """-H_ff^{-1} g_f (sparse direct solve); if that is not a descent direction,
    H_ff + tau I with tau = 1e-8 max diag, times 10 until it is."""
    g = problem.gradient(x, xt)
    H = problem.free_hessian(problem.hessian(x)).tocsc()
    gf = g.reshape(-1)[problem.free_dofs]
    tau = 0.0
    dmax = float(H.diagonal().max())
    for _ in range(20):
        M = H if tau == 0.0 else (H + tau * sp.identity(H.shape[0], format="csc"))
        df = spla.spsolve(M, -gf)
        if np.all(np.isfinite(df)) and float(df @ gf) < 0.0:
            break
        tau = 1e-8 * dmax if tau == 0.0 else tau * 10.0
    d = np.zeros(3 * problem.n)
    d[problem.free_dofs] = df
    return d.reshape(problem.n, 3)


def newton(problem: Problem, x0, xt=None, tol: float = 1e-6, max_iters: int = 50,
           line_search: bool = True):
    """Newton's method with Armijo backtracking (c = 1e-4, halving, <= 30 steps)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    g = problem.gradient(x, xt)
    hist = History([problem.energy(x, xt)], [problem.free_gradient_norm(g)])
    g0 = hist.grad_norm[0]
    for it in range(max_iters):
        if g0 == 0.0 or hist.grad_norm[-1] <= tol * g0:
            hist.converged = True
            break
        d = newton_direction(problem, x, xt)
        a = backtracking(problem, x, d, xt, c=1e-4, g=g) if line_search else 1.0
        if a == 0.0:
            a = 1.0
        x = x + a * d
        g = problem.gradient(x, xt)
        hist.energy.append(problem.energy(x, xt))
        hist.grad_norm.append(problem.free_gradient_norm(g))
        hist.iterations = it + 1
    else:
        hist.converged = g0 == 0.0 or hist.grad_norm[-1] <= tol * g0
    return x, hist


def normalized_residual(problem: Problem, grad_norm: float) -> float:
    """||g|| / (V n E), divided by h for dynamics (Sec. 4.1, termination criteria)."""
    r = grad_norm / (problem.total_volume() * problem.n * problem.model.E)
    return r / problem.h if problem.dynamic else r


def time_step(problem: Problem, topo: Topology, sup, bases, x_t, v_t, kind: str = "cc",
              schedule: str = "colored", tol: float = 1e-6, max_iters: int = 200, stats=None):
    """One backward Euler step: x^{t+1} = argmin E (Eq. 1-2), v^{t+1} = (x^{t+1} - x^t) / h.
    The solve starts from x^t with pinned vertices at their (fixed) targets."""
    xt = problem.inertial_target(x_t, v_t)
    x1, hist = solve(problem, topo, sup, bases, x_t, xt, kind, schedule, tol, max_iters, stats=stats)
    v1 = (x1 - x_t) / problem.h
    return x1, v1, hist
