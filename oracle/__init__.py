"""Plain FP64 CPU oracle for Coordinate Condensation (arxiv 2510.12053).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import, call or execute anything in this package.
The CUDA library never calls into it, and it never calls into the CUDA
library: the two share no code.  Their only common dependency is the seeded
input generator ``meshgen`` (meshes, boundary conditions, random numbers),
which holds none of the method's arithmetic.

Everything is float64 NumPy/SciPy, written for a reader checking it against
the paper by eye: per-tet quantities are evaluated for all tets at once with
``einsum`` on the formula itself; per-vertex solves are plain Python loops.

Modules
-------
``material``  stable Neo-Hookean and linear (Hooke) energy densities with
              their first and second derivatives (energy of Eq. 2).
``fem``       rest data, per-tet energy / gradient / Hessian, global assembly
              of ``E = 1/2 (x - xt)^T M (x - xt) + h^2 Psi(x)`` (Eq. 2).
``topology``  vertex-tet and vertex-vertex adjacency, greedy colouring, k-rings.
``subspace``  perturbation bases ``U_i = -H_CC^{-1} H_Ci`` (Eq. 4-5, Sec. 3.1).
``solvers``   coordinate descent (Eq. 3), JGS2 (Eq. 7), Coordinate
              Condensation (Eq. 9-12, Algorithm 1), Newton, line search,
              termination measures (Sec. 4.1).
``mlp``       the subspace network (no counterpart in the paper): forward and
              backward passes with the bfloat16 rounding points of the
              tensor-core path, mean squared error, Adam.
``learned``   stencil slots, network inputs and targets, assembly of learned
              bases, and the per-vertex fallback rule (residual of Eq. 5).

Parity status: every function listed above is pinned by ``tests/test_oracle_*``
against finite differences, invariants, textbook formulas or brute force,
except the convergence *rates* of truncated-basis CC on 3D stable Neo-Hookean
meshes, which the paper does not print (parity unpinned for rates; pinned
only through GPU-vs-oracle trajectories).
"""
