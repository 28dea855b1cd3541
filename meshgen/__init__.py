"""Seeded synthetic inputs for the Coordinate Condensation hot path.

This module is the only code shared by the FP64 oracle (``oracle/``) and the
CUDA path (``paper_2510_12053_gb300``) and by the tests that compare them.
It builds meshes, boundary conditions and material parameters and draws the
random numbers the inputs need.  It holds none of the method's arithmetic: no
energy, no derivative, no subspace, no solve.

Workloads follow the paper's tests, transposed to 3D tetrahedral meshes:

* stretch of a box with one face clamped and the opposite face pulled along
  its normal (teaser and mesh-resolution test, Section 4.2);
* a cantilever beam under gravity (subspace-quality test, Section 4.4),
  integrated with backward Euler (Eq. 2 and its footnote);
* jittered boxes of random size and material for batching and for training a
  learned subspace (no counterpart in the paper).

Grid convention ("Kuhn" 6-tet split, consistent diagonals):
vertex ``(i, j, k)`` has id ``i + (nx+1) * (j + (ny+1) * k)``; cells are
enumerated x-fastest; each cell yields 6 tets, one per permutation ``p`` of the
axes (lexicographic order), with corners ``v0 = (i,j,k)``, ``v1 = v0 + e[p0]``,
``v2 = v1 + e[p1]``, ``v3 = v0 + (1,1,1)``.  Odd permutations have ``v1`` and
``v2`` swapped so that every tet is positively oriented.

Random numbers come from a counter-based generator: the SplitMix64 output
function (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to ``seed + (counter + 1) * golden_gamma``.
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import List, Optional

import numpy as np

_GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter) -> np.ndarray:
    """SplitMix64 output for ``seed`` at integer ``counter`` (array-valued)."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * _GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counter) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of :func:`splitmix64`."""
    return (splitmix64(seed, counter) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, counter) -> np.ndarray:
    """Standard normal doubles by Box-Muller on two counter streams."""
    c = np.asarray(counter, dtype=np.uint64)
    u1 = 1.0 - uniform01(seed, 2 * c)
    u2 = uniform01(seed, 2 * c + np.uint64(1))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


@dataclasses.dataclass
class Material:
    """Isotropic material: Young's modulus E [Pa], Poisson ratio nu, density rho."""

    E: float
    nu: float
    rho: float = 1000.0


@dataclasses.dataclass
class Scene:
    """One simulation input.

    ``X`` rest positions ``[n, 3]`` float64; ``tets`` ``[T, 4]`` int32;
    ``pinned`` ``[n]`` uint8 (1 = Dirichlet vertex); ``x0`` initial positions
    ``[n, 3]`` (pinned rows hold their prescribed targets); ``v0`` initial
    velocities ``[n, 3]`` or None (quasistatic); ``h`` time step (0 for
    quasistatic); ``gravity`` acceleration vector ``[3]``.
    """

    name: str
    X: np.ndarray
    tets: np.ndarray
    pinned: np.ndarray
    x0: np.ndarray
    material: Material
    v0: Optional[np.ndarray] = None
    h: float = 0.0
    gravity: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(3))
    dims: tuple = ()
    cell: float = 1.0

    @property
    def n(self) -> int:
        return int(self.X.shape[0])

    @property
    def T(self) -> int:
        return int(self.tets.shape[0])

    @property
    def dynamic(self) -> bool:
        return self.h > 0.0


def grid_vertices(nx: int, ny: int, nz: int, cell: float = 1.0) -> np.ndarray:
    """Lattice positions ``[n, 3]`` with ids ``i + (nx+1)(j + (ny+1)k)``."""
    i, j, k = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    ijk = np.stack([i.ravel(order="F"), j.ravel(order="F"), k.ravel(order="F")], axis=1)
    # ravel(order="F") with indexing="ij" makes i the fastest index
    return ijk.astype(np.float64) * cell


def kuhn_tets(nx: int, ny: int, nz: int) -> np.ndarray:
    """Tets ``[6*nx*ny*nz, 4]`` of the Kuhn split, positively oriented."""
    sx, sy = nx + 1, (nx + 1) * (ny + 1)
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = ci.ravel(order="F"), cj.ravel(order="F"), ck.ravel(order="F")
    base = ci + sx * cj + sy * ck
    step = np.array([1, sx, sy], dtype=np.int64)
    out = np.empty((base.size, 6, 4), dtype=np.int64)
    for p_idx, perm in enumerate(itertools.permutations(range(3))):
        v0 = base
        v1 = v0 + step[perm[0]]
        v2 = v1 + step[perm[1]]
        v3 = v0 + step.sum()
        inversions = sum(1 for a in range(3) for b in range(a + 1, 3) if perm[a] > perm[b])
        if inversions % 2 == 1:
            v1, v2 = v2, v1
        out[:, p_idx, 0], out[:, p_idx, 1], out[:, p_idx, 2], out[:, p_idx, 3] = v0, v1, v2, v3
    return out.reshape(-1, 4).astype(np.int32)


def lattice_colors(nx: int, ny: int, nz: int) -> np.ndarray:
    """``(i + j + k) mod 4`` of every vertex's lattice coordinates ``[n]``.

    A vertex colouring of the Kuhn grid in which no two vertices of a tet
    share a colour: every tet edge joins ``v`` and ``v + d`` with ``d`` one of
    the seven non-zero 0/1 vectors (or its negative), whose coordinates sum to
    1, 2 or 3, never to a multiple of 4.  Jitter moves vertices, not edges, so
    it holds for jittered grids too."""
    i, j, k = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    return ((i + j + k).ravel(order="F") % 4).astype(np.int32)


def boundary_mask(nx: int, ny: int, nz: int) -> np.ndarray:
    """1 for vertices on the box surface."""
    i, j, k = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    on = (i == 0) | (i == nx) | (j == 0) | (j == ny) | (k == 0) | (k == nz)
    return on.ravel(order="F")


def jitter(X: np.ndarray, dims, cell: float, amount: float, seed: int) -> np.ndarray:
    """Move interior vertices by ``amount * cell * u`` per axis, ``u`` in [-1, 1)."""
    n = X.shape[0]
    ctr = np.arange(3 * n, dtype=np.uint64)
    u = 2.0 * uniform01(seed, ctr).reshape(n, 3) - 1.0
    inner = ~boundary_mask(*dims)
    Y = X.copy()
    Y[inner] += amount * cell * u[inner]
    return Y


def stretch_box(nx: int, ny: int, nz: int, *, E: float = 1e5, nu: float = 0.45, rho: float = 1000.0,
                size: float = 1.0, factor: float = 1.5, jitter_amount: float = 0.0, seed: int = 0,
                axis: int = 0, init: str = "linear", name: str = "") -> Scene:
    """Quasistatic stretch: face ``axis = 0`` clamped at rest, face ``axis = L``
    moved to ``factor * L`` along the axis (the other two coordinates stay at
    rest).  ``size`` is the box length along ``axis``; cells are cubes.

    ``init = "linear"`` starts from the rest shape stretched uniformly along
    the axis (the linear interpolation of the two clamped faces);
    ``init = "face"`` starts from the rest shape with only the pulled face
    moved.
    """
    dims = (nx, ny, nz)
    cell = size / dims[axis]
    X = grid_vertices(nx, ny, nz, cell)
    if jitter_amount > 0.0:
        X = jitter(X, dims, cell, jitter_amount, seed)
    tets = kuhn_tets(nx, ny, nz)
    L = dims[axis] * cell
    lo = np.isclose(X[:, axis], 0.0)
    hi = np.isclose(X[:, axis], L)
    pinned = (lo | hi).astype(np.uint8)
    x0 = X.copy()
    if init == "linear":
        x0[:, axis] = X[:, axis] * factor
    elif init == "face":
        x0[hi, axis] = factor * L
    else:
        raise ValueError(init)
    x0[lo] = X[lo]
    x0[hi, axis] = factor * L
    return Scene(name or f"stretch{nx}x{ny}x{nz}", X, tets, pinned, x0, Material(E, nu, rho),
                 dims=dims, cell=cell)


def cantilever(nx: int, ny: int, nz: int, *, cell: float, E: float = 1e7, nu: float = 0.45,
               rho: float = 1000.0, h: float = 1.0 / 60.0, g: float = 9.8, name: str = "") -> Scene:
    """Dynamic cantilever: long axis z, the z = 0 face clamped, gravity along -y,
    backward Euler with step ``h``, starting at rest with zero velocity."""
    dims = (nx, ny, nz)
    X = grid_vertices(nx, ny, nz, cell)
    tets = kuhn_tets(nx, ny, nz)
    pinned = np.isclose(X[:, 2], 0.0).astype(np.uint8)
    return Scene(name or f"beam{nx}x{ny}x{nz}", X, tets, pinned, X.copy(), Material(E, nu, rho),
                 v0=np.zeros_like(X), h=h, gravity=np.array([0.0, -g, 0.0]), dims=dims, cell=cell)


def twist_box(nx: int, ny: int, nz: int, *, E: float = 1e5, nu: float = 0.3, rho: float = 1000.0,
              angle: float = 1.5707963267948966, jitter_amount: float = 0.0, seed: int = 0,
              name: str = "twist") -> Scene:
    """Bar along z (``nz`` cells long, unit cell size scaled so the longest
    side is 1), both end faces clamped, the z = L face turned by ``angle``
    about the bar's axis.  Initial guess: every cross-section turned by
    ``angle * z / L`` (a uniform twist), so elements start far from their rest
    orientation."""
    cell = 1.0 / max(nx, ny, nz)
    X = grid_vertices(nx, ny, nz, cell)
    if jitter_amount > 0.0:
        X = jitter(X, (nx, ny, nz), cell, jitter_amount, seed)
    tets = kuhn_tets(nx, ny, nz)
    L = nz * cell
    cx, cy = 0.5 * nx * cell, 0.5 * ny * cell
    lo = np.isclose(X[:, 2], 0.0)
    hi = np.isclose(X[:, 2], L)
    pinned = (lo | hi).astype(np.uint8)
    th = angle * X[:, 2] / L
    c, s_ = np.cos(th), np.sin(th)
    x0 = X.copy()
    x0[:, 0] = cx + c * (X[:, 0] - cx) - s_ * (X[:, 1] - cy)
    x0[:, 1] = cy + s_ * (X[:, 0] - cx) + c * (X[:, 1] - cy)
    return Scene(name, X, tets, pinned, x0, Material(E, nu, rho), dims=(nx, ny, nz), cell=cell)


def random_box(index: int, seed: int, *, side_lo: int = 4, side_hi: int = 24, E_lo: float = 1e4,
               E_hi: float = 1e7, nu_lo: float = 0.30, nu_hi: float = 0.49, f_lo: float = 1.1,
               f_hi: float = 1.8, jitter_amount: float = 0.0, init: str = "linear") -> Scene:
    """Box number ``index`` of a seeded family: sides uniform in
    ``{side_lo..side_hi}`` cells, unit total length along the longest side,
    ``E`` log-uniform, ``nu`` uniform, a random face clamped and the opposite
    face stretched by a factor uniform in ``[f_lo, f_hi]``.

    Draws use counters ``16 * index + slot`` of :func:`uniform01`.
    """
    u = uniform01(seed, 16 * index + np.arange(8, dtype=np.uint64))
    span = side_hi - side_lo + 1
    sides = [side_lo + min(int(u[a] * span), span - 1) for a in range(3)]
    E = float(np.exp(np.log(E_lo) + u[3] * (np.log(E_hi) - np.log(E_lo))))
    nu = float(nu_lo + u[4] * (nu_hi - nu_lo))
    face = min(int(u[5] * 6), 5)
    factor = float(f_lo + u[6] * (f_hi - f_lo))
    axis, flip = face // 2, face % 2 == 1
    cell = 1.0 / max(sides)
    nx, ny, nz = sides
    X = grid_vertices(nx, ny, nz, cell)
    if jitter_amount > 0.0:
        X = jitter(X, (nx, ny, nz), cell, jitter_amount, seed ^ (0x5DEECE66D * (index + 1)))
    tets = kuhn_tets(nx, ny, nz)
    L = sides[axis] * cell
    coord = X[:, axis] if not flip else L - X[:, axis]
    lo = np.isclose(coord, 0.0)
    hi = np.isclose(coord, L)
    pinned = (lo | hi).astype(np.uint8)
    x0 = X.copy()
    # stretch along the axis away from the clamped face
    if init == "linear":
        new = coord * factor
    else:
        new = coord.copy()
        new[hi] = factor * L
    new[lo] = 0.0
    new[hi] = factor * L
    x0[:, axis] = new if not flip else L - new
    return Scene(f"box{index}", X, tets, pinned, x0, Material(E, nu, 1000.0), dims=(nx, ny, nz), cell=cell)


def random_boxes(count: int, seed: int, **kw) -> List[Scene]:
    return [random_box(i, seed, **kw) for i in range(count)]


# Named workloads (the sizes of the paper-shaped tests)
def cube8_stretch(E: float = 1e5, init: str = "linear") -> Scene:
    """8x8x8-cell unit cube (729 vertices, 3 072 tets), clamped at x=0, pulled to 1.5 at x=1."""
    return stretch_box(8, 8, 8, E=E, nu=0.45, init=init, name="cube8_stretch")


def cube32_stretch(E: float = 1e5, seed: int = 0, init: str = "linear") -> Scene:
    """32x32x32-cell unit cube (35 937 vertices, 196 608 tets), jittered by +-5% of a cell."""
    return stretch_box(32, 32, 32, E=E, nu=0.45, jitter_amount=0.05, seed=seed, init=init,
                       name="cube32_stretch")


def cube48_stretch(E: float = 1e6, seed: int = 0, init: str = "linear", nu: float = 0.45,
                   jitter_amount: float = 0.05) -> Scene:
    """48x48x48-cell unit cube (117 649 vertices, 663 552 tets)."""
    return stretch_box(48, 48, 48, E=E, nu=nu, jitter_amount=jitter_amount, seed=seed, init=init,
                       name="cube48_stretch")


def beam_dynamic(nx: int = 64, ny: int = 64, nz: int = 256) -> Scene:
    """Cantilever of 1/64 m cells (64x64x256 cells: 1 085 825 vertices, 6 291 456 tets)."""
    return cantilever(nx, ny, nz, cell=1.0 / 64.0, E=1e7, nu=0.45, rho=1000.0, h=1.0 / 60.0,
                      name=f"beam{nx}x{ny}x{nz}")


# ---------------------------------------------------------------------------
# Learned-subspace inputs: training meshes, initial weights, minibatch draws
# ---------------------------------------------------------------------------
def training_boxes(count: int, seed: int, side_lo: int = 4, side_hi: int = 12,
                   jitter_amount: float = 0.05) -> List[Scene]:
    """Jittered random boxes for training the subspace network: sides uniform
    in ``{side_lo..side_hi}`` cells, otherwise the batch family of
    :func:`random_box` (random clamped face, stretch, ``E``, ``nu``)."""
    return [random_box(i, seed, side_lo=side_lo, side_hi=side_hi, jitter_amount=jitter_amount)
            for i in range(count)]


def mlp_dims(hidden: int = 256, layers: int = 3, slots: int = 64, channels: int = 4,
             extra: int = 2, out_per_slot: int = 9) -> List[int]:
    """Layer widths of the subspace network: input, ``layers`` hidden widths, output."""
    return [slots * channels + extra] + [hidden] * layers + [slots * out_per_slot]


def mlp_param_count(dims: List[int]) -> int:
    return sum(dims[l + 1] * dims[l] + dims[l + 1] for l in range(len(dims) - 1))


def mlp_init(dims: List[int], seed: int, out_scale: float = 0.1) -> np.ndarray:
    """Initial parameters as one float32 vector, layer by layer: W_l row-major
    ``[dims[l+1], dims[l]]`` followed by b_l ``[dims[l+1]]``.  Hidden weights
    are normal with variance 2 / fan_in (He et al. 2015), the output layer's
    are scaled by ``out_scale``; biases start at zero."""
    parts, ctr = [], 0
    L = len(dims) - 1
    for l in range(L):
        n_out, n_in = dims[l + 1], dims[l]
        z = normal(seed, np.arange(ctr, ctr + n_out * n_in, dtype=np.uint64))
        ctr += n_out * n_in
        std = np.sqrt(2.0 / n_in) * (out_scale if l == L - 1 else 1.0)
        parts.append((z * std).astype(np.float32))
        parts.append(np.zeros(n_out, dtype=np.float32))
    return np.concatenate(parts)


def batch_indices(seed: int, step0: int, steps: int, batch: int, n: int) -> np.ndarray:
    """Minibatch sample indices ``[steps, batch]`` int32 for training steps
    ``step0 .. step0 + steps - 1``, drawn uniformly with replacement from
    ``n`` samples (counter ``step * batch + b``)."""
    c = np.arange(step0 * batch, (step0 + steps) * batch, dtype=np.uint64)
    idx = np.minimum((uniform01(seed, c) * n).astype(np.int64), n - 1)
    return idx.astype(np.int32).reshape(steps, batch)
