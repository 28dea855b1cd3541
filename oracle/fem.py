"""Finite-element energy of Eq. 2 on linear tetrahedra, in float64.

    E(x) = 1/2 (x - xt)^T M (x - xt) + h^2 Psi(x)        (Eq. 2, dynamic)
    E(x) = Psi(x)                                        (quasistatic reading)
    Psi(x) = sum_t V_t Psi(F_t),   F_t = D_s(x) D_m^{-1}

with ``D_s = [x1 - x0, x2 - x0, x3 - x0]`` (columns), ``V_t = |det D_m| / 6``,
lumped mass ``m_j = rho * sum_{t containing j} V_t / 4`` and the backward
Euler target ``xt = x^t + h v^t + h^2 g`` (footnote of Eq. 2, with gravity
``g`` folded into the target).  Positions are ``[n, 3]`` arrays; the global
DOF of vertex ``j``, axis ``a`` is ``3 j + a``.

Shape vectors: F = sum_v x_v (x) G_v with G_v = row v-1 of D_m^{-1} for
v = 1..3 and G_0 = -(G_1 + G_2 + G_3).  Hence
    dE_t/dx_v      = V_t P G_v
    d2E_t/dx_v dx_w = V_t sum_bd dP_ab/dF_cd G_v[b] G_w[d].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .material import Model


class Problem:
    """Rest data and energy evaluation for one tet mesh.

    ``pinned`` vertices are Dirichlet: they are removed from the unknowns
    (their gradient rows and Hessian rows/columns are dropped by ``free_*``).
    """

    def __init__(self, X, tets, pinned, model: Model, rho: float = 1000.0, h: float = 0.0,
                 gravity=None):
        self.X = np.asarray(X, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        self.n = self.X.shape[0]
        self.T = self.tets.shape[0]
        self.pinned = np.asarray(pinned).astype(bool)
        self.free = ~self.pinned
        self.model = model
        self.rho = rho
        self.h = float(h)
        self.gravity = np.zeros(3) if gravity is None else np.asarray(gravity, dtype=np.float64)
        Dm = self.edges(self.X)
        self.Bm = np.linalg.inv(Dm)
        self.vol = np.abs(np.linalg.det(Dm)) / 6.0
        G = np.empty((self.T, 4, 3))
        G[:, 1:, :] = self.Bm
        G[:, 0, :] = -self.Bm.sum(axis=1)
        self.G = G
        self.mass = np.zeros(self.n)
        np.add.at(self.mass, self.tets.ravel(), np.repeat(rho * self.vol / 4.0, 4))
        self.free_dofs = np.flatnonzero(np.repeat(self.free, 3))

    # ---- per-tet kinematics -------------------------------------------------
    def edges(self, x):
        """D_s [T, 3, 3]; column c is x_{c+1} - x_0."""
        x = np.asarray(x)
        p = x[self.tets]  # [T, 4, 3]
        return np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0], p[:, 3] - p[:, 0]], axis=2)

    def deformation(self, x):
        return self.edges(x) @ self.Bm

    @property
    def dynamic(self) -> bool:
        return self.h > 0.0

    @property
    def elastic_weight(self) -> float:
        """h^2 for the dynamic energy, 1 for quasistatics."""
        return self.h * self.h if self.dynamic else 1.0

    # ---- per-tet derivatives of V_t Psi(F_t) -------------------------------
    def tet_energy(self, x):
        return self.vol * self.model.energy(self.deformation(x))

    def tet_gradient(self, x):
        """[T, 4, 3]: g[t, v, a] = V_t sum_b P_ab G_v[b]."""
        P = self.model.stress(self.deformation(x))
        return self.vol[:, None, None] * np.einsum("tvb,tab->tva", self.G, P)

    def tet_hessian(self, x):
        """[T, 4, 3, 4, 3]: K[t, v, a, w, c] = V_t sum_bd dP_ab/dF_cd G_v[b] G_w[d]."""
        dP = self.model.dstress(self.deformation(x))
        return self.vol[:, None, None, None, None] * np.einsum(
            "tabcd,tvb,twd->tvawc", dP, self.G, self.G, optimize=True)

    # ---- inertial target ----------------------------------------------------
    def inertial_target(self, x_t, v_t):
        """xt = x^t + h v^t + h^2 g (backward Euler, gravity in the target)."""
        return x_t + self.h * v_t + self.h * self.h * self.gravity[None, :]

    # ---- global quantities ---------------------------------------------------
    def energy(self, x, xt=None):
        e = self.elastic_weight * self.tet_energy(x).sum()
        if self.dynamic:
            d = x - xt
            e += 0.5 * np.sum(self.mass[:, None] * d * d)
        return float(e)

    def gradient(self, x, xt=None):
        """Full gradient [n, 3] (pinned rows included; callers mask them)."""
        g = np.zeros((self.n, 3))
        np.add.at(g, self.tets, self.elastic_weight * self.tet_gradient(x))
        if self.dynamic:
            g += self.mass[:, None] * (x - xt)
        return g

    def hessian(self, x):
        """Full Hessian as a 3n x 3n CSR matrix (pinned rows included)."""
        K = self.elastic_weight * self.tet_hessian(x)
        dof = 3 * self.tets[:, :, None] + np.arange(3)[None, None, :]  # [T, 4, 3]
        rows = np.broadcast_to(dof[:, :, :, None, None], K.shape).ravel()
        cols = np.broadcast_to(dof[:, None, None, :, :], K.shape).ravel()
        H = sp.coo_matrix((K.ravel(), (rows, cols)), shape=(3 * self.n, 3 * self.n)).tocsr()
        if self.dynamic:
            H = H + sp.diags(np.repeat(self.mass, 3))
        H.sum_duplicates()
        return H.tocsr()

    def free_gradient_norm(self, g):
        return float(np.linalg.norm(g[self.free]))

    def free_hessian(self, H):
        return H[self.free_dofs][:, self.free_dofs]

    def total_volume(self) -> float:
        return float(self.vol.sum())


def problem_from_scene(scene, kind: str = "snh") -> Problem:
    """Build a :class:`Problem` from a ``meshgen.Scene``."""
    m = scene.material
    return Problem(scene.X, scene.tets, scene.pinned, Model(kind, m.E, m.nu), rho=m.rho,
                   h=scene.h, gravity=scene.gravity)
