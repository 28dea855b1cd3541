"""Energy densities Psi(F) and their derivatives, vectorised over tets.

The paper's elastic potential Psi in Eq. 2 is left generic (it uses Fixed
Corotational elasticity, Sec. 4.1).  This build uses the stable Neo-Hookean
density in its rest-stable form without the logarithmic term:

    Psi(F) = mu/2 (tr(F^T F) - 3) - mu (J - 1) + lam_hat/2 (J - 1)^2,
    J = det F,  mu = E / (2 (1 + nu)),  lam = E nu / ((1 + nu)(1 - 2 nu)),
    lam_hat = lam + mu,

for which the linearisation at F = I is Hooke's law with (E, nu).
Derivatives (C = cof F = dJ/dF):

    P      = mu F - mu C + lam_hat (J - 1) C
    dP/dF  = mu I_9 + lam_hat vec(C) vec(C)^T + (lam_hat (J - 1) - mu) d2J/dF2

with d2J/dF_ab dF_cd = eps_ace eps_bdf F_ef.  Index convention: F_ab, a = row
(spatial axis), b = column (material axis).

``fcr`` is the paper's Fixed Corotational density (Sec. 4.1),

    Psi(F) = mu ||F - R||_F^2 + lam/2 (J - 1)^2,  F = R S (polar decomposition),
    P      = 2 mu (F - R) + lam (J - 1) C,
    dP[dF] = 2 mu (dF - dR) + lam (C : dF) C + lam (J - 1) d2J/dF2 : dF,

with dR = R [w]_x, (tr(S) I - S) w = axial(R^T dF - dF^T R) (differentiating
F = R S: the skew part of R^T dF is (W S + S W)/2 with W = R^T dR).  Its
linearisation at F = I is Hooke's law with (mu, lam).

``linear`` is the small-strain Hooke density Psi = mu eps:eps + lam/2 tr(eps)^2,
eps = sym(F) - I, used only to build the quadratic problems on which the
paper's single-iteration claim (Sec. 4.3) is exact.
"""
from __future__ import annotations

import numpy as np

# Levi-Civita symbol eps[a, b, c]
EPS = np.zeros((3, 3, 3))
EPS[0, 1, 2] = EPS[1, 2, 0] = EPS[2, 0, 1] = 1.0
EPS[0, 2, 1] = EPS[2, 1, 0] = EPS[1, 0, 2] = -1.0


def lame(E: float, nu: float):
    """Lame parameters (mu, lam) of an isotropic material."""
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam


def snh_params(E: float, nu: float):
    """(mu, lam_hat) with lam_hat = lam + mu (rest-stable, Hooke-consistent)."""
    mu, lam = lame(E, nu)
    return mu, lam + mu


def det3(F: np.ndarray) -> np.ndarray:
    """J = det F for F of shape [..., 3, 3] via J = 1/6 eps_ace eps_bdf F_ab F_cd F_ef."""
    return np.einsum("ace,bdf,...ab,...cd,...ef->...", EPS, EPS, F, F, F, optimize=True) / 6.0


def cofactor(F: np.ndarray) -> np.ndarray:
    """C_ab = dJ/dF_ab = 1/2 eps_ace eps_bdf F_cd F_ef."""
    return 0.5 * np.einsum("ace,bdf,...cd,...ef->...ab", EPS, EPS, F, F, optimize=True)


def det_hessian(F: np.ndarray) -> np.ndarray:
    """d2J/dF_ab dF_cd = eps_ace eps_bdf F_ef, shape [..., 3, 3, 3, 3] (a, b, c, d)."""
    return np.einsum("ace,bdf,...ef->...abcd", EPS, EPS, F, optimize=True)


def snh_energy(F: np.ndarray, mu: float, lam_hat: float) -> np.ndarray:
    J = det3(F)
    I_C = np.einsum("...ab,...ab->...", F, F)
    return 0.5 * mu * (I_C - 3.0) - mu * (J - 1.0) + 0.5 * lam_hat * (J - 1.0) ** 2


def snh_stress(F: np.ndarray, mu: float, lam_hat: float) -> np.ndarray:
    """First Piola-Kirchhoff stress P = dPsi/dF, shape [..., 3, 3]."""
    J = det3(F)
    C = cofactor(F)
    return mu * F - mu * C + (lam_hat * (J - 1.0))[..., None, None] * C


def snh_dstress(F: np.ndarray, mu: float, lam_hat: float) -> np.ndarray:
    """dP_ab/dF_cd, shape [..., 3, 3, 3, 3]."""
    J = det3(F)
    C = cofactor(F)
    eye9 = np.einsum("ac,bd->abcd", np.eye(3), np.eye(3))
    out = mu * eye9 + lam_hat * np.einsum("...ab,...cd->...abcd", C, C)
    out = out + ((lam_hat * (J - 1.0)) - mu)[..., None, None, None, None] * det_hessian(F)
    return out


def polar_rotation(F: np.ndarray) -> np.ndarray:
    """R of F = R S with R a proper rotation, from the SVD F = U diag(s) V^T:
    R = U diag(1, 1, det(U V^T)) V^T (the closest rotation when det F > 0)."""
    U, _, Vt = np.linalg.svd(F)
    d = np.sign(np.linalg.det(U @ Vt))
    D = np.zeros(F.shape[:-2] + (3, 3))
    D[..., 0, 0] = 1.0
    D[..., 1, 1] = 1.0
    D[..., 2, 2] = d
    return U @ D @ Vt


def fcr_energy(F: np.ndarray, mu: float, lam: float) -> np.ndarray:
    R = polar_rotation(F)
    J = det3(F)
    return mu * np.einsum("...ab,...ab->...", F - R, F - R) + 0.5 * lam * (J - 1.0) ** 2


def fcr_stress(F: np.ndarray, mu: float, lam: float) -> np.ndarray:
    R = polar_rotation(F)
    J = det3(F)
    return 2.0 * mu * (F - R) + (lam * (J - 1.0))[..., None, None] * cofactor(F)


def fcr_dstress(F: np.ndarray, mu: float, lam: float) -> np.ndarray:
    """dP_ab/dF_cd, shape [..., 3, 3, 3, 3], one basis direction E_cd at a time."""
    R = polar_rotation(F)
    S = np.swapaxes(R, -1, -2) @ F
    J = det3(F)
    C = cofactor(F)
    K = np.einsum("...aa->...", S)[..., None, None] * np.eye(3) - S
    Kinv = np.linalg.inv(K)
    d2J = det_hessian(F)
    out = np.zeros(F.shape[:-2] + (3, 3, 3, 3))
    for c in range(3):
        for d in range(3):
            E = np.zeros((3, 3))
            E[c, d] = 1.0
            G = np.swapaxes(R, -1, -2) @ E
            A = G - np.swapaxes(G, -1, -2)
            ax = np.stack([A[..., 2, 1], A[..., 0, 2], A[..., 1, 0]], axis=-1)
            w = np.einsum("...ij,...j->...i", Kinv, ax)
            W = np.einsum("ijk,...k->...ij", -EPS, w)      # [w]_x: W v = w x v
            dR = R @ W
            dP = 2.0 * mu * (E - dR) + (lam * C[..., c, d])[..., None, None] * C \
                + (lam * (J - 1.0))[..., None, None] * d2J[..., :, :, c, d]
            out[..., :, :, c, d] = dP
    return out


def linear_energy(F: np.ndarray, mu: float, lam: float) -> np.ndarray:
    eps = 0.5 * (F + np.swapaxes(F, -1, -2)) - np.eye(3)
    tr = np.einsum("...aa->...", eps)
    return mu * np.einsum("...ab,...ab->...", eps, eps) + 0.5 * lam * tr ** 2


def linear_stress(F: np.ndarray, mu: float, lam: float) -> np.ndarray:
    eps = 0.5 * (F + np.swapaxes(F, -1, -2)) - np.eye(3)
    tr = np.einsum("...aa->...", eps)
    return 2.0 * mu * eps + lam * tr[..., None, None] * np.eye(3)


def linear_dstress(F: np.ndarray, mu: float, lam: float) -> np.ndarray:
    # P = mu (F + F^T) - 2 mu I + lam (tr F - 3) I
    I = np.eye(3)
    d = mu * (np.einsum("ac,bd->abcd", I, I) + np.einsum("ad,bc->abcd", I, I)) \
        + lam * np.einsum("ab,cd->abcd", I, I)
    return np.broadcast_to(d, F.shape[:-2] + (3, 3, 3, 3)).copy()


class Model:
    """Energy density with parameters bound: ``kind`` in {"snh", "fcr", "linear"}."""

    def __init__(self, kind: str, E: float, nu: float):
        self.kind, self.E, self.nu = kind, E, nu
        if kind == "snh":
            self.a, self.b = snh_params(E, nu)
        elif kind in ("linear", "fcr"):
            self.a, self.b = lame(E, nu)
        else:
            raise ValueError(kind)

    def energy(self, F):
        return {"snh": snh_energy, "fcr": fcr_energy, "linear": linear_energy}[self.kind](F, self.a, self.b)

    def stress(self, F):
        return {"snh": snh_stress, "fcr": fcr_stress, "linear": linear_stress}[self.kind](F, self.a, self.b)

    def dstress(self, F):
        return {"snh": snh_dstress, "fcr": fcr_dstress, "linear": linear_dstress}[self.kind](F, self.a, self.b)
