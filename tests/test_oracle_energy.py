"""Pins of the oracle's energy, gradient and Hessian (Eq. 2) against
finite differences, invariants and the textbook linear-elastic stiffness."""
import numpy as np
import pytest

import meshgen
from oracle import fem, material


def _rotation(seed):
    A = meshgen.normal(seed, np.arange(9)).reshape(3, 3)
    Q, R = np.linalg.qr(A)
    Q = Q @ np.diag(np.sign(np.diag(R)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


def _perturbed(scene, amp, seed):
    n = scene.n
    d = meshgen.normal(seed, np.arange(3 * n)).reshape(n, 3) * amp * scene.cell
    return scene.x0 + d * (scene.pinned == 0)[:, None]


@pytest.fixture(scope="module")
def small():
    return meshgen.stretch_box(2, 2, 3, E=1e5, nu=0.45, factor=1.3, jitter_amount=0.05, seed=7)


@pytest.mark.parametrize("kind", ["snh", "fcr", "linear"])
@pytest.mark.parametrize("dynamic", [False, True])
def test_gradient_matches_central_differences(small, kind, dynamic):
    pb = fem.problem_from_scene(small, kind)
    xt = None
    if dynamic:
        pb = fem.Problem(small.X, small.tets, small.pinned, material.Model(kind, 1e5, 0.45), rho=1000.0,
                         h=0.01, gravity=[0.0, -9.8, 0.0])
        v = meshgen.normal(11, np.arange(3 * small.n)).reshape(-1, 3)
        xt = pb.inertial_target(small.x0, v)
    x = _perturbed(small, 0.2, 3)
    g = pb.gradient(x, xt)
    eps = 1e-6 * small.cell
    gfd = np.zeros_like(x)
    for v in range(small.n):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, a] += eps
            xm[v, a] -= eps
            gfd[v, a] = (pb.energy(xp, xt) - pb.energy(xm, xt)) / (2 * eps)
    assert np.linalg.norm(gfd - g) <= 1e-6 * np.linalg.norm(g)


@pytest.mark.parametrize("kind", ["snh", "fcr", "linear"])
def test_hessian_matches_central_differences(small, kind):
    pb = fem.problem_from_scene(small, kind)
    x = _perturbed(small, 0.2, 4)
    H = pb.hessian(x).toarray()
    eps = 1e-6 * small.cell
    Hfd = np.zeros_like(H)
    for v in range(small.n):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[v, a] += eps
            xm[v, a] -= eps
            Hfd[:, 3 * v + a] = ((pb.gradient(xp) - pb.gradient(xm)) / (2 * eps)).ravel()
    assert np.linalg.norm(Hfd - H) <= 1e-6 * np.linalg.norm(H)
    assert np.allclose(H, H.T, rtol=0, atol=1e-9 * np.abs(H).max())


@pytest.mark.parametrize("kind", ["snh", "fcr"])
def test_zero_energy_and_gradient_at_rest(small, kind):
    pb = fem.problem_from_scene(small, kind)
    assert abs(pb.energy(small.X)) <= 1e-12 * small.material.E * pb.total_volume()
    g = pb.gradient(small.X)
    assert np.abs(g).max() <= 1e-10 * small.material.E * small.cell ** 2


@pytest.mark.parametrize("kind", ["snh", "fcr"])
def test_rotation_and_translation_invariance(small, kind):
    pb = fem.problem_from_scene(small, kind)
    x = _perturbed(small, 0.3, 5)
    R = _rotation(9)
    t = np.array([0.3, -1.2, 2.0])
    y = x @ R.T + t
    assert pb.energy(y) == pytest.approx(pb.energy(x), rel=1e-12)
    np.testing.assert_allclose(pb.gradient(y), pb.gradient(x) @ R.T, rtol=0,
                               atol=1e-9 * np.abs(pb.gradient(x)).max())


@pytest.mark.parametrize("kind", ["snh", "fcr"])
def test_rest_hessian_is_textbook_linear_elastic_stiffness(kind):
    """V B^T D B with B built from barycentric shape gradients (4x4 inverse)
    and D the isotropic Voigt matrix of (E, nu): pins lam_hat = lam + mu for
    stable Neo-Hookean and (mu, lam) for Fixed Corotational."""
    E, nu = 3.7e5, 0.41
    X = np.array([[0.0, 0.0, 0.0], [1.1, 0.1, 0.0], [0.2, 0.9, 0.1], [0.1, 0.2, 1.3]])
    tets = np.array([[0, 1, 2, 3]])
    pb = fem.Problem(X, tets, np.zeros(4), material.Model(kind, E, nu))
    M = np.hstack([np.ones((4, 1)), X])
    C = np.linalg.inv(M)            # N_v(X) = sum_k C[k, v] [1, X]_k
    grads = C[1:, :].T              # [4, 3]
    V = abs(np.linalg.det(M)) / 6.0
    B = np.zeros((6, 12))
    for v in range(4):
        nx, ny, nz = grads[v]
        B[:, 3 * v:3 * v + 3] = [[nx, 0, 0], [0, ny, 0], [0, 0, nz], [0, nz, ny], [nz, 0, nx], [ny, nx, 0]]
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] = lam + 2 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    K_book = V * B.T @ D @ B
    K = pb.hessian(X).toarray()
    np.testing.assert_allclose(K, K_book, rtol=0, atol=1e-10 * np.abs(K_book).max())


def test_diagonal_vertex_blocks_spd_far_from_rest(small):
    pb = fem.problem_from_scene(small)
    x = _perturbed(small, 1.5, 6)   # large random deformation, inverted tets likely
    H = pb.hessian(x)
    for v in range(small.n):
        blk = H[3 * v:3 * v + 3][:, 3 * v:3 * v + 3].toarray()
        assert np.linalg.eigvalsh(blk).min() > 0


def test_cofactor_and_determinant_match_linear_algebra():
    F = meshgen.normal(2, np.arange(45)).reshape(5, 3, 3)
    np.testing.assert_allclose(material.det3(F), np.linalg.det(F), rtol=1e-12)
    cof = np.linalg.det(F)[:, None, None] * np.linalg.inv(F).transpose(0, 2, 1)
    np.testing.assert_allclose(material.cofactor(F), cof, rtol=1e-10, atol=1e-12)


def test_mass_and_volume(small):
    pb = fem.problem_from_scene(small)
    nx, ny, nz = small.dims
    box = nx * ny * nz * small.cell ** 3
    assert pb.total_volume() == pytest.approx(box, rel=1e-12)
    assert pb.mass.sum() == pytest.approx(small.material.rho * box, rel=1e-12)
    assert np.all(pb.vol > 0)


def test_mesh_counts_match_workload_definitions():
    rows = [list(map(int, l.split())) for l in open(
        __file__.replace("test_oracle_energy.py", "golden/mesh_counts.txt")) if l.strip() and l[0] != "#"]
    for nx, ny, nz, nv, nt in rows:
        X = meshgen.grid_vertices(nx, ny, nz)
        T = meshgen.kuhn_tets(nx, ny, nz)
        assert X.shape[0] == nv and T.shape[0] == nt
        assert T.min() == 0 and T.max() == nv - 1      # every vertex is a corner of some tet


def test_polar_rotation_matches_scipy_and_is_proper():
    from scipy.linalg import polar
    F = np.stack([np.eye(3) + 0.4 * meshgen.normal(20 + k, np.arange(9)).reshape(3, 3) for k in range(20)])
    F = F[np.linalg.det(F) > 0]
    R = material.polar_rotation(F)
    for Fk, Rk in zip(F, R):
        np.testing.assert_allclose(Rk, polar(Fk)[0], rtol=0, atol=1e-12)
        assert np.linalg.det(Rk) == pytest.approx(1.0, abs=1e-12)
    Q = _rotation(4)
    S = np.array([[1.3, 0.1, 0.0], [0.1, 0.9, 0.2], [0.0, 0.2, 1.1]])
    np.testing.assert_allclose(material.polar_rotation(Q @ S), Q, rtol=0, atol=1e-12)


def test_fcr_energy_closed_forms():
    """Psi(R S) = mu |S - I|^2 + lam/2 (det S - 1)^2, independent of R."""
    mu, lam = material.lame(2e5, 0.35)
    S = np.array([[1.2, 0.05, 0.0], [0.05, 0.8, 0.1], [0.0, 0.1, 1.05]])
    Q = _rotation(6)
    want = mu * np.sum((S - np.eye(3)) ** 2) + 0.5 * lam * (np.linalg.det(S) - 1.0) ** 2
    assert material.fcr_energy(Q @ S, mu, lam) == pytest.approx(want, rel=1e-13)
    assert material.fcr_energy(Q, mu, lam) == pytest.approx(0.0, abs=1e-20)
