"""Pins of the oracle's perturbation bases (Eq. 4-5), local updates (Eq. 3, 7,
9-12) and solvers against brute force, closed forms and the paper's claims."""
import numpy as np
import pytest

import meshgen
from oracle import fem, material, solvers, subspace, topology


def _setup(n=3, kind="snh", nu=0.3, factor=1.05, jit=0.05, seed=1):
    sc = meshgen.stretch_box(n, n, n, E=1e5, nu=nu, factor=factor, jitter_amount=jit, seed=seed)
    pb = fem.problem_from_scene(sc, kind)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    return sc, pb, topo


def _state(sc, amp=0.01, seed=3):
    d = meshgen.normal(seed, np.arange(3 * sc.n)).reshape(-1, 3) * amp
    return sc.x0 + d * (sc.pinned == 0)[:, None]


def test_global_basis_two_constructions_agree():
    sc, pb, topo = _setup()
    H = pb.hessian(sc.X)
    for i in np.flatnonzero(pb.free)[:4]:
        S1, U1 = subspace.global_basis(pb, H, int(i))
        S2, U2 = subspace.global_basis_inverse(pb, H, int(i))
        np.testing.assert_array_equal(S1, S2)
        np.testing.assert_allclose(U1, U2, rtol=0, atol=1e-10 * np.abs(U1).max())


def test_basis_solves_block_system_with_zero_complementary_force():
    """Eq. 4: [H_ii H_iC; H_Ci H_CC][I; U] = [df; 0], and df = (W_ii)^{-1}."""
    sc, pb, topo = _setup()
    H = pb.hessian(sc.X).toarray()
    F = np.flatnonzero(pb.free)
    Fd = subspace.dofs(F)
    W = np.linalg.inv(H[np.ix_(Fd, Fd)])
    for p, i in enumerate(F[:3]):
        S, U = subspace.global_basis(pb, pb.hessian(sc.X), int(i))
        I, C = subspace.dofs([i]), subspace.dofs(S)
        Uf = U.reshape(-1, 3)
        lower = H[np.ix_(C, I)] + H[np.ix_(C, C)] @ Uf
        assert np.abs(lower).max() <= 1e-9 * np.abs(H).max()
        df = H[np.ix_(I, I)] + H[np.ix_(I, C)] @ Uf
        np.testing.assert_allclose(df, np.linalg.inv(W[3 * p:3 * p + 3, 3 * p:3 * p + 3]), rtol=1e-8)


def test_local_basis_residual_and_full_ring_equals_global():
    sc, pb, topo = _setup(n=2)
    H = pb.hessian(sc.X)
    sup, bases = subspace.build_local_bases(pb, topo, k=6)   # k >= diameter: whole mesh
    for i in np.flatnonzero(pb.free):
        S, U = subspace.global_basis(pb, H, int(i))
        np.testing.assert_array_equal(sup[i], S)
        np.testing.assert_allclose(bases[i], U, rtol=0, atol=1e-10 * max(1.0, np.abs(U).max()))
    sup2, bases2 = subspace.build_local_bases(pb, topo, k=1)
    for i in np.flatnonzero(pb.free):
        P = subspace.dofs(sup2[i])
        if len(P):
            r = H[P][:, P].toarray() @ bases2[i].reshape(-1, 3) + H[P][:, subspace.dofs([i])].toarray()
            assert np.abs(r).max() <= 1e-9 * abs(H).max()


def test_cc_update_is_first_block_of_the_reduced_block_system():
    """Eq. 9-12 against a direct solve of Eq. 10 with an explicit dense B_i."""
    sc, pb, topo = _setup(n=3, factor=1.2)
    x = _state(sc, 0.02)
    sup, bases = subspace.build_local_bases(pb, topo, 1)
    H = pb.hessian(x).toarray()
    g = pb.gradient(x)
    Hs = pb.hessian(x)
    for i in np.flatnonzero(pb.free)[::3]:
        B = np.zeros((3 * pb.n, 6))
        B[3 * i:3 * i + 3, :3] = np.eye(3)
        for s, j in enumerate(sup[i]):
            B[3 * j:3 * j + 3, 3:] = bases[i][s]
        q = np.linalg.solve(B.T @ H @ B, -B.T @ g.ravel())
        dx = solvers.local_update("cc", Hs, g, int(i), sup[i], bases[i])
        np.testing.assert_allclose(dx, q[:3], rtol=1e-9, atol=1e-14)


def test_jgs2_and_cd_updates_match_their_formulas():
    sc, pb, topo = _setup(n=3, factor=1.2)
    x = _state(sc, 0.02)
    sup, bases = subspace.build_local_bases(pb, topo, 1)
    H = pb.hessian(x).toarray()
    g = pb.gradient(x)
    for i in np.flatnonzero(pb.free)[::4]:
        I, P = subspace.dofs([i]), subspace.dofs(sup[i])
        Uf = bases[i].reshape(-1, 3)
        M = H[np.ix_(I, I)] + Uf.T @ H[np.ix_(P, P)] @ Uf
        rhs = g[i] + Uf.T @ g.ravel()[P]
        np.testing.assert_allclose(solvers.local_update("jgs2", pb.hessian(x), g, int(i), sup[i], bases[i]),
                                   -np.linalg.solve(M, rhs), rtol=1e-9)
        np.testing.assert_allclose(solvers.local_update("cd", pb.hessian(x), g, int(i), sup[i], bases[i]),
                                   -np.linalg.solve(H[np.ix_(I, I)], g[i]), rtol=1e-12)


def test_exact_current_basis_cc_jacobi_step_equals_newton_step():
    """With untruncated bases built at the current x, S is the exact Schur
    complement and the Jacobi CC direction is the Newton direction."""
    sc, pb, topo = _setup(n=3, factor=1.05)
    x = _state(sc, 0.01)
    assert np.linalg.eigvalsh(pb.free_hessian(pb.hessian(x)).toarray()).min() > 0
    sup, bases = subspace.all_global_bases(pb, x)
    st = solvers.Stats()
    d_cc = solvers.jacobi_direction(pb, sup, bases, x, None, "cc", st)
    d_nt = solvers.newton_direction(pb, x)
    assert st.fallback_empty + st.fallback_reduced + st.fallback_schur == 0
    assert np.abs(d_cc - d_nt).max() <= 1e-10 * np.abs(d_nt).max()
    # JGS2 "strictly adds stiffness" (Sec. 3.1): H_ii + Ht - H_ii is PSD; CC deflates it
    H = pb.hessian(x)
    g = pb.gradient(x)
    for i in np.flatnonzero(pb.free)[:5]:
        H_ii, g_i, A, Ht, b = solvers.local_terms(H, g, int(i), sup[i], bases[i])
        assert np.linalg.eigvalsh(Ht).min() > 0
        S = A @ np.linalg.solve(Ht, A.T)
        assert np.linalg.eigvalsh(S).min() > -1e-9 * np.abs(S).max()


@pytest.mark.parametrize("schedule", ["jacobi", "colored"])
def test_quadratic_problem_converges_in_one_iteration_with_exact_rest_basis(schedule):
    """Sec. 4.3: for a quadratic energy and the rest-shape basis the Schur
    complement is the exact global response: a single iteration solves it."""
    sc, pb, topo = _setup(n=3, kind="linear", nu=0.45, factor=1.5)
    sup, bases = subspace.all_global_bases(pb)
    x, hist = solvers.solve(pb, topo, sup, bases, sc.x0, kind="cc", schedule=schedule, max_iters=1)
    assert hist.iterations == 1
    assert hist.rel[-1] <= 1e-10
    xn, hn = solvers.newton(pb, sc.x0, tol=1e-13)
    np.testing.assert_allclose(x, xn, rtol=0, atol=1e-10)


def test_one_free_vertex_cc_equals_cd_equals_newton():
    sc = meshgen.stretch_box(2, 2, 2, E=1e5, nu=0.45, factor=1.3)
    pinned = np.ones(sc.n, dtype=np.uint8)
    centre = 1 + 3 * (1 + 3 * 1)
    pinned[centre] = 0
    pb = fem.Problem(sc.X, sc.tets, pinned, material.Model("snh", 1e5, 0.45))
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    x = sc.x0.copy()
    x[centre] += [0.05, -0.02, 0.03]
    sup, bases = subspace.build_local_bases(pb, topo, 2)
    assert len(sup[centre]) == 0
    st = solvers.Stats()
    d_cc = solvers.jacobi_direction(pb, sup, bases, x, None, "cc", st)
    d_cd = solvers.jacobi_direction(pb, sup, bases, x, None, "cd")
    d_nt = solvers.newton_direction(pb, x)
    assert st.fallback_empty == 1
    np.testing.assert_allclose(d_cc, d_cd, rtol=0, atol=1e-15)
    np.testing.assert_allclose(d_cc, d_nt, rtol=1e-10, atol=1e-15)


def test_newton_converges_quadratically_on_stretch():
    sc = meshgen.stretch_box(4, 4, 4, E=1e5, nu=0.45, factor=1.5)
    pb = fem.problem_from_scene(sc)
    x, hist = solvers.newton(pb, sc.x0, tol=1e-12, max_iters=30)
    assert hist.converged
    g = hist.grad_norm
    tail = [k for k in range(1, len(g)) if g[k - 1] < 1e-2 * g[0]]
    assert len(tail) >= 2
    # ||g_{k+1}|| <= K ||g_k||^2 in the last iterations (quadratic convergence)
    K = max(g[k] / g[k - 1] ** 2 for k in tail if g[k] > 1e-14 * g[0])
    assert K * g[tail[0] - 1] < 0.5


def test_coloured_cc_beats_coloured_cd_on_compressible_stretch():
    """The paper's central claim (Sec. 4.2-4.3), checked qualitatively on a
    3D stretch with the truncated 2-ring basis at nu = 0.3."""
    sc, pb, topo = _setup(n=4, nu=0.3, factor=1.2, jit=0.0)
    sup, bases = subspace.build_local_bases(pb, topo, 2)
    _, h_cc = solvers.solve(pb, topo, sup, bases, sc.x0, kind="cc", schedule="colored", max_iters=12, tol=0)
    _, h_cd = solvers.solve(pb, topo, sup, bases, sc.x0, kind="cd", schedule="colored", max_iters=12, tol=0)
    assert h_cc.rel[-1] < 0.1 * h_cd.rel[-1]


def test_spd_guard_agrees_with_eigenvalues():
    for s in range(40):
        A = meshgen.normal(100 + s, np.arange(9)).reshape(3, 3)
        M = A @ A.T - (s % 3) * 0.7 * np.eye(3)
        ev = np.linalg.eigvalsh(M)
        if ev.min() > 1e-6 * ev.max():
            assert solvers.spd_ok(M)
        if ev.min() < -1e-6 * abs(ev).max():
            assert not solvers.spd_ok(M)


def test_backtracking_line_search_decreases_energy():
    sc, pb, topo = _setup(n=3, nu=0.45, factor=1.5, jit=0.0)
    sup, bases = subspace.build_local_bases(pb, topo, 2)
    d = solvers.jacobi_direction(pb, sup, bases, sc.x0, None, "cc")
    a = solvers.backtracking(pb, sc.x0, d)
    assert 0 < a <= 1
    assert pb.energy(sc.x0 + a * d) < pb.energy(sc.x0)


def test_normalized_residual_of_a_uniformly_stretched_tet_in_closed_form():
    """Sec. 4.1's termination value ||g|| / (V n E) (divided by h for dynamics)
    on the unit corner tet (D_m = I, V = 1/6, n = 4) stretched to F = diag(s, 1, 1).
    By hand: cof F = diag(1, s, s), J = s, so the stable Neo-Hookean stress is
    P = diag((mu + lam_hat)(s - 1), (s - 1)(lam_hat s - mu), (s - 1)(lam_hat s - mu));
    the corner gradients are V P e_1, V P e_2, V P e_3 and minus their sum, hence
    ||g||^2 = 2 V^2 (P_00^2 + 2 P_11^2)."""
    E, nu, s = 1e5, 0.3, 1.2
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    mu = E / (2 * (1 + nu))
    lam_hat = E * nu / ((1 + nu) * (1 - 2 * nu)) + mu
    P00, P11 = (mu + lam_hat) * (s - 1), (s - 1) * (lam_hat * s - mu)
    g_closed = np.sqrt(2 * (P00 ** 2 + 2 * P11 ** 2)) / 6
    expect = g_closed / ((1 / 6) * 4 * E)
    x = X * np.array([s, 1.0, 1.0])
    pb = fem.Problem(X, np.array([[0, 1, 2, 3]]), np.zeros(4, np.uint8), material.Model("snh", E, nu))
    g = pb.free_gradient_norm(pb.gradient(x))
    assert g == pytest.approx(g_closed, rel=1e-13)
    assert solvers.normalized_residual(pb, g) == pytest.approx(expect, rel=1e-13)
    h = 0.01
    pbd = fem.Problem(X, np.array([[0, 1, 2, 3]]), np.zeros(4, np.uint8), material.Model("snh", E, nu), h=h)
    assert solvers.normalized_residual(pbd, g) == pytest.approx(expect / h, rel=1e-13)


def test_backward_euler_step_of_a_free_body_is_ballistic():
    """Eq. 2 and its footnote on a body with no pinned vertex, starting at a
    translate of its rest shape with one velocity v0 everywhere, under gravity
    g: the elastic energy vanishes on every translate of the rest shape, so the
    minimiser of Eq. 2 is the inertial target itself and one backward Euler
    step must give exactly x1 = x0 + h v0 + h^2 g and v1 = v0 + h g (free fall).
    A target with h instead of h^2, a flipped gravity or a velocity divided by
    h^2 all fail here."""
    X = meshgen.grid_vertices(2, 2, 2, 0.5)
    tets = meshgen.kuhn_tets(2, 2, 2)
    n = X.shape[0]
    h, g = 1.0 / 60.0, np.array([0.0, -9.8, 0.0])
    v0 = np.broadcast_to([0.3, -0.2, 0.1], (n, 3)).copy()
    x0 = X + np.array([0.1, 0.2, -0.05])
    pb = fem.Problem(X, tets, np.zeros(n, np.uint8), material.Model("snh", 1e5, 0.3), rho=1000.0, h=h, gravity=g)
    np.testing.assert_allclose(pb.inertial_target(x0, v0), x0 + h * v0 + h * h * g, rtol=0, atol=1e-15)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    sup, U = subspace.build_local_bases(pb, topo, 2)
    for kind in ("cc", "cd"):
        x1, v1, hist = solvers.time_step(pb, topo, sup, U, x0, v0, kind=kind, tol=1e-13, max_iters=400)
        assert hist.converged, kind
        np.testing.assert_allclose(x1, x0 + h * v0 + h * h * g, rtol=0, atol=1e-13)
        np.testing.assert_allclose(v1, v0 + h * g, rtol=0, atol=1e-11)


# ---------------------------------------------------------------- corotated bases (Sec. 3.1)
def _rot(axis, ang):
    from scipy.spatial.transform import Rotation
    return Rotation.from_rotvec(np.asarray(axis, dtype=float) / np.linalg.norm(axis) * ang).as_matrix()


def test_vertex_rotations_closed_forms():
    sc, pb, topo = _setup(n=3, jit=0.05)
    Q = _rot([1.0, 2.0, -0.5], 0.7)
    R = solvers.vertex_rotations(pb, topo, pb.X @ Q.T + np.array([0.3, -1.0, 2.0]))
    np.testing.assert_allclose(R, np.broadcast_to(Q, R.shape), rtol=0, atol=1e-12)   # rigid motion -> Q
    S = np.diag([1.5, 0.8, 1.1])
    R = solvers.vertex_rotations(pb, topo, pb.X @ S)                                  # pure stretch -> I
    np.testing.assert_allclose(R, np.broadcast_to(np.eye(3), R.shape), rtol=0, atol=1e-12)
    R = solvers.vertex_rotations(pb, topo, _state(sc, 0.02, 5))
    for Rj in R:
        np.testing.assert_allclose(Rj @ Rj.T, np.eye(3), rtol=0, atol=1e-12)
        assert np.linalg.det(Rj) == pytest.approx(1.0, abs=1e-12)
    R = solvers.vertex_rotations(pb, topo, -pb.X)                                    # inverted: det A < 0 -> I
    np.testing.assert_allclose(R, np.broadcast_to(np.eye(3), R.shape), rtol=0, atol=0)


def test_corotated_sweep_is_equivariant_under_rigid_rotation():
    """E(Qx) = E(x), g(Qx) = Q g, H(Qx) = Q H Q^T and R_j(Qx) = Q R_j(x), so the
    rotated bases carry Q and the corotated sweep commutes with Q; the fixed
    rest bases do not."""
    sc, pb, topo = _setup(n=3, jit=0.05, factor=1.2)
    sup, U = subspace.build_local_bases(pb, topo, 2)
    x = _state(sc, 0.02, 7)
    Q = _rot([0.3, -1.0, 0.4], 1.1)
    xr = solvers.sweep(pb, topo, sup, U, x, kind="cc", corotated=True)
    xq = solvers.sweep(pb, topo, sup, U, x @ Q.T, kind="cc", corotated=True)
    np.testing.assert_allclose(xq, xr @ Q.T, rtol=0, atol=1e-10 * np.abs(xr).max())
    xf = solvers.sweep(pb, topo, sup, U, x, kind="cc")
    xfq = solvers.sweep(pb, topo, sup, U, x @ Q.T, kind="cc")
    assert np.abs(xfq - xf @ Q.T).max() > 1e-6 * np.abs(xf - x).max()


def test_corotated_equals_fixed_when_nothing_rotates():
    sc, pb, topo = _setup(n=3, jit=0.05, factor=1.2)
    sup, U = subspace.build_local_bases(pb, topo, 2)
    x = pb.X @ np.diag([1.2, 1.0, 1.0])   # a pure stretch of the rest shape: every R_j = I
    a = solvers.sweep(pb, topo, sup, U, x, kind="cc", corotated=True)
    b = solvers.sweep(pb, topo, sup, U, x, kind="cc")
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13 * np.abs(b).max())


def test_corotated_bases_help_a_twisted_bar():
    sc = meshgen.twist_box(2, 2, 6, angle=np.pi / 2, nu=0.3)
    pb = fem.problem_from_scene(sc)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    sup, U = subspace.build_local_bases(pb, topo, 2)
    _, hf = solvers.solve(pb, topo, sup, U, sc.x0, kind="cc", tol=1e-4, max_iters=80)
    _, hr = solvers.solve(pb, topo, sup, U, sc.x0, kind="cc", tol=1e-4, max_iters=80, corotated=True)
    assert hr.converged and hr.iterations < hf.iterations


def test_global_line_search_never_increases_the_energy():
    """Sec. 4.4: with backtracking on the accumulated direction the energy is
    non-increasing, here on a nearly incompressible stretch where plain
    coloured CC blows up within a few sweeps."""
    sc = meshgen.stretch_box(4, 3, 3, E=1e5, nu=0.45, factor=1.5, jitter_amount=0.05, seed=2)
    pb = fem.problem_from_scene(sc)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    sup, U = subspace.build_local_bases(pb, topo, 2)
    for schedule in ("colored", "jacobi"):
        _, h = solvers.solve(pb, topo, sup, U, sc.x0, kind="cc", schedule=schedule, tol=1e-12, max_iters=8,
                             line_search=True)
        assert all(b <= a for a, b in zip(h.energy, h.energy[1:])), schedule
    _, hp = solvers.solve(pb, topo, sup, U, sc.x0, kind="cc", tol=1e-12, max_iters=8)
    assert max(hp.energy) > hp.energy[0]


# ---------------------------------------------------------------- restarted bases (Sec. 4.4)
def test_rebuilt_bases_at_rest_equal_the_rest_bases_and_solve_eq5_at_x():
    sc, pb, topo = _setup(n=3, jit=0.05, factor=1.3)
    sup, U = subspace.build_local_bases(pb, topo, 2)
    same, kept = subspace.rebuild_bases_at(pb, sup, [np.zeros_like(u) for u in U], pb.X)
    assert kept == 0
    for a, b in zip(same, U):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * max(1.0, np.abs(b).max() if b.size else 1.0))
    x = _state(sc, 0.03, 9)
    Ux, kept = subspace.rebuild_bases_at(pb, sup, U, x)
    H = pb.hessian(x)
    for i in np.flatnonzero(pb.free)[:6]:      # Eq. 5 at x: H_PP U + H_Pi = 0
        P, I = subspace.dofs(sup[i]), subspace.dofs([int(i)])
        R = H[P][:, P] @ Ux[i].reshape(-1, 3) + H[P][:, I].toarray()
        assert np.abs(R).max() <= 1e-9 * np.abs(H[P][:, I].toarray()).max()


def test_restarted_bases_help_the_twisted_bar():
    sc = meshgen.twist_box(2, 2, 6, angle=np.pi / 2, nu=0.3)
    pb = fem.problem_from_scene(sc)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    sup, U = subspace.build_local_bases(pb, topo, 2)
    _, hf = solvers.solve(pb, topo, sup, U, sc.x0, kind="cc", tol=1e-4, max_iters=80)
    _, hr = solvers.solve(pb, topo, sup, U, sc.x0, kind="cc", tol=1e-4, max_iters=80, restart_every=5)
    assert hr.converged and hr.iterations < hf.iterations


def test_stored_cube16_trajectory_is_the_oracles():
    """The fixture the GPU trajectory test compares against
    (tests/golden/cube16_trajectory.txt, written by make_cube16_trajectory.py)
    starts where the oracle starts: its first sweep's energy and gradient norm
    are recomputed here from the oracle."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cube16_trajectory.txt")
    rows = {}
    E = None
    for line in open(path):
        key, _, rest = line.partition(" ")
        if key == "E":
            E = float(rest)
        elif key in ("energy", "gnorm") and E == 1e4:
            rows[key] = np.array([float(v) for v in rest.split()])
    sc = meshgen.stretch_box(16, 16, 16, E=1e4, nu=0.3, factor=1.5, jitter_amount=0.05, seed=0)
    pb = fem.problem_from_scene(sc)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    sup, U = subspace.build_local_bases(pb, topo, 2)
    x, hist = solvers.solve(pb, topo, sup, U, sc.x0, kind="cc", tol=0.0, max_iters=1)
    assert len(rows["energy"]) == 51 and len(rows["gnorm"]) == 51
    np.testing.assert_allclose(hist.energy, rows["energy"][:2], rtol=1e-13)
    np.testing.assert_allclose(hist.grad_norm, rows["gnorm"][:2], rtol=1e-12)
