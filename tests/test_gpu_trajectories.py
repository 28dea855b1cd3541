"""GPU parity on whole trajectories and on the backward-Euler step.

* A free body under gravity: one backward Euler step through cc_solve_step
  must land on the closed form x1 = x0 + h v0 + h^2 g, v1 = v0 + h g (Eq. 2
  and its footnote; the elastic energy vanishes on translates of the rest
  shape).
* A three-mesh batch: every mesh of cc_solve_batch against the oracle's own
  coloured CC sweeps on that mesh (float64 to 1e-11 of the positions, mixed
  to 1e-5 of the bounding-box diagonal and its residual to 1e-4).
* The 16^3 jittered stretch cube (the 32^3 workload's shape at a size the
  oracle finishes offline): 50 mixed-precision sweeps for E = 1e4 and 1e7
  against the oracle trajectory stored in tests/golden/cube16_trajectory.txt
  (written by make_cube16_trajectory.py from the oracle alone): energy and
  gradient norm within 1e-4 relative at every sweep, sampled final positions
  within 1e-5 of the bounding-box diagonal.
"""
import os

import numpy as np
import pytest

import meshgen
from oracle import fem, material, solvers, subspace, topology

torch = pytest.importorskip("torch")
import paper_2510_12053_gb300 as cc  # noqa: E402

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cube16_trajectory.txt")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_free_body_backward_euler_step_is_ballistic(precision):
    X = meshgen.grid_vertices(3, 2, 2, 0.5)
    tets = meshgen.kuhn_tets(3, 2, 2)
    n = X.shape[0]
    h, g = 1.0 / 60.0, np.array([0.0, -9.8, 0.0])
    v0 = np.broadcast_to([0.3, -0.2, 0.1], (n, 3)).copy()
    x0 = X + np.array([0.1, 0.2, -0.05])
    m = cc.Mesh(X, tets, np.zeros(n, np.uint8), E=1e5, nu=0.3, rho=1000.0, h=h, gravity=g)
    m.color()
    m.build_subspace(2)
    xd, vd = cc.to_soa(x0), cc.to_soa(v0)
    # float64 reaches 1e-12 of the first residual; the mixed path's float-float
    # gradient carries ~1e-10 of it (cancelling stresses near rest)
    r = m.solve_step(xd, vd, precision=precision, tol=1e-12 if precision == "fp64" else 1e-9, max_iters=400)
    assert r.converged
    tol = 1e-12 if precision == "fp64" else 1e-9
    np.testing.assert_allclose(cc.from_soa(xd), x0 + h * v0 + h * h * g, rtol=0, atol=tol)
    np.testing.assert_allclose(cc.from_soa(vd), v0 + h * g, rtol=0, atol=tol / h)
    m.close()


def _batch_scenes():
    a = meshgen.stretch_box(4, 3, 3, E=3e5, nu=0.30, factor=1.3, jitter_amount=0.05, seed=1)
    b = meshgen.stretch_box(3, 3, 3, E=2e6, nu=0.25, factor=1.2, axis=1, seed=2)
    c = meshgen.stretch_box(3, 4, 3, E=5e4, nu=0.30, factor=1.1, jitter_amount=0.05, seed=3, axis=2)
    return [a, b, c]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_meshes_follow_the_oracle(precision):
    scenes = _batch_scenes()
    sweeps = 6
    batch = cc.Mesh.from_scenes(scenes)
    batch.color()
    batch.build_subspace(2)
    off = batch.batch_offsets()
    xd = cc.to_soa(np.concatenate([sc.x0 for sc in scenes]))
    res = batch.solve_batch(xd, precision=precision, tol=0.0, max_iters=sweeps, check_every=1)
    xb = cc.from_soa(xd)
    for k, sc in enumerate(scenes):
        pb = fem.problem_from_scene(sc)
        topo = topology.Topology(pb.n, pb.tets, pb.free)
        sup, U = subspace.build_local_bases(pb, topo, 2)
        x, hist = solvers.solve(pb, topo, sup, U, sc.x0, kind="cc", tol=0.0, max_iters=sweeps)
        assert res["iterations"][k] == sweeps
        assert res["g0"][k] == pytest.approx(hist.grad_norm[0], rel=1e-9 if precision == "fp64" else 1e-5)
        xk = xb[off[k]:off[k + 1]]
        if precision == "fp64":
            np.testing.assert_allclose(xk, x, rtol=0, atol=1e-11 * np.abs(x).max())
            assert res["g_final"][k] == pytest.approx(hist.grad_norm[-1], rel=1e-7)
        else:
            diag = np.linalg.norm(sc.X.max(0) - sc.X.min(0))
            assert np.abs(xk - x).max() <= 1e-5 * diag
            assert res["g_final"][k] == pytest.approx(hist.grad_norm[-1], rel=1e-4)


def _golden():
    runs, cur = [], None
    for line in open(GOLDEN):
        key, _, rest = line.partition(" ")
        if key == "E":
            cur = {"E": float(rest)}
            runs.append(cur)
        elif key in ("energy", "gnorm", "x"):
            cur[key] = np.array([float(v) for v in rest.split()])
        elif key == "sample":
            cur[key] = np.array([int(v) for v in rest.split()])
    return runs


@pytest.mark.parametrize("run", [0, 1], ids=["E1e4", "E1e7"])
def test_cube16_mixed_trajectory_matches_stored_oracle_trajectory(run):
    gold = _golden()[run]
    sc = meshgen.stretch_box(16, 16, 16, E=gold["E"], nu=0.3, factor=1.5, jitter_amount=0.05, seed=0)
    m = cc.Mesh.from_scene(sc)
    m.color()
    m.build_subspace(2)
    xd = cc.to_soa(sc.x0)
    E0, _, g0 = m.energy_grad(xd, precision="fp64", want_grad=False)
    E_g, G_g = [E0], [g0]
    for _ in range(len(gold["energy"]) - 1):
        m.sweep(xd, update="cc", schedule="colored", precision="mixed")
        E, _, gn = m.energy_grad(xd, precision="fp64", want_grad=False)
        E_g.append(E)
        G_g.append(gn)
    E_g, G_g = np.array(E_g), np.array(G_g)
    assert np.max(np.abs(E_g - gold["energy"]) / np.abs(gold["energy"])) <= 1e-4
    assert np.max(np.abs(G_g - gold["gnorm"]) / gold["gnorm"]) <= 1e-4
    diag = np.linalg.norm(sc.X.max(0) - sc.X.min(0))
    xs = cc.from_soa(xd)[gold["sample"]].ravel()
    assert np.abs(xs - gold["x"]).max() <= 1e-5 * diag
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_three_ring_dynamic_cantilever_sweeps_follow_the_oracle(precision):
    """The cantilever workload's method at a size the oracle finishes: 3-ring
    rest bases (M + h^2 K), backward Euler target with gravity, two coloured
    CC sweeps of the first step, against the oracle's own sweeps."""
    scene = meshgen.cantilever(4, 4, 12, cell=1.0 / 64.0, E=1e7, nu=0.45)
    pb = fem.problem_from_scene(scene)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    sup, U = subspace.build_local_bases(pb, topo, 3)
    xt = pb.inertial_target(scene.X, scene.v0)
    x_o = scene.X.copy()
    for _ in range(2):
        x_o = solvers.sweep(pb, topo, sup, U, x_o, xt, "cc", "colored")
    m = cc.Mesh.from_scene(scene)
    m.color()
    m.build_subspace(3)
    assert m.info().support_max > 64
    xd, vd = cc.to_soa(scene.X), cc.to_soa(scene.v0)
    r = m.solve_step(xd, vd, precision=precision, tol=0.0, max_iters=2, min_iters=2)
    assert r.iterations == 2
    step = np.abs(x_o - scene.X).max()
    tol = 1e-9 if precision == "fp64" else 1e-4
    assert np.abs(cc.from_soa(xd) - x_o).max() <= tol * step
    m.close()
