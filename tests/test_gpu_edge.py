"""Degenerate inputs on the GPU, against the FP64 oracle: a single free
vertex (its support is empty, so CC falls back to the vertex's own Newton
step, which is also what CD does), a single tet, and the inputs the boundary
rejects (no free vertex, too few vertices, a vertex id out of range, an empty
colour range)."""
import dataclasses

import numpy as np
import pytest

import meshgen
from oracle import fem, solvers, subspace, topology

torch = pytest.importorskip("torch")
import paper_2510_12053_gb300 as cc  # noqa: E402

pytestmark = pytest.mark.gpu


def _with_free(scene, free_ids):
    pinned = np.ones(scene.n, dtype=np.uint8)
    pinned[list(free_ids)] = 0
    return dataclasses.replace(scene, pinned=pinned)


def _oracle(scene, k):
    pb = fem.problem_from_scene(scene)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    sup, U = subspace.build_local_bases(pb, topo, k)
    return pb, topo, sup, U


def _perturbed(scene, amp=0.08, seed=4):
    d = meshgen.normal(seed, np.arange(3 * scene.n)).reshape(-1, 3) * amp * scene.cell
    return scene.x0 + d * (scene.pinned == 0)[:, None]


def test_mesh_without_free_vertex_is_rejected():
    """Nothing to solve: the boundary says so instead of building empty state."""
    scene = _with_free(meshgen.stretch_box(2, 2, 2, E=1e5, nu=0.3, factor=1.2), [])
    with pytest.raises(cc.CCError) as e:
        cc.Mesh.from_scene(scene)
    assert e.value.status == cc.ERR_INVALID_ARG


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_single_free_vertex_takes_its_newton_step(precision):
    base = meshgen.stretch_box(2, 2, 2, E=1e5, nu=0.3, factor=1.2)
    centre = int(np.argmin(np.linalg.norm(base.X - base.X.mean(axis=0), axis=1)))
    scene = _with_free(base, [centre])
    pb, topo, sup, U = _oracle(scene, 2)
    assert len(sup[centre]) == 0
    x0 = _perturbed(scene)
    x_cc = solvers.sweep(pb, topo, sup, U, x0, None, "cc", "colored")
    x_cd = solvers.sweep(pb, topo, sup, U, x0, None, "cd", "colored")
    np.testing.assert_allclose(x_cc, x_cd, rtol=0, atol=1e-15)
    m = cc.Mesh.from_scene(scene)
    m.color()
    m.build_subspace(2)
    xd = cc.to_soa(x0)
    st = m.sweep(xd, update="cc", precision=precision)
    assert (st.updates, st.fallback_empty) == (1, 1)
    d_o, d_g = x_cc - x0, cc.from_soa(xd) - x0
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert np.abs(d_g - d_o).max() <= tol * np.abs(d_o).max()


def test_single_tet_mesh():
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    tets = np.array([[0, 1, 2, 3]], dtype=np.int32)
    pinned = np.array([1, 1, 1, 0], dtype=np.uint8)
    x0 = X.copy()
    x0[3] = [0.1, -0.05, 1.3]
    scene = meshgen.Scene(name="tet", X=X, tets=tets, pinned=pinned, x0=x0,
                          material=meshgen.Material(E=1e5, nu=0.3, rho=1000.0))
    pb, topo, sup, U = _oracle(scene, 1)
    x_o = solvers.sweep(pb, topo, sup, U, x0, None, "cc", "colored")
    m = cc.Mesh.from_scene(scene)
    m.color()
    m.build_subspace(1)
    assert m.info().num_colors == 4
    xd = cc.to_soa(x0)
    m.sweep(xd, update="cc", precision="fp64")
    assert np.abs(cc.from_soa(xd) - x_o).max() <= 1e-12 * np.abs(x_o - x0).max()


def test_boundary_rejects_degenerate_inputs():
    scene = meshgen.stretch_box(2, 2, 2, E=1e5, nu=0.3, factor=1.2)
    with pytest.raises(cc.CCError) as e:                      # fewer than four vertices
        cc.Mesh(scene.X[:3], scene.tets[:0], scene.pinned[:3], E=1e5, nu=0.3)
    assert e.value.status == cc.ERR_INVALID_ARG
    bad = scene.tets.copy()
    bad[0, 0] = scene.n                                       # vertex id out of range
    with pytest.raises(cc.CCError) as e:
        cc.Mesh(scene.X, bad, scene.pinned, E=1e5, nu=0.3)
    assert e.value.status == cc.ERR_INVALID_ARG
    m = cc.Mesh.from_scene(scene)
    m.color()
    m.build_subspace(2)
    k = m.info().num_colors
    with pytest.raises(cc.CCError) as e:                      # empty colour range
        m.sweep(cc.to_soa(scene.x0), color_begin=k, color_end=k)
    assert e.value.status == cc.ERR_INVALID_ARG
