"""Batches: several independent meshes solved as one disjoint union
(cc_build_batch / cc_solve_batch) must reproduce the meshes' own colourings,
bases and solves bit for bit, and stop each mesh at its own tolerance."""
import numpy as np
import pytest

import meshgen
from oracle import topology

torch = pytest.importorskip("torch")
import paper_2510_12053_gb300 as cc  # noqa: E402

pytestmark = pytest.mark.gpu


def _scenes():
    a = meshgen.stretch_box(5, 4, 6, E=3e5, nu=0.30, factor=1.3, jitter_amount=0.05, seed=1)
    b = meshgen.stretch_box(4, 4, 4, E=2e6, nu=0.25, factor=1.2, axis=1, seed=2)
    c = meshgen.stretch_box(6, 3, 4, E=5e4, nu=0.30, factor=1.1, jitter_amount=0.05, seed=3, axis=2)
    return [a, b, c]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()


def test_union_colours_and_bases_equal_each_mesh():
    scenes = _scenes()
    batch = cc.Mesh.from_scenes(scenes)
    cols = batch.color()
    batch.build_subspace(2)
    off = batch.batch_offsets()
    sp, si, U = batch.export("sup_ptr"), batch.export("sup_idx"), batch.export("U").reshape(-1, 3, 3)
    for k, sc in enumerate(scenes):
        m = cc.Mesh.from_scene(sc)
        ck = m.color()
        m.build_subspace(2)
        np.testing.assert_array_equal(cols[off[k]:off[k + 1]], ck)
        np.testing.assert_array_equal(ck, topology.Topology(sc.n, sc.tets, sc.pinned == 0).color)
        spk, sik, Uk = m.export("sup_ptr"), m.export("sup_idx"), m.export("U").reshape(-1, 3, 3)
        for v in range(sc.n):
            g = off[k] + v
            np.testing.assert_array_equal(si[sp[g]:sp[g + 1]] - off[k], sik[spk[v]:spk[v + 1]])
            np.testing.assert_array_equal(U[sp[g]:sp[g + 1]], Uk[spk[v]:spk[v + 1]])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("graph", [False, True])
def test_batch_solve_equals_individual_solves(precision, graph):
    scenes = _scenes()
    batch = cc.Mesh.from_scenes(scenes)
    batch.color()
    batch.build_subspace(2)
    off = batch.batch_offsets()
    x0 = np.concatenate([sc.x0 for sc in scenes])
    xd = cc.to_soa(x0)
    res = batch.solve_batch(xd, precision=precision, tol=1e-6, max_iters=200, check_every=1, use_graph=graph)
    xb = cc.from_soa(xd)
    assert np.all(res["status"] == 1)
    for k, sc in enumerate(scenes):
        m = cc.Mesh.from_scene(sc)
        m.color()
        m.build_subspace(2)
        xk = cc.to_soa(sc.x0)
        r = m.solve_step(xk, precision=precision, tol=1e-6, max_iters=200, check_every=1)
        assert r.converged
        assert res["iterations"][k] == r.iterations
        np.testing.assert_array_equal(xb[off[k]:off[k + 1]], cc.from_soa(xk))
        assert res["g0"][k] == pytest.approx(r.g0, rel=1e-12)


def test_batch_freezes_a_diverging_mesh_and_finishes_the_others():
    scenes = _scenes()
    bad = meshgen.stretch_box(5, 5, 5, E=1e5, nu=0.45, factor=1.5)   # diverges with 2-ring bases
    scenes = [scenes[0], bad, scenes[2]]
    batch = cc.Mesh.from_scenes(scenes)
    batch.color()
    batch.build_subspace(2)
    xd = cc.to_soa(np.concatenate([sc.x0 for sc in scenes]))
    res = batch.solve_batch(xd, precision="mixed", tol=1e-6, max_iters=300, check_every=2)
    assert res["status"][0] == 1 and res["status"][2] == 1
    assert res["status"][1] == -1


def test_autotune_picks_a_candidate_and_keeps_results():
    scenes = _scenes()
    batch = cc.Mesh.from_scenes(scenes)
    batch.color()
    batch.build_subspace(2)
    x0 = cc.to_soa(np.concatenate([sc.x0 for sc in scenes]))
    before = x0.clone()
    res_a = batch.solve_batch(x0.clone(), precision="mixed", tol=1e-6, max_iters=200, check_every=1)
    tune = batch.autotune(x0, precision="mixed", sweeps=2)
    assert torch.equal(x0, before)                      # x is not modified
    assert tune["couple_threads"] in (32, 64, 128, 256) and tune["gather_warps"] in (2, 4, 8)
    assert all(v > 0 for v in tune["couple_ms"] + tune["gather_ms"])
    assert tune["couple_ms"][(32, 64, 128, 256).index(tune["couple_threads"])] == min(tune["couple_ms"])
    assert tune["gather_ms"][(2, 4, 8).index(tune["gather_warps"])] == min(tune["gather_ms"])
    if tune["couple_threads"] != 32:
        assert all(v > 0 for v in tune["row_lanes_ms"])
        assert tune["row_lanes_ms"][(1, 2, 4, 8).index(tune["couple_row_lanes"])] == min(tune["row_lanes_ms"])
    xb = x0.clone()
    res_b = batch.solve_batch(xb, precision="mixed", tol=1e-6, max_iters=200, check_every=1)
    assert np.all(res_b["status"] == 1)
    assert np.all(np.abs(res_b["iterations"] - res_a["iterations"]) <= 2)
