"""Concurrent solves (cc_solve_concurrent): several independent meshes, each on
its own stream and host thread, must give each mesh's own cc_solve_step result
bit for bit, follow the oracle, keep a failing mesh from stopping the others,
and refuse arguments under which the solves could not run side by side."""
import numpy as np
import pytest

import meshgen
from oracle import fem, solvers, subspace, topology

torch = pytest.importorskip("torch")
import paper_2510_12053_gb300 as cc  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()


def _scenes():
    a = meshgen.stretch_box(5, 4, 6, E=3e5, nu=0.30, factor=1.3, jitter_amount=0.05, seed=1)
    b = meshgen.stretch_box(4, 4, 4, E=2e6, nu=0.25, factor=1.2, axis=1, seed=2)
    c = meshgen.cantilever(3, 3, 8, cell=1 / 16, E=1e5, nu=0.3)      # dynamic (h > 0)
    d = meshgen.stretch_box(6, 3, 4, E=5e4, nu=0.30, factor=1.1, jitter_amount=0.05, seed=3, axis=2)
    return [a, b, c, d]


def _meshes(scenes, k=2):
    out = []
    for sc in scenes:
        m = cc.Mesh.from_scene(sc, stream=torch.cuda.Stream())
        m.color()
        m.build_subspace(k)
        out.append(m)
    torch.cuda.synchronize()
    return out


def _inputs(scenes):
    xs = [cc.to_soa(sc.x0) for sc in scenes]
    vs = [cc.to_soa(sc.v0) if sc.h > 0 else None for sc in scenes]
    torch.cuda.synchronize()
    return xs, vs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("graph", [False, True])
def test_concurrent_solves_equal_separate_solves(precision, graph):
    scenes = _scenes()
    meshes = _meshes(scenes)
    kw = dict(precision=precision, tol=1e-6, max_iters=200, check_every=4, use_graph=graph, history=True)
    xs, vs = _inputs(scenes)
    sep = [m.solve_step(x, v, **kw) for m, x, v in zip(meshes, xs, vs)]
    torch.cuda.synchronize()
    xc, vc = _inputs(scenes)
    con = cc.solve_concurrent(meshes, xc, vc, **kw)
    torch.cuda.synchronize()
    for k in range(len(scenes)):
        assert sep[k].converged and con[k].converged
        assert con[k].iterations == sep[k].iterations
        assert con[k].g_final == sep[k].g_final and con[k].energy == sep[k].energy
        assert con[k].updates == sep[k].updates
        np.testing.assert_array_equal(con[k].residuals, sep[k].residuals)
        assert torch.equal(xc[k], xs[k])
        if vs[k] is not None:
            assert torch.equal(vc[k], vs[k])


def test_concurrent_solves_follow_the_oracle():
    """Three fp64 sweeps on a dynamic cantilever and a quasistatic box at once,
    against the oracle's coloured CC sweeps (Alg. 1) of each."""
    scenes = [meshgen.cantilever(3, 3, 8, cell=1 / 16, E=1e5, nu=0.3),
              meshgen.stretch_box(5, 4, 6, E=3e5, nu=0.30, factor=1.3, jitter_amount=0.05, seed=1)]
    meshes = _meshes(scenes)
    xs, vs = _inputs(scenes)
    res = cc.solve_concurrent(meshes, xs, vs, precision="fp64", tol=0.0, max_iters=3, min_iters=3)
    torch.cuda.synchronize()
    for sc, x, v, r in zip(scenes, xs, vs, res):
        pb = fem.problem_from_scene(sc)
        topo = topology.Topology(pb.n, pb.tets, pb.free)
        sup, U = subspace.build_local_bases(pb, topo, 2)
        xt = pb.inertial_target(sc.x0, sc.v0) if sc.h > 0 else None
        x_o = sc.x0.copy()
        for _ in range(3):
            x_o = solvers.sweep(pb, topo, sup, U, x_o, xt, "cc", "colored")
        assert r.iterations == 3
        np.testing.assert_allclose(cc.from_soa(x), x_o, rtol=0, atol=1e-12 * np.abs(x_o).max())
        if v is not None:
            v_o = (x_o - sc.x0) / sc.h
            np.testing.assert_allclose(cc.from_soa(v), v_o, rtol=0, atol=1e-9 * max(np.abs(v_o).max(), 1e-30))
        assert r.energy == pytest.approx(pb.energy(x_o, xt), rel=1e-11)


def test_a_failing_mesh_does_not_stop_the_others():
    good = _scenes()
    bad = meshgen.stretch_box(5, 5, 5, E=1e5, nu=0.45, factor=1.5)   # diverges with 2-ring bases
    scenes = [good[0], bad, good[3]]
    meshes = _meshes(scenes)
    kw = dict(precision="mixed", tol=1e-6, max_iters=300, check_every=2)
    xs, _ = _inputs(scenes)
    try:
        res = cc.solve_concurrent(meshes, xs, **kw)
        statuses = [cc.OK if r.converged else cc.ERR_NOT_CONVERGED for r in res]
    except cc.CCError as e:
        assert "mesh 1" in str(e)
        statuses = e.statuses
    torch.cuda.synchronize()
    assert statuses[0] == cc.OK and statuses[2] == cc.OK
    assert statuses[1] != cc.OK
    for k in (0, 2):
        xk = cc.to_soa(scenes[k].x0)
        torch.cuda.synchronize()
        r = meshes[k].solve_step(xk, **kw)
        torch.cuda.synchronize()
        assert r.converged
        assert torch.equal(xs[k], xk)


def test_concurrent_solve_refuses_shared_or_default_streams():
    scenes = _scenes()[:2]
    s = torch.cuda.Stream()
    shared = [cc.Mesh.from_scene(sc, stream=s) for sc in scenes]
    default = cc.Mesh.from_scene(scenes[0])
    own = cc.Mesh.from_scene(scenes[1], stream=torch.cuda.Stream())
    own2 = cc.Mesh.from_scene(scenes[1], stream=torch.cuda.Stream())
    for m in shared + [default, own, own2]:
        m.color()
        m.build_subspace(1)
    x0 = [cc.to_soa(sc.x0) for sc in scenes]
    torch.cuda.synchronize()
    before = [x.clone() for x in x0]
    cases = [(shared, x0, "share a stream"), ([default, own], x0, "default stream"),
             ([own, own], [x0[1], x0[1].clone()], "twice"), ([own, own2], [x0[1], x0[1]], "share x")]
    for ms, xs, msg in cases:
        with pytest.raises(cc.CCError) as ei:
            cc.solve_concurrent(ms, xs, max_iters=5)
        assert ei.value.status == cc.ERR_INVALID_ARG and msg in str(ei.value)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(x0, before))      # nothing ran
