"""GPU (CUDA C-ABI) vs FP64 oracle parity.

Integer outputs (adjacency, colours, supports) must be bit-identical.  A
float64 sweep must match the oracle to 1e-12 relative in x (and its update to
1e-9 relative).  Mixed-precision results are checked against tolerances
derived from float32 Hessian arithmetic: float32 coupling products carry about
1e-6 relative error, amplified by the condition of the 3x3 local systems.
"""
import numpy as np
import pytest

import meshgen
from oracle import fem, material, solvers, subspace, topology

torch = pytest.importorskip("torch")
import paper_2510_12053_gb300 as cc  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _oracle(scene, k=None):
    pb = fem.problem_from_scene(scene)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    if k is None:
        return pb, topo, None, None
    sup, U = subspace.build_local_bases(pb, topo, k)
    return pb, topo, sup, U


def _gpu(scene, k=None):
    m = cc.Mesh.from_scene(scene)
    m.color()
    if k is not None:
        m.build_subspace(k)
    return m


def _state(scene, amp, seed):
    d = meshgen.normal(seed, np.arange(3 * scene.n)).reshape(-1, 3) * amp * scene.cell
    return scene.x0 + d * (scene.pinned == 0)[:, None]


def _box(nu=0.3, factor=1.2, dims=(6, 6, 6), jit=0.05, seed=2, E=1e5):
    return meshgen.stretch_box(*dims, E=E, nu=nu, factor=factor, jitter_amount=jit, seed=seed)


# ---------------------------------------------------------------- integers
@pytest.mark.parametrize("scene", [meshgen.cube8_stretch(), _box(dims=(7, 5, 6), seed=5)],
                         ids=["cube8", "box7x5x6"])
def test_adjacency_and_colouring_bit_exact(scene):
    pb, topo, _, _ = _oracle(scene)
    m = cc.Mesh.from_scene(scene)
    cols = m.color()
    np.testing.assert_array_equal(m.export("vt_ptr"), topo.vt_ptr)
    np.testing.assert_array_equal(m.export("vt_tet"), topo.vt_tet)
    np.testing.assert_array_equal(m.export("vt_corner"), topo.vt_corner)
    np.testing.assert_array_equal(m.export("nbr_ptr"), topo.nbr_ptr)
    np.testing.assert_array_equal(m.export("nbr_idx"), topo.nbr_idx)
    np.testing.assert_array_equal(cols, topo.color)
    np.testing.assert_allclose(m.export("mass"), pb.mass, rtol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_supports_bit_exact_and_bases_match(k):
    scene = _box(dims=(6, 5, 4), seed=3)
    pb, topo, sup, U = _oracle(scene, k)
    m = _gpu(scene, k)
    sp, si, Ug = m.export("sup_ptr"), m.export("sup_idx"), m.export("U").reshape(-1, 3, 3)
    for v in range(pb.n):
        np.testing.assert_array_equal(si[sp[v]:sp[v + 1]], sup[v])
        if len(sup[v]):
            np.testing.assert_allclose(Ug[sp[v]:sp[v + 1]], U[v], rtol=0, atol=1e-10 * max(1.0, np.abs(U[v]).max()))


# ---------------------------------------------------------------- energy
@pytest.mark.parametrize("dynamic", [False, True])
def test_energy_and_gradient(dynamic):
    if dynamic:
        scene = meshgen.cantilever(3, 4, 7, cell=1 / 16, E=1e6, nu=0.45)
    else:
        scene = _box(dims=(5, 6, 4), factor=1.3)
    pb, _, _, _ = _oracle(scene)
    x = _state(scene, 0.3, 8)
    xt = None
    if dynamic:
        v = meshgen.normal(9, np.arange(3 * scene.n)).reshape(-1, 3) * 0.1
        xt = pb.inertial_target(scene.X, v)
    E_o = pb.energy(x, xt)
    g_o = pb.gradient(x, xt)
    g_o[~pb.free] = 0.0
    m = cc.Mesh.from_scene(scene)
    xd = cc.to_soa(x)
    xtd = cc.to_soa(xt) if dynamic else None
    for prec, tol in [("fp64", 1e-12), ("mixed", 1e-10)]:
        E, g, gn = m.energy_grad(xd, xtd, precision=prec)
        gg = cc.from_soa(g)
        assert E == pytest.approx(E_o, rel=1e-12)
        assert np.abs(gg - g_o).max() <= tol * np.abs(g_o).max()
        assert gn == pytest.approx(np.linalg.norm(g_o), rel=max(tol, 1e-13))


# ---------------------------------------------------------------- one sweep, FP64
@pytest.mark.parametrize("update", ["cc", "cd", "jgs2"])
@pytest.mark.parametrize("schedule", ["colored", "jacobi"])
def test_one_fp64_sweep_matches_oracle(update, schedule):
    scene = _box()
    pb, topo, sup, U = _oracle(scene, 2)
    x0 = _state(scene, 0.05, 4)
    st_o = solvers.Stats()
    x_o = solvers.sweep(pb, topo, sup, U, x0, None, update, schedule, st_o)
    m = _gpu(scene, 2)
    xd = cc.to_soa(x0)
    st = m.sweep(xd, update=update, schedule=schedule, precision="fp64")
    x_g = cc.from_soa(xd)
    assert np.abs(x_g - x_o).max() <= 1e-12 * np.abs(x_o).max()
    d_o, d_g = x_o - x0, x_g - x0
    assert np.abs(d_g - d_o).max() <= 1e-9 * np.abs(d_o).max()
    assert (st.fallback_empty, st.fallback_reduced, st.fallback_schur) == \
        (st_o.fallback_empty, st_o.fallback_reduced, st_o.fallback_schur)


@pytest.mark.parametrize("threads,lanes", [(32, 0)] + [(t, r) for t in (64, 128, 256) for r in (1, 2, 4, 8)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_every_coupling_launch_shape_matches_oracle(threads, lanes, precision):
    """One CC sweep with each coupling-kernel shape (32 = one warp per vertex;
    otherwise threads per vertex x threads per block row)."""
    scene = _box(dims=(7, 6, 5), seed=9)
    pb, topo, sup, U = _oracle(scene, 2)
    x0 = _state(scene, 0.05, 6)
    x_o = solvers.sweep(pb, topo, sup, U, x0, None, "cc", "colored")
    m = _gpu(scene, 2)
    m.set_launch_shape(couple_threads=threads, couple_row_lanes=lanes)
    xd = cc.to_soa(x0)
    m.sweep(xd, update="cc", schedule="colored", precision=precision)
    d_o, d_g = x_o - x0, cc.from_soa(xd) - x0
    tol = 1e-9 if precision == "fp64" else 1e-4
    assert np.abs(d_g - d_o).max() <= tol * np.abs(d_o).max()


def test_launch_shape_rejects_unknown_values():
    m = _gpu(_box(dims=(3, 3, 3)), 2)
    with pytest.raises(cc.CCError):
        m.set_launch_shape(couple_threads=96)
    with pytest.raises(cc.CCError):
        m.set_launch_shape(gather_warps=3)
    with pytest.raises(cc.CCError):
        m.set_launch_shape(couple_row_lanes=3)


def test_pinned_rows_untouched_and_colour_range():
    scene = _box()
    m = _gpu(scene, 2)
    xd = cc.to_soa(scene.x0)
    before = cc.from_soa(xd)
    m.sweep(xd, update="cc", schedule="colored", precision="fp64", color_begin=0, color_end=1)
    after = cc.from_soa(xd)
    cols = m.export("color")
    moved = np.any(after != before, axis=1)
    assert not np.any(moved & (scene.pinned == 1))
    assert np.all(cols[moved] == 0)


# ---------------------------------------------------------------- mixed precision trajectory
def test_mixed_trajectory_matches_oracle_over_50_sweeps():
    """Energy and gradient-norm trajectories within 1e-4 relative over 50
    coloured CC sweeps; final positions within 1e-5 of the bbox diagonal."""
    scene = meshgen.stretch_box(8, 8, 8, E=1e5, nu=0.3, factor=1.5, name="cube8_nu03")
    pb, topo, sup, U = _oracle(scene, 2)
    x = scene.x0.copy()
    E_o, G_o = [], []
    for _ in range(50):
        x = solvers.sweep(pb, topo, sup, U, x, None, "cc", "colored")
        E_o.append(pb.energy(x))
        G_o.append(np.linalg.norm(pb.gradient(x)[pb.free]))
    m = _gpu(scene, 2)
    xd = cc.to_soa(scene.x0)
    E_g, G_g = [], []
    for _ in range(50):
        m.sweep(xd, update="cc", schedule="colored", precision="mixed")
        E, _, gn = m.energy_grad(xd, precision="fp64", want_grad=False)
        E_g.append(E)
        G_g.append(gn)
    E_o, G_o, E_g, G_g = map(np.array, (E_o, G_o, E_g, G_g))
    assert np.max(np.abs(E_g - E_o) / np.abs(E_o)) <= 1e-4
    assert np.max(np.abs(G_g - G_o) / G_o) <= 1e-4
    diag = np.linalg.norm(scene.X.max(0) - scene.X.min(0))
    assert np.abs(cc.from_soa(xd) - x).max() <= 1e-5 * diag


def test_mixed_solve_reaches_tolerance_and_matches_fp64():
    scene = meshgen.stretch_box(8, 8, 8, E=1e5, nu=0.3, factor=1.2, name="cube8_nu03")
    m = _gpu(scene, 2)
    res = {}
    for prec in ["fp64", "mixed"]:
        xd = cc.to_soa(scene.x0)
        r = m.solve_step(xd, precision=prec, tol=1e-6, max_iters=120, history=True)
        res[prec] = (r, cc.from_soa(xd))
        assert r.converged and r.g_final <= 1e-6 * r.g0
    (r64, x64), (rmx, xmx) = res["fp64"], res["mixed"]
    diag = np.linalg.norm(scene.X.max(0) - scene.X.min(0))
    assert np.abs(x64 - xmx).max() <= 1e-5 * diag
    assert abs(r64.iterations - rmx.iterations) <= 2


def test_graph_replay_matches_launch_by_launch_and_profiles():
    scene = meshgen.stretch_box(8, 8, 8, E=1e5, nu=0.3, factor=1.2, name="cube8_nu03")
    m = _gpu(scene, 2)
    out = {}
    for graph in (False, True):
        m.profile_enable(True)
        xd = cc.to_soa(scene.x0)
        r = m.solve_step(xd, precision="mixed", tol=0.0, max_iters=24, min_iters=24, check_every=8,
                         use_graph=graph, history=True)
        prof = m.profile_read()
        m.profile_enable(False)
        out[graph] = (cc.from_soa(xd), r.residuals)
        assert r.iterations == 24
        for k in ("tet_eval", "gather", "local_solve", "reduce"):
            assert prof[k]["launches"] > 0 and prof[k]["ms"] > 0, (graph, k)
        assert prof["total_launches"] >= 24 * 8 * 3
    np.testing.assert_array_equal(out[False][0], out[True][0])
    np.testing.assert_array_equal(out[False][1], out[True][1])


# ---------------------------------------------------------------- dynamics
def test_dynamic_step_matches_oracle():
    scene = meshgen.cantilever(3, 3, 8, cell=1 / 16, E=1e5, nu=0.3)
    pb, topo, sup, U = _oracle(scene, 2)
    xt = pb.inertial_target(scene.X, scene.v0)
    x_o = scene.X.copy()
    for _ in range(3):
        x_o = solvers.sweep(pb, topo, sup, U, x_o, xt, "cc", "colored")
    v_o = (x_o - scene.X) / scene.h
    m = _gpu(scene, 2)
    xd, vd = cc.to_soa(scene.X), cc.to_soa(scene.v0)
    r = m.solve_step(xd, vd, precision="fp64", tol=0.0, max_iters=3, min_iters=3)
    assert r.iterations == 3
    np.testing.assert_allclose(cc.from_soa(xd), x_o, rtol=0, atol=1e-12 * np.abs(x_o).max())
    np.testing.assert_allclose(cc.from_soa(vd), v_o, rtol=0, atol=1e-9 * max(np.abs(v_o).max(), 1e-30))
    assert r.energy == pytest.approx(pb.energy(x_o, xt), rel=1e-11)


# ---------------------------------------------------------------- full size, sampled
def test_cube32_full_size_sampled_updates():
    """32^3 jittered cube (35 937 vertices): the GPU's first-colour updates
    (the bench's launch configuration) against the oracle's local updates for
    sampled vertices, float64 and mixed."""
    scene = meshgen.cube32_stretch(E=1e5)
    pb = fem.problem_from_scene(scene)
    m = _gpu(scene, 2)
    cols = m.export("color")
    sp, si, Ug = m.export("sup_ptr"), m.export("sup_idx"), m.export("U").reshape(-1, 3, 3)
    free0 = np.flatnonzero((cols == 0) & pb.free)
    rng = meshgen.uniform01(77, np.arange(40))
    sample = np.unique(free0[(rng * len(free0)).astype(int)])
    # oracle: rest Hessian bases for the sample, then updates from g, H at x0
    H0 = pb.hessian(scene.X)
    nb_ptr, nb_idx = topology.vertex_neighbors(pb.n, pb.tets)
    x0 = scene.x0
    g = pb.gradient(x0)
    H = pb.hessian(x0)
    expect = {}
    for i in sample:
        S = np.array([j for j in topology.k_ring(int(i), 2, nb_ptr, nb_idx) if j != i and pb.free[j]])
        np.testing.assert_array_equal(si[sp[i]:sp[i + 1]], S)
        Ui = subspace.local_basis(H0, int(i), S)
        np.testing.assert_allclose(Ug[sp[i]:sp[i + 1]], Ui, rtol=0, atol=1e-10 * np.abs(Ui).max())
        expect[int(i)] = solvers.local_update("cc", H, g, int(i), S, Ui)
    for prec, tol in [("fp64", 1e-9), ("mixed", 1e-4)]:
        xd = cc.to_soa(x0)
        m.sweep(xd, update="cc", schedule="colored", precision=prec, color_begin=0, color_end=1)
        d = cc.from_soa(xd) - x0
        scale = max(np.abs(dx).max() for dx in expect.values())
        for i, dx in expect.items():
            assert np.abs(d[i] - dx).max() <= tol * max(np.abs(dx).max(), 1e-3 * scale), (prec, i)


# ---------------------------------------------------------------- errors
def test_errors_are_reported_not_raised_from_c():
    scene = _box(dims=(3, 3, 3))
    m = cc.Mesh.from_scene(scene)
    xd = cc.to_soa(scene.x0)
    with pytest.raises(cc.CCError) as e:
        m.sweep(xd)  # not coloured yet
    assert e.value.status == cc.ERR_STATE
    m.color()
    with pytest.raises(cc.CCError) as e:
        m.sweep(xd, update="cc")  # no subspace yet
    assert e.value.status == cc.ERR_STATE
    with pytest.raises(cc.CCError) as e:
        m.build_subspace(0)
    assert e.value.status == cc.ERR_INVALID_ARG
    bad = scene.tets.copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(cc.CCError) as e:
        cc.Mesh(scene.X, bad, scene.pinned, E=1e5, nu=0.3)
    assert e.value.status == cc.ERR_INVALID_ARG
    with pytest.raises(cc.CCError) as e:
        cc.Mesh(scene.X, scene.tets, scene.pinned, E=1e5, nu=0.5)
    assert e.value.status == cc.ERR_INVALID_ARG


# ---------------------------------------------------------------- corotated bases (Sec. 3.1)
@pytest.mark.parametrize("schedule", ["colored", "jacobi"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_corotated_sweep_matches_oracle(schedule, precision):
    scene = meshgen.twist_box(3, 3, 6, angle=np.pi / 2, nu=0.3, jitter_amount=0.05, seed=4)
    pb, topo, sup, U = _oracle(scene, 2)
    x0 = scene.x0
    x_o = solvers.sweep(pb, topo, sup, U, x0, None, "cc", schedule, corotated=True)
    x_f = solvers.sweep(pb, topo, sup, U, x0, None, "cc", schedule)
    m = _gpu(scene, 2)
    xd = cc.to_soa(x0)
    m.sweep(xd, update="cc", schedule=schedule, precision=precision, corotated=True)
    x_g = cc.from_soa(xd)
    d_o, d_g = x_o - x0, x_g - x0
    tol = 1e-9 if precision == "fp64" else 1e-4
    assert np.abs(d_g - d_o).max() <= tol * np.abs(d_o).max()
    if precision == "fp64":
        assert np.abs(x_g - x_o).max() <= 1e-12 * np.abs(x_o).max()
    assert np.abs(x_f - x_o).max() > 1e-3 * np.abs(d_o).max()    # the rotation matters here


def test_corotated_solve_follows_the_oracle_and_beats_fixed_bases():
    scene = meshgen.twist_box(3, 3, 8, angle=np.pi / 2, nu=0.3)
    pb, topo, sup, U = _oracle(scene, 2)
    _, h_o = solvers.solve(pb, topo, sup, U, scene.x0, kind="cc", tol=1e-6, max_iters=200, corotated=True)
    m = _gpu(scene, 2)
    res = {}
    for corot in (False, True):
        xd = cc.to_soa(scene.x0)
        res[corot] = m.solve_step(xd, precision="mixed", tol=1e-6, max_iters=200, corotated=corot,
                                  use_graph=True, check_every=1)
    assert h_o.converged and res[True].converged
    assert abs(res[True].iterations - h_o.iterations) <= 2
    assert res[True].iterations < res[False].iterations


# ---------------------------------------------------------------- global line search (Sec. 4.4)
def test_line_search_follows_the_oracle_where_plain_cc_blows_up():
    scene = meshgen.stretch_box(4, 3, 3, E=1e5, nu=0.45, factor=1.5, jitter_amount=0.05, seed=2)
    pb, topo, sup, U = _oracle(scene, 2)
    iters = 8
    _, h_o = solvers.solve(pb, topo, sup, U, scene.x0, kind="cc", tol=1e-12, max_iters=iters, line_search=True)
    m = _gpu(scene, 2)
    xd = cc.to_soa(scene.x0)
    r = m.solve_step(xd, precision="fp64", tol=1e-12, max_iters=iters, line_search=True, history=True)
    hist = r.residuals[:iters + 1]
    np.testing.assert_allclose(hist, h_o.grad_norm, rtol=1e-8)
    assert r.energy == pytest.approx(h_o.energy[-1], rel=1e-10)
    assert h_o.energy[-1] <= h_o.energy[0]
    # mixed precision: finite and energy-decreasing where the plain mixed solve is not
    xm = cc.to_soa(scene.x0)
    e0 = m.energy_grad(cc.to_soa(scene.x0), precision="fp64", want_grad=False)[0]
    rm = m.solve_step(xm, precision="mixed", tol=1e-12, max_iters=iters, line_search=True)
    assert np.isfinite(rm.g_final) and rm.energy <= e0
    xp = cc.to_soa(scene.x0)
    try:
        rp = m.solve_step(xp, precision="mixed", tol=1e-12, max_iters=iters)
        blew_up = rp.g_final > 10 * rp.g0
    except cc.CCError:
        blew_up = True
    assert blew_up


def test_batch_line_search_equals_each_mesh_line_search():
    """Sec. 4.4's line search inside a batch: every mesh backtracks on its own
    energy, so each follows its own single-mesh line-search solve (here one
    mesh that plain CC blows up and one that converges)."""
    scenes = [meshgen.stretch_box(4, 3, 3, E=1e5, nu=0.45, factor=1.5, jitter_amount=0.05, seed=2),
              meshgen.stretch_box(3, 3, 4, E=2e5, nu=0.3, factor=1.2, seed=3)]
    b = cc.Mesh.from_scenes(scenes)
    b.color()
    b.build_subspace(2)
    off = b.batch_offsets()
    xd = cc.to_soa(np.concatenate([sc.x0 for sc in scenes]))
    iters = 8
    res = b.solve_batch(xd, precision="fp64", tol=1e-12, max_iters=iters, line_search=True)
    xb = cc.from_soa(xd)
    for k, sc in enumerate(scenes):
        m = _gpu(sc, 2)
        xk = cc.to_soa(sc.x0)
        r = m.solve_step(xk, precision="fp64", tol=1e-12, max_iters=iters, line_search=True)
        assert res["iterations"][k] == r.iterations
        assert res["status"][k] != -1
        np.testing.assert_allclose(xb[off[k]:off[k + 1]], cc.from_soa(xk), rtol=0,
                                   atol=1e-10 * np.abs(cc.from_soa(xk)).max())
        m.close()



# ---------------------------------------------------------------- restarted bases (Sec. 4.4)
def test_bases_rebuilt_at_x_match_the_oracle():
    scene = _box(dims=(5, 4, 4), seed=7, factor=1.3)
    pb, topo, sup, U = _oracle(scene, 2)
    x = _state(scene, 0.03, 9)
    Ux, kept_o = subspace.rebuild_bases_at(pb, sup, U, x)
    m = _gpu(scene, 2)
    kept = m.build_subspace_at(cc.to_soa(x))
    assert kept == kept_o == 0
    sp, Ug = m.export("sup_ptr"), m.export("U").reshape(-1, 3, 3)
    for v in np.flatnonzero(pb.free):
        np.testing.assert_allclose(Ug[sp[v]:sp[v + 1]], Ux[v], rtol=0, atol=1e-10 * max(1.0, np.abs(Ux[v]).max()))


def test_restarted_solve_follows_the_oracle():
    scene = meshgen.twist_box(3, 3, 8, angle=np.pi / 2, nu=0.3)
    pb, topo, sup, U = _oracle(scene, 2)
    _, h_o = solvers.solve(pb, topo, sup, U, scene.x0, kind="cc", tol=1e-6, max_iters=200, restart_every=5)
    _, h_f = solvers.solve(pb, topo, sup, U, scene.x0, kind="cc", tol=1e-6, max_iters=200)
    m = _gpu(scene, 2)
    r = m.solve_step(cc.to_soa(scene.x0), precision="fp64", tol=1e-6, max_iters=200, restart_every=5, check_every=1)
    assert h_o.converged and r.converged
    assert abs(r.iterations - h_o.iterations) <= 1 and h_o.iterations < h_f.iterations


# ---------------------------------------------------------------- Fixed Corotational material (Sec. 4.1)
def _fcr_oracle(scene, k=None):
    pb = fem.problem_from_scene(scene, "fcr")
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    if k is None:
        return pb, topo, None, None
    sup, U = subspace.build_local_bases(pb, topo, k)
    return pb, topo, sup, U


@pytest.mark.parametrize("dynamic", [False, True])
def test_fcr_energy_and_gradient(dynamic):
    if dynamic:
        scene = meshgen.cantilever(3, 4, 7, cell=1 / 16, E=1e6, nu=0.45)
    else:
        scene = _box(dims=(5, 6, 4), factor=1.3)
    pb, _, _, _ = _fcr_oracle(scene)
    x = _state(scene, 0.08, 8)
    assert np.all(material.det3(pb.deformation(x)) > 0)   # the GPU path needs non-inverted tets
    xt = None
    if dynamic:
        v = meshgen.normal(9, np.arange(3 * scene.n)).reshape(-1, 3) * 0.1
        xt = pb.inertial_target(scene.X, v)
    E_o = pb.energy(x, xt)
    g_o = pb.gradient(x, xt)
    g_o[~pb.free] = 0.0
    m = cc.Mesh.from_scene(scene, model="fcr")
    xd = cc.to_soa(x)
    xtd = cc.to_soa(xt) if dynamic else None
    for prec, tol in [("fp64", 1e-12), ("mixed", 1e-10)]:
        E, g, gn = m.energy_grad(xd, xtd, precision=prec)
        assert E == pytest.approx(E_o, rel=1e-12)
        assert np.abs(cc.from_soa(g) - g_o).max() <= tol * np.abs(g_o).max()
    # an inverted tet has no rotation to extract on the GPU: the energy is NaN
    xi = scene.X.copy()
    xi[pb.free] *= -1.0
    assert np.any(material.det3(pb.deformation(xi)) <= 0)
    for prec in ("fp64", "mixed"):
        assert np.isnan(m.energy_grad(cc.to_soa(xi), xtd, precision=prec, want_grad=False)[0])


@pytest.mark.parametrize("update", ["cc", "cd"])
def test_fcr_one_fp64_sweep_matches_oracle(update):
    scene = _box()
    pb, topo, sup, U = _fcr_oracle(scene, 2)
    x0 = _state(scene, 0.05, 4)
    x_o = solvers.sweep(pb, topo, sup, U, x0, None, update, "colored")
    m = cc.Mesh.from_scene(scene, model="fcr")
    m.color()
    m.build_subspace(2)
    xd = cc.to_soa(x0)
    m.sweep(xd, update=update, precision="fp64")
    x_g = cc.from_soa(xd)
    assert np.abs(x_g - x_o).max() <= 1e-12 * np.abs(x_o).max()
    assert np.abs((x_g - x0) - (x_o - x0)).max() <= 1e-9 * np.abs(x_o - x0).max()


def test_fcr_mixed_solve_follows_the_oracle():
    scene = meshgen.stretch_box(5, 4, 4, E=1e5, nu=0.3, factor=1.5, jitter_amount=0.05, seed=1)
    pb, topo, sup, U = _fcr_oracle(scene, 2)
    _, h_o = solvers.solve(pb, topo, sup, U, scene.x0, kind="cc", tol=1e-6, max_iters=150)
    m = cc.Mesh.from_scene(scene, model="fcr")
    m.color()
    m.build_subspace(2)
    r = m.solve_step(cc.to_soa(scene.x0), precision="mixed", tol=1e-6, max_iters=150, check_every=1)
    assert h_o.converged and r.converged
    assert abs(r.iterations - h_o.iterations) <= 2
    assert r.energy == pytest.approx(h_o.energy[-1], rel=1e-8)


def test_batch_rejects_mixed_material_models():
    a = meshgen.stretch_box(3, 3, 3, E=1e5, nu=0.3)
    descs = (cc.MeshDesc * 2)()
    keep = []
    for k, model in enumerate((0, 1)):
        X = np.ascontiguousarray(a.X)
        T = np.ascontiguousarray(a.tets, dtype=np.int32)
        P = np.ascontiguousarray(a.pinned, dtype=np.uint8)
        keep += [X, T, P]
        descs[k] = cc.MeshDesc(X.ctypes.data, X.shape[0], T.ctypes.data, T.shape[0], P.ctypes.data,
                               cc.Material(1e5, 0.3, 1000.0, model))
    out = cc.ctypes.c_void_p()
    rc = cc.lib().cc_build_batch(descs, 2, 0.0, None, None, cc.ctypes.byref(out))
    assert rc == cc.ERR_INVALID_ARG
