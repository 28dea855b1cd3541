"""Learned-subspace network and bases on the GPU against the FP64 oracle.

* the tcgen05 BF16 GEMM against an exact product of the same BF16 inputs
  (every N tile, split K);
* forward pass, loss and gradients against ``oracle.mlp`` evaluated with the
  same BF16 rounding points.  The GPU accumulates in float32 and rounds to
  BF16 where the oracle rounds a float64 value, so a handful of stored BF16
  values differ by one unit in the last place; the tolerances below (1e-3
  relative per tensor) bound that effect;
* Adam against the oracle's update on the same gradient;
* network inputs (bit for bit, the two material channels within one BF16
  step), targets, Eq. 5 residuals and the fallback set against
  ``oracle.learned``;
* a trained network against the method without it.
"""
import numpy as np
import pytest

import meshgen
from oracle import fem, learned, mlp, solvers, subspace, topology

torch = pytest.importorskip("torch")
import paper_2510_12053_gb300 as cc  # noqa: E402
from paper_2510_12053_gb300 import learned as cclearn  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _bf16(rows, cols, seed, ld=None, scale=1.0):
    """(CUDA bf16 tensor [rows, ld], float64 numpy of its first cols columns)."""
    a = (scale * meshgen.normal(seed, np.arange(rows * cols))).reshape(rows, cols).astype(np.float32)
    t = torch.zeros((rows, ld or cols), dtype=torch.bfloat16)
    t[:, :cols] = torch.from_numpy(a).to(torch.bfloat16)
    return t.cuda(), t[:, :cols].double().numpy()


# ---------------------------------------------------------------- GEMM
GEMM_CASES = [(128, 64, 64, 0, 0), (300, 256, 320, 0, 0), (1000, 576, 256, 0, 0), (257, 192, 200, 0, 0),
              (8192, 256, 576, 0, 0), (64, 128, 1000, 0, 0), (300, 256, 320, 64, 0), (300, 256, 320, 128, 0),
              (576, 256, 8192, 0, 16), (256, 258, 1000, 64, 5), (256, 256, 4096, 128, 64),
              (40000, 256, 258, 0, 0), (20000, 576, 256, 192, 0), (5000, 64, 64, 64, 0)]


@pytest.mark.parametrize("one_tile", [False, True], ids=["persistent", "one-tile"])
@pytest.mark.parametrize("M,N,K,tile,splits", GEMM_CASES)
def test_gemm_bf16_matches_exact_product(M, N, K, tile, splits, one_tile):
    ld = (K + 7) // 8 * 8
    A, An = _bf16(M, K, 1 + M, ld)
    B, Bn = _bf16(N, K, 2 + N, ld)
    C = cc.gemm_bf16_tn(A[:, :K], B[:, :K], n_tile=tile, k_splits=splits, one_tile_per_cta=one_tile)
    torch.cuda.synchronize()
    ref = An @ Bn.T
    err = np.abs(C.cpu().double().numpy() - ref).max()
    assert err <= 1e-5 * np.abs(ref).max() + 1e-6, err


# ---------------------------------------------------------------- activation
def test_activation_matches_erf_within_its_published_bound():
    """erf by Abramowitz-Stegun 7.1.26 (|error| <= 1.5e-7) against the oracle's
    erf (scipy, float64) and CUDA's erff through torch; GELU and GELU' against
    the oracle's erf-form formulas."""
    from scipy.special import erf as erf64
    x = np.concatenate([np.linspace(-9, 9, 20001), meshgen.normal(3, np.arange(20000)) * 2]).astype(np.float32)
    out = cc.mlp_activation(torch.from_numpy(x).cuda()).cpu().double().numpy()
    xd = x.astype(np.float64)
    # 1.5e-7 (the formula) + float32 evaluation (approximate reciprocal and __expf,
    # a few ulps each, amplified by the polynomial) < 1e-6, i.e. < 1/4000 of a BF16 step
    assert np.max(np.abs(out[:, 0] - erf64(xd))) <= 1e-6
    ref_cuda = torch.erf(torch.from_numpy(x).cuda()).cpu().double().numpy()
    assert np.max(np.abs(out[:, 0] - ref_cuda)) <= 1e-6
    g, gp = mlp.gelu(xd), mlp.gelu_grad(xd)
    assert np.max(np.abs(out[:, 1] - g) / np.maximum(1.0, np.abs(xd))) <= 1e-6
    assert np.max(np.abs(out[:, 2] - gp)) <= 2e-6


# ---------------------------------------------------------------- network
def _net(dims, max_batch, seed):
    net = cc.MLP(dims[0], dims[1], len(dims) - 2, dims[-1], max_batch=max_batch)
    p = meshgen.mlp_init(dims, seed, out_scale=1.0)
    p += (0.05 * meshgen.normal(seed + 7, np.arange(p.size))).astype(np.float32) * _bias_mask(dims)
    net.set_params(p)
    return net, p.astype(np.float64)


def _bias_mask(dims):
    m = np.zeros(meshgen.mlp_param_count(dims), dtype=np.float32)
    for _, sb in mlp.layer_slices(dims):
        m[sb] = 1.0
    return m


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


DIMS = [meshgen.mlp_dims(), [30, 40, 40, 24], [258, 64, 16]]
# shapes the one-kernel inference covers besides the full network (hidden
# widths multiples of 64 up to 256, output a multiple of 64)
FUSED_DIMS = [[100, 128, 128, 192], [8, 256, 64], [300, 192, 192, 192, 192, 320]]


@pytest.mark.parametrize("dims", DIMS + FUSED_DIMS[:1],
                         ids=["full", "small", "one-hidden", "fused-small"])
def test_forward_matches_oracle(dims):
    rows = 1000
    net, p = _net(dims, 64, 3)
    X, Xn = _bf16(rows, dims[0], 11, (dims[0] + 7) // 8 * 8)
    Y = net.forward(X).cpu().double().numpy()
    Yo, _ = mlp.forward(p, dims, Xn, rounding=True)
    assert _rel(Y, Yo) <= 1e-3
    assert np.abs(Y - Yo).max() <= 1e-2 * np.abs(Yo).max()


def test_forward_at_full_size_on_sampled_rows():
    """Inference over the 112 847 free vertices of the 48^3 cube: 257 sampled
    rows against the oracle, evaluated one by one."""
    dims = DIMS[0]
    rows = 112847
    net, p = _net(dims, 64, 4)
    X, Xn = _bf16(rows, dims[0], 12, 264)
    Y = net.forward(X)
    torch.cuda.synchronize()
    pick = np.unique((meshgen.uniform01(13, np.arange(256)) * rows).astype(np.int64).tolist() + [rows - 1])
    Yo, _ = mlp.forward(p, dims, Xn[pick], rounding=True)
    Ys = Y[torch.from_numpy(pick).cuda()].cpu().double().numpy()
    assert _rel(Ys, Yo) <= 1e-3
    assert np.abs(Ys - Yo).max() <= 1e-2 * np.abs(Yo).max()


@pytest.mark.parametrize("kind", [1, 2], ids=["multicast", "pair"])
@pytest.mark.parametrize("dims", [DIMS[0]] + FUSED_DIMS, ids=["full", "three-layer", "in8", "five-layer"])
@pytest.mark.parametrize("rows", [1, 127, 129, 1000, 2 * 152 * 128 + 5, 112847])
def test_fused_inference_equals_per_layer_bit_for_bit(dims, rows, kind):
    """The one-kernel inference (activations in shared memory, two tiles in
    flight per SM, SM pairs sharing weight tiles by multicast, or SM-pair
    M = 256 MMAs) against one GEMM launch per layer: the same MMAs, bias, GELU
    and BF16 rounding, so the same bits, for ragged row counts and odd numbers
    of 256-row super-tiles per SM pair (2 * 152 * 128 + 5 rows leaves some
    pairs a super-tile without a partner)."""
    if rows == 112847 and dims != DIMS[0]:
        pytest.skip("full row count on the full network only")
    net, _ = _net(dims, 64, 21)
    ld = (dims[0] + 7) // 8 * 8 + 8  # a row stride wider than the inputs
    X, _ = _bf16(rows, dims[0], 22, ld)
    net.set_fused(kind)
    Yf = net.forward(X[:, :dims[0]]).clone()
    net.set_fused(0)
    Yl = net.forward(X[:, :dims[0]])
    net.set_fused(1)
    torch.cuda.synchronize()
    assert torch.isfinite(Yf).all()
    assert torch.equal(Yf, Yl)


def test_inference_kernel_choice_is_checked():
    net, _ = _net(DIMS[0], 64, 1)
    for bad in (-1, 3):
        with pytest.raises(cc.CCError) as e:
            net.set_fused(bad)
        assert e.value.status == cc.ERR_INVALID_ARG
    net.set_fused(2)
    net.set_fused(0)


def test_fused_inference_writes_a_strided_output_and_nothing_else():
    """Y with a leading dimension wider than the output: the padding columns
    stay untouched, the rows match the dense result bit for bit."""
    dims = DIMS[0]
    rows = 777
    net, _ = _net(dims, 64, 23)
    X, _ = _bf16(rows, dims[0], 24, 264)
    dense = net.forward(X).clone()
    Y = torch.full((rows, dims[-1] + 4), 7.0, dtype=torch.float32, device="cuda")
    net.forward(X, out=Y[:, :dims[-1]])
    torch.cuda.synchronize()
    assert torch.equal(Y[:, :dims[-1]], dense)
    assert bool((Y[:, dims[-1]:] == 7.0).all())


@pytest.mark.parametrize("dims,B", [(DIMS[0], 1000), (DIMS[0], 4096), (DIMS[1], 77), (DIMS[2], 333)],
                         ids=["full-1000", "full-4096", "small-77", "one-hidden-333"])
def test_loss_and_gradient_match_oracle(dims, B):
    net, p = _net(dims, B, 5)
    X, Xn = _bf16(B, dims[0], 13, (dims[0] + 7) // 8 * 8)
    Tn = (0.3 * meshgen.normal(17, np.arange(B * dims[-1]))).reshape(B, dims[-1]).astype(np.float32)
    loss, g = net.loss_grad(X, torch.from_numpy(Tn).cuda())
    g = g.cpu().double().numpy()
    lo, go = mlp.loss_and_grad(p, dims, Xn, Tn.astype(np.float64), rounding=True)
    assert abs(loss - lo) <= 1e-5 * lo
    for l, (sw, sb) in enumerate(mlp.layer_slices(dims)):
        assert _rel(g[sw], go[sw]) <= 1e-3, (l, "W", _rel(g[sw], go[sw]))
        assert _rel(g[sb], go[sb]) <= 1e-3, (l, "b", _rel(g[sb], go[sb]))


def test_adam_step_matches_oracle():
    dims = DIMS[1]
    net, p = _net(dims, 16, 9)
    m = v = np.zeros_like(p)
    for t in range(1, 4):
        g = (meshgen.normal(40 + t, np.arange(p.size)) * 10.0 ** (-t)).astype(np.float32)
        net.adam_step(torch.from_numpy(g).cuda(), lr=1e-2)
        p, m, v = mlp.adam_step(p, g.astype(np.float64), m, v, t, 1e-2)
        np.testing.assert_allclose(net.get_params(), p, rtol=0, atol=1e-6)


def test_training_losses_follow_the_oracle():
    dims = DIMS[1]
    n, B, steps, lr = 96, 32, 5, 1e-3
    net, p = _net(dims, B, 21)
    X, Xn = _bf16(n, dims[0], 23, 32)
    Tn = (0.3 * meshgen.normal(29, np.arange(n * dims[-1]))).reshape(n, dims[-1]).astype(np.float32)
    idx = meshgen.batch_indices(31, 0, steps, B, n)
    losses = net.train(X, torch.from_numpy(Tn).cuda(), torch.from_numpy(idx).cuda(), B, lr=lr)
    m = v = np.zeros_like(p)
    for t in range(steps):
        lo, go = mlp.loss_and_grad(p, dims, Xn[idx[t]], Tn[idx[t]].astype(np.float64), rounding=True)
        assert abs(losses[t] - lo) <= 1e-3 * lo, (t, losses[t], lo)
        p, m, v = mlp.adam_step(p, go, m, v, t + 1, lr)


@pytest.mark.parametrize("dims", [DIMS[0], DIMS[1]], ids=["full", "small"])
def test_training_steps_replayed_from_one_graph_equal_single_steps(dims):
    """cc_mlp_train runs its first step directly and replays the others from
    one captured step (minibatch, loss slot and Adam step number read from a
    device step counter): a 7-step call gives the same bits, parameters and
    losses, as seven one-step calls."""
    n, B, steps = 3000, 512, 7
    X, _ = _bf16(n, dims[0], 41, (dims[0] + 7) // 8 * 8)
    Tn = (0.3 * meshgen.normal(43, np.arange(n * dims[-1]))).reshape(n, dims[-1]).astype(np.float32)
    T = torch.from_numpy(Tn).cuda()
    idx = torch.from_numpy(meshgen.batch_indices(47, 0, steps, B, n)).cuda()
    a, _ = _net(dims, B, 45)
    b, _ = _net(dims, B, 45)
    la = a.train(X, T, idx, B, lr=1e-3)
    lb = np.concatenate([b.train(X, T, idx[t:t + 1].contiguous(), B, lr=1e-3) for t in range(steps)])
    assert np.array_equal(la, lb)
    assert np.array_equal(a.get_params(), b.get_params())
    assert la[-1] < la[0]


def test_training_reduces_the_loss():
    dims = [30, 64, 64, 24]
    n, B = 4096, 512
    teacher, _ = _net(dims, 8, 77)
    X, _ = _bf16(n, dims[0], 41, 32)
    T = teacher.forward(X)
    net, _ = _net(dims, B, 78)
    idx = torch.from_numpy(meshgen.batch_indices(43, 0, 400, B, n)).cuda()
    losses = net.train(X, T, idx, B, lr=3e-3)
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.2 * losses[:5].mean()


# ---------------------------------------------------------------- inputs and targets
def _train_scenes(count, seed, lo=4, hi=7):
    return meshgen.training_boxes(count, seed, side_lo=lo, side_hi=hi)


@pytest.mark.parametrize("which", ["single", "union"])
def test_learned_inputs_and_targets_match_oracle(which):
    scenes = _train_scenes(3, 5) if which == "union" else [meshgen.stretch_box(5, 4, 4, E=3e5, nu=0.33,
                                                                               jitter_amount=0.05, seed=6)]
    m = cc.Mesh.from_scenes(scenes) if which == "union" else cc.Mesh.from_scene(scenes[0])
    m.color()
    m.build_subspace(2)
    X, T = m.learned_inputs(targets=True)
    X = X.cpu()[:, :learned.D_IN + 6].double().numpy()
    T = T.cpu().double().numpy()
    r0 = 0
    for sc in scenes:
        pb = fem.problem_from_scene(sc)
        topo = topology.Topology(pb.n, pb.tets, pb.free)
        rows, _, Fb = learned.features(pb, topo)
        sup, bases = subspace.build_local_bases(pb, topo, 2)
        To = learned.targets(pb, topo, sup, bases)
        nr = len(rows)
        Xg, Tg = X[r0:r0 + nr], T[r0:r0 + nr]
        np.testing.assert_array_equal(Xg[:, :256], Fb[:, :256])
        assert np.all(Xg[:, 258:] == 0.0)
        np.testing.assert_allclose(Xg[:, 256:258], Fb[:, 256:258], rtol=2.0 ** -7, atol=0)
        np.testing.assert_allclose(Tg, To, rtol=0, atol=1e-6 * max(1.0, np.abs(To).max()))
        np.testing.assert_array_equal(Tg == 0.0, To == 0.0)
        r0 += nr
    assert r0 == X.shape[0]


def test_inputs_reject_a_mesh_off_the_lattice():
    sc = meshgen.stretch_box(4, 4, 4, E=1e5, nu=0.3, jitter_amount=0.0)
    X = sc.X.copy()
    X[:, 0] *= 2.7        # cells 2.7 times longer in x: offsets leave the stencil
    m = cc.Mesh(X, sc.tets, sc.pinned, E=1e5, nu=0.3)
    m.color()
    with pytest.raises(cc.CCError) as e:
        m.learned_inputs()
    assert e.value.status == cc.ERR_INVALID_ARG


# ---------------------------------------------------------------- residuals and fallback
def _constant_net(pattern_seed=3):
    """A network whose output is its last bias (all weights zero): every
    vertex receives the same 64 blocks, exactly representable on both sides."""
    dims = meshgen.mlp_dims()
    p = np.zeros(meshgen.mlp_param_count(dims), dtype=np.float32)
    b = np.zeros(576, dtype=np.float32)
    st = learned.stencil()
    for s in range(64):
        c = 0.45 if s < 14 else 0.12
        blk = c * np.eye(3) + 0.02 * meshgen.normal(pattern_seed, np.arange(9 * s, 9 * s + 9)).reshape(3, 3)
        b[9 * s:9 * s + 9] = blk.ravel()
    p[mlp.layer_slices(dims)[-1][1]] = b
    net = cc.MLP(max_batch=256)
    net.set_params(p)
    return net, b.astype(np.float64)


def test_learned_bases_residuals_and_fallback_match_oracle():
    sc = meshgen.stretch_box(5, 4, 4, E=1e5, nu=0.3, factor=1.2, jitter_amount=0.05, seed=8)
    net, b = _constant_net()
    m = cc.Mesh.from_scene(sc)
    m.color()
    stats, rho = m.build_learned_subspace(net, tau=1.0, want_rho=True)
    rho = rho.cpu().numpy()
    pb = fem.problem_from_scene(sc)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    rows = np.flatnonzero(pb.free)
    sup, lb = learned.assemble(pb, topo, np.tile(b, (len(rows), 1)))
    out, F, rho_o = learned.with_fallback(pb, sup, lb, tau=1.0)
    np.testing.assert_allclose(rho, rho_o[rows], rtol=1e-10, atol=1e-14)
    near = np.abs(rho_o - 1.0) <= 1e-9
    Fg = {int(rows[r]) for r in range(len(rows)) if len(sup[rows[r]]) and rho[r] >= 1.0}
    assert {int(i) for i in F if not near[i]} == {i for i in Fg if not near[i]}
    assert stats["n_fallback"] == len(Fg) and 0 < len(Fg) < len(rows)
    sp, si, Ug = m.export("sup_ptr"), m.export("sup_idx"), m.export("U").reshape(-1, 3, 3)
    for i in rows:
        np.testing.assert_array_equal(si[sp[i]:sp[i + 1]], sup[i])
        if len(sup[i]):
            np.testing.assert_allclose(Ug[sp[i]:sp[i + 1]], out[i], rtol=0,
                                       atol=1e-10 * max(1.0, np.abs(out[i]).max()))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_learned_bases_solve_follows_the_oracle_sweep_by_sweep(precision):
    """Coloured CC with learned bases (the network's output assembled per
    vertex, Eq. 5 fallback to patch solves) against the oracle's solve with
    its own assembly of the same network output: the residual after every
    sweep and the final energy.  float64: 1e-8; mixed: 1e-4 of the start."""
    sc = meshgen.stretch_box(5, 4, 4, E=1e5, nu=0.3, factor=1.2, jitter_amount=0.05, seed=8)
    net, b = _constant_net()
    m = cc.Mesh.from_scene(sc)
    m.color()
    m.build_learned_subspace(net, tau=1.0)
    pb = fem.problem_from_scene(sc)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    rows = np.flatnonzero(pb.free)
    sup, lb = learned.assemble(pb, topo, np.tile(b, (len(rows), 1)))
    bases, _, _ = learned.with_fallback(pb, sup, lb, tau=1.0)
    iters = 25
    _, h_o = solvers.solve(pb, topo, sup, bases, sc.x0, kind="cc", tol=0.0, max_iters=iters)
    r = m.solve_step(cc.to_soa(sc.x0), precision=precision, tol=0.0, max_iters=iters, check_every=1,
                     history=True)
    hist = np.asarray(r.residuals[:iters + 1])
    go = np.asarray(h_o.grad_norm)
    assert len(hist) == len(go) and h_o.rel[-1] < 1e-2
    if precision == "fp64":
        # residuals fall seven orders of magnitude: compare to 1e-8 each, or to
        # 1e-10 of the start (the scale of the termination test, Sec. 4.1)
        np.testing.assert_allclose(hist, go, rtol=1e-8, atol=1e-10 * go[0])
        assert r.energy == pytest.approx(h_o.energy[-1], rel=1e-10)
    else:
        assert np.abs(hist - go).max() <= 1e-4 * go[0]
        assert r.energy == pytest.approx(h_o.energy[-1], rel=1e-6)


def test_learned_subspace_rejects_dynamic_meshes_and_wrong_networks():
    sc = meshgen.cantilever(2, 2, 4, cell=0.25, E=1e5, nu=0.3, h=0.01)
    m = cc.Mesh.from_scene(sc)
    m.color()
    net, _ = _constant_net()
    with pytest.raises(cc.CCError):
        m.build_learned_subspace(net)
    sq = cc.Mesh.from_scene(meshgen.stretch_box(3, 3, 3, E=1e5, nu=0.3))
    sq.color()
    with pytest.raises(cc.CCError):
        sq.build_learned_subspace(cc.MLP(30, 16, 1, 24, max_batch=8))


# ---------------------------------------------------------------- what the network gains
def _indices(seed):
    return lambda s0, cnt, batch, n: meshgen.batch_indices(seed, s0, cnt, batch, n)


def test_trained_network_gains_over_the_method_without_it():
    """Train on computed bases of 120 jittered boxes, evaluate on a held-out
    stretch box: the learned bases keep most vertices off the patch solve,
    converge like the computed ones (and like the oracle's curve), and far
    faster than coordinate descent, the method without any subspace."""
    scenes = _train_scenes(120, 2024, 4, 8)
    X, T, _ = cclearn.training_set(scenes)
    net = cc.MLP(max_batch=2048)
    net.set_params(meshgen.mlp_init(meshgen.mlp_dims(), 1))
    untrained = cc.MLP(max_batch=256)
    untrained.set_params(meshgen.mlp_init(meshgen.mlp_dims(), 1))
    losses, secs = cclearn.train(net, X, T, _indices(7), steps=3000, batch=2048, lr=1e-3)
    assert losses[-50:].mean() < 0.05 * losses[:10].mean()

    sc = meshgen.stretch_box(6, 6, 6, E=1e6, nu=0.3, factor=1.3, jitter_amount=0.05, seed=99)
    xs = cc.to_soa(sc.x0)

    def run(kind):
        m = cc.Mesh.from_scene(sc)
        m.color()
        st = None
        if kind == "learned":
            st, _ = m.build_learned_subspace(net)
        elif kind == "untrained":
            st, _ = m.build_learned_subspace(untrained)
        elif kind == "computed":
            m.build_subspace(2)
        x = xs.clone()
        r = m.solve_step(x, update="cd" if kind == "cd" else "cc", precision="mixed", tol=1e-6, max_iters=400,
                         history=True)
        return r, st

    rL, sL = run("learned")
    rU, sU = run("untrained")
    rC, _ = run("computed")
    rD, _ = run("cd")
    pb = fem.problem_from_scene(sc)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    sup, bases = subspace.build_local_bases(pb, topo, 2)
    _, hist = solvers.solve(pb, topo, sup, bases, sc.x0, kind="cc", tol=1e-6, max_iters=200)
    print(f"\nlearned: {rL.iterations} sweeps, fallback {sL['n_fallback']}/{sL['n_free']}; untrained fallback "
          f"{sU['n_fallback']}; computed {rC.iterations}; oracle computed {hist.iterations}; "
          f"cd {rD.iterations} (converged {rD.converged}); training {secs:.2f}s")
    assert rL.converged and rC.converged and hist.converged
    assert sL["n_fallback"] <= 0.25 * sL["n_free"]          # most patch solves avoided
    assert sU["n_fallback"] >= 2 * max(sL["n_fallback"], 1)  # training is what avoids them
    assert rL.iterations <= 1.5 * hist.iterations + 2        # near the oracle's computed-basis curve
    assert (not rD.converged) or rD.iterations >= 2 * rL.iterations


def test_parameters_round_trip_through_a_file(tmp_path):
    dims = meshgen.mlp_dims()
    a = cc.MLP(max_batch=256)
    p = meshgen.mlp_init(dims, 3)
    a.set_params(p)
    path = str(tmp_path / "net.bin")
    a.save(path)
    b = cc.MLP(max_batch=256)
    b.load(path)
    np.testing.assert_array_equal(b.get_params(), a.get_params())
    other = cc.MLP(hidden=128, max_batch=256)
    with pytest.raises(cc.CCError):
        other.load(path)
    for net in (a, b, other):
        net.close()
