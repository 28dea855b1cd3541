"""Pins of the learned-subspace oracle (``oracle/mlp.py``, ``oracle/learned.py``):
finite differences, an independent autograd implementation, closed forms of
Adam, GELU and bfloat16 rounding, lattice symmetries of the stencil, inputs
and targets, and degenerate cases of the fallback rule."""
import numpy as np
import pytest
import torch

import meshgen
from oracle import fem, learned, material, mlp, subspace, topology


# ---------------------------------------------------------------- bfloat16 --
def test_bf16_rounding_closed_forms():
    one = 1.0
    assert mlp.bf16(one) == 1.0
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0                    # tie -> even (1.0)
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6     # tie -> even (mantissa 2)
    assert mlp.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert mlp.bf16(-2.5) == -2.5
    assert mlp.bf16(0.0) == 0.0


def test_bf16_matches_torch_conversion():
    x = meshgen.normal(11, np.arange(20000)) * np.exp(meshgen.normal(12, np.arange(20000)) * 3)
    x32 = x.astype(np.float32)
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x32), ref)


# -------------------------------------------------------------------- GELU --
def test_gelu_closed_forms():
    z = np.linspace(-6, 6, 241)
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert mlp.gelu_grad(np.array(0.0)) == 0.5
    np.testing.assert_allclose(mlp.gelu(z) - mlp.gelu(-z), z, rtol=0, atol=1e-14)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, rtol=0, atol=1e-8)
    ref = torch.nn.functional.gelu(torch.from_numpy(z), approximate="none").numpy()
    np.testing.assert_allclose(mlp.gelu(z), ref, rtol=1e-14, atol=1e-15)


# --------------------------------------------------------------------- MLP --
def _tiny(seed=5):
    dims = [6, 5, 5, 4]
    p = meshgen.mlp_init(dims, seed, out_scale=1.0).astype(np.float64)
    p += 0.1 * meshgen.normal(seed + 1, np.arange(len(p)))
    X = meshgen.normal(seed + 2, np.arange(7 * 6)).reshape(7, 6)
    T = meshgen.normal(seed + 3, np.arange(7 * 4)).reshape(7, 4)
    return dims, p, X, T


def test_mlp_gradient_matches_finite_differences():
    dims, p, X, T = _tiny()
    _, g = mlp.loss_and_grad(p, dims, X, T, rounding=False)
    h = 1e-6
    fd = np.zeros_like(p)
    for k in range(len(p)):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (mlp.loss_and_grad(p + e, dims, X, T, rounding=False)[0]
                 - mlp.loss_and_grad(p - e, dims, X, T, rounding=False)[0]) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-6 * np.max(np.abs(g))


def test_mlp_matches_autograd_at_full_width():
    dims = meshgen.mlp_dims()
    p = meshgen.mlp_init(dims, 3).astype(np.float64)
    X = meshgen.normal(4, np.arange(16 * dims[0])).reshape(16, dims[0])
    T = 0.1 * meshgen.normal(5, np.arange(16 * dims[-1])).reshape(16, dims[-1])
    loss, g = mlp.loss_and_grad(p, dims, X, T, rounding=False)
    pt = torch.tensor(p, requires_grad=True)
    h = torch.from_numpy(X)
    o = 0
    for l in range(len(dims) - 1):
        W = pt[o:o + dims[l + 1] * dims[l]].view(dims[l + 1], dims[l])
        o += dims[l + 1] * dims[l]
        b = pt[o:o + dims[l + 1]]
        o += dims[l + 1]
        h = h @ W.T + b
        if l < len(dims) - 2:
            h = torch.nn.functional.gelu(h, approximate="none")
    lt = torch.mean((h - torch.from_numpy(T)) ** 2)
    lt.backward()
    assert abs(loss - lt.item()) <= 1e-13 * lt.item()
    ref = pt.grad.numpy()
    assert np.max(np.abs(g - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_rounded_network_stays_within_bfloat16_error():
    dims = meshgen.mlp_dims()
    p = meshgen.mlp_init(dims, 3).astype(np.float64)
    X = meshgen.normal(4, np.arange(32 * dims[0])).reshape(32, dims[0])
    T = 0.1 * meshgen.normal(5, np.arange(32 * dims[-1])).reshape(32, dims[-1])
    Y64, _ = mlp.forward(p, dims, X, rounding=False)
    Y16, _ = mlp.forward(p, dims, X, rounding=True)
    rel = np.linalg.norm(Y16 - Y64) / np.linalg.norm(Y64)
    assert 1e-4 < rel < 3e-2           # rounding happened, at bfloat16 size
    _, g64 = mlp.loss_and_grad(p, dims, X, T, rounding=False)
    _, g16 = mlp.loss_and_grad(p, dims, X, T, rounding=True)
    for sw, sb in mlp.layer_slices(dims):
        assert np.linalg.norm(g16[sw] - g64[sw]) <= 5e-2 * np.linalg.norm(g64[sw])


def test_adam_closed_forms():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p0 = np.array([1.0, 2.0, 3.0, 4.0])
    m = v = np.zeros(4)
    lr, eps = 1e-2, 1e-8
    p = p0
    for t in range(1, 6):   # constant gradient: bias-corrected m, v equal g, g^2
        p, m, v = mlp.adam_step(p, g, m, v, t, lr, eps=eps)
        np.testing.assert_allclose(p, p0 - t * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-13)
    assert p[3] == 4.0


def test_adam_trains_the_tiny_network():
    dims, p, X, T = _tiny(9)
    m = v = np.zeros_like(p)
    l0 = mlp.loss_and_grad(p, dims, X, T, rounding=False)[0]
    for t in range(1, 301):
        loss, g = mlp.loss_and_grad(p, dims, X, T, rounding=False)
        p, m, v = mlp.adam_step(p, g, m, v, t, 1e-2)
    assert loss < 0.2 * l0


# ---------------------------------------------------------------- stencil --
def test_stencil_is_the_kuhn_two_ring():
    st = learned.stencil()
    assert len(st) == learned.SLOTS == 64 and len(set(st)) == 64
    one = [o for o in st[:14]]
    pos = [o for o in one if min(o) >= 0]
    # 1-ring of the consistent-diagonal split: the 7 nonzero 0/1 vectors and negatives
    assert sorted(pos) == sorted(o for o in np.ndindex(2, 2, 2) if any(o))
    assert sorted(one) == sorted(pos + [tuple(-c for c in o) for o in pos])
    sums = {tuple(a + b for a, b in zip(u, w)) for u in one for w in one}
    assert set(st[14:]) == sums - set(one) - {(0, 0, 0)}
    assert set(st) == {tuple(-c for c in o) for o in st}
    assert st[:14] == sorted(st[:14]) and st[14:] == sorted(st[14:])


def _grid(nx, ny, nz, jit=0.0, nu=0.3, E=1e5, seed=2, scale=1.0):
    sc = meshgen.stretch_box(nx, ny, nz, E=E, nu=nu, factor=1.1, jitter_amount=jit, seed=seed)
    X = sc.X * scale
    pb = fem.Problem(X, sc.tets, sc.pinned, material.Model("snh", E, nu), rho=1000.0)
    return sc, pb, topology.Topology(pb.n, pb.tets, pb.free)


def _vid(sc, i, j, k):
    nx, ny, _ = sc.dims
    return i + (nx + 1) * (j + (ny + 1) * k)


def test_features_of_an_unjittered_lattice():
    sc, pb, topo = _grid(6, 5, 5, E=1e5, nu=0.3)
    rows, F, Fb = learned.features(pb, topo)
    cell = sc.cell
    r = {int(v): k for k, v in enumerate(rows)}
    c = _vid(sc, 3, 2, 2)
    assert learned.lattice_spacing(pb.X, topo, c) == pytest.approx(cell, rel=1e-15)
    f = F[r[c]]
    assert np.all(f[3:256:4] == 1.0)                 # every slot holds a free vertex
    assert np.max(np.abs(np.delete(f[:256], np.s_[3::4]))) < 1e-12
    assert f[256] == pytest.approx((5.0 - 5.5) / 1.5) and f[257] == pytest.approx(-1.0)
    # vertex next to the clamped face x = 0: offsets with dx = -2 are absent, dx = -1 pinned
    b = _vid(sc, 1, 2, 2)
    st = learned.stencil()
    for s, o in enumerate(st):
        state = F[r[b], 4 * s + 3]
        expect = 0.0 if o[0] == -2 else (-1.0 if o[0] == -1 else 1.0)
        assert state == expect, (o, state)


def test_features_corner_vertex_keeps_the_in_box_offsets():
    sc, pb, topo = _grid(4, 4, 4)
    table = learned.slot_table()
    c = _vid(sc, 1, 0, 0)        # on three... two faces (y = 0, z = 0), next to the clamp
    got = {s for _, s, _ in learned.offsets(pb.X, topo, c, table)}
    want = {s for o, s in table.items() if o[1] >= 0 and o[2] >= 0 and o[0] >= -1}
    assert got == want


def test_features_are_invariant_to_scale_and_translation():
    sc, pb, topo = _grid(4, 4, 3, jit=0.05)
    _, F1, _ = learned.features(pb, topo)
    pb2 = fem.Problem(pb.X * 4.0 + np.array([3.0, -1.0, 0.5]), pb.tets, sc.pinned, pb.model, rho=1000.0)
    _, F2, _ = learned.features(pb2, topo)
    np.testing.assert_allclose(F2, F1, rtol=0, atol=1e-12)
    assert np.max(np.abs(F1[:, :256:4])) > 0.05      # jitter is visible


def test_targets_have_point_symmetry_and_translation_invariance():
    sc, pb, topo = _grid(8, 7, 7, nu=0.35)
    sup = topo.supports(2)
    H = pb.hessian(pb.X)
    table = learned.slot_table()
    st = learned.stencil()
    rowsU = {}
    for v in (_vid(sc, 3, 3, 3), _vid(sc, 4, 3, 3)):
        U = subspace.local_basis(H, v, sup[v])
        slot_of = {j: s for j, s, _ in learned.offsets(pb.X, topo, v, table)}
        row = np.zeros((64, 3, 3))
        for a, j in enumerate(sup[v]):
            row[slot_of[int(j)]] = U[a]
        rowsU[v] = row
        for s, o in enumerate(st):      # U(i + o) = U(i - o) under the lattice's point symmetry
            t = table[tuple(-c for c in o)]
            np.testing.assert_allclose(row[s], row[t], rtol=0, atol=1e-12)
    a, b = rowsU.values()
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
    assert np.abs(a[:14]).max() > 0.1


def test_targets_and_assembly_round_trip():
    sc, pb, topo = _grid(4, 3, 3, jit=0.05)
    sup, bases = subspace.build_local_bases(pb, topo, 2)
    Y = learned.targets(pb, topo, sup, bases)
    sup2, back = learned.assemble(pb, topo, Y)
    for i in range(pb.n):
        np.testing.assert_array_equal(sup2[i], sup[i])
        np.testing.assert_array_equal(back[i], bases[i])
    assert np.count_nonzero(np.abs(Y).sum(axis=1)) == int(pb.free.sum())


# ---------------------------------------------------------------- fallback --
def _fallback_case():
    sc = meshgen.stretch_box(4, 3, 3, E=1e5, nu=0.3, factor=1.2, jitter_amount=0.05, seed=4)
    pb = fem.problem_from_scene(sc)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    sup, bases = subspace.build_local_bases(pb, topo, 2)
    return sc, pb, topo, sup, bases


def test_basis_residual_closed_forms():
    """rho = 0 for the computed basis, 1 for U = 0 (coordinate descent), and
    |1 - c| for c times the computed basis (Eq. 5 is linear in U)."""
    sc, pb, topo, sup, bases = _fallback_case()
    free = pb.free
    rho = learned.basis_residual(pb, sup, bases)
    assert np.max(rho[free]) < 1e-12
    rho0 = learned.basis_residual(pb, sup, [np.zeros_like(U) for U in bases])
    np.testing.assert_allclose(rho0[free], 1.0, rtol=0, atol=1e-15)
    for c in (0.5, 1.25, -1.0):
        rc = learned.basis_residual(pb, sup, [c * U for U in bases])
        np.testing.assert_allclose(rc[free], abs(1 - c), rtol=0, atol=1e-12)
    assert np.all(rho[~free] == 0.0)


def test_fallback_set_thresholds():
    sc, pb, topo, sup, bases = _fallback_case()
    F, _ = learned.fallback_set(pb, sup, bases)
    assert len(F) == 0
    F0, _ = learned.fallback_set(pb, sup, [np.zeros_like(U) for U in bases])
    np.testing.assert_array_equal(F0, np.flatnonzero(pb.free))    # ties fall back
    F2, _ = learned.fallback_set(pb, sup, [2.5 * U for U in bases], tau=1.0)
    np.testing.assert_array_equal(F2, np.flatnonzero(pb.free))    # rho = 1.5
    F3, _ = learned.fallback_set(pb, sup, [1.5 * U for U in bases], tau=0.6)
    assert len(F3) == 0


def test_fallback_replaces_exactly_the_failing_vertices_with_computed_bases():
    sc, pb, topo, sup, bases = _fallback_case()
    bad = subspace.add_noise(bases, 0.05, seed=9)
    out, F, rho = learned.with_fallback(pb, sup, bad)
    assert 0 < len(F) < int(pb.free.sum())
    Fs = set(int(i) for i in F)
    for i in np.flatnonzero(pb.free):
        ref = bases[i] if int(i) in Fs else bad[i]
        np.testing.assert_allclose(out[i], ref, rtol=0, atol=1e-12)
        assert (rho[i] >= 1.0) == (int(i) in Fs)
    after = learned.basis_residual(pb, sup, out)
    assert np.max(after[pb.free]) < 1.0
