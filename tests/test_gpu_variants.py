"""Kernel variants of the sweep (cc_set_sweep_variant) compute the same
method: the condensation fused into the coupling kernel gives results bit
for bit equal to the separate launch (same float64 arithmetic per vertex,
whichever CTA runs it); block rows formed from the positions agree with the
per-tet-store gather within float32 rounding, and every variant follows the
oracle's mixed-precision trajectory within the mixed tolerances."""
import numpy as np
import pytest

import meshgen
from oracle import fem, solvers, subspace, topology

torch = pytest.importorskip("torch")
import paper_2510_12053_gb300 as cc  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _scene():
    return meshgen.stretch_box(7, 6, 5, E=1e5, nu=0.3, factor=1.4, jitter_amount=0.05, seed=4)


def _run(scene, variant, sweeps, precision="mixed", update="cc", threads=0):
    m = cc.Mesh.from_scene(scene)
    m.color()
    m.build_subspace(2)
    m.set_sweep_variant(*variant)
    if threads:
        m.set_launch_shape(couple_threads=threads)
    xd = cc.to_soa(scene.x0)
    st = None
    for _ in range(sweeps):
        st = m.sweep(xd, update=update, schedule="colored", precision=precision)
    torch.cuda.synchronize()
    m.close()
    return cc.from_soa(xd), st


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("update", ["cc", "jgs2"])
@pytest.mark.parametrize("threads", [64, 128, 256])
def test_fused_condensation_is_bit_identical(precision, update, threads):
    sc = _scene()
    xa, sa = _run(sc, (0, 0), 4, precision, update, threads)
    xb, sb = _run(sc, (0, 1), 4, precision, update, threads)
    np.testing.assert_array_equal(xa, xb)
    assert (sa.fallback_empty, sa.fallback_reduced, sa.fallback_schur) == \
           (sb.fallback_empty, sb.fallback_reduced, sb.fallback_schur)


def test_row_build_variants_follow_the_oracle():
    sc = _scene()
    pb = fem.problem_from_scene(sc)
    topo = topology.Topology(pb.n, pb.tets, pb.free)
    sup, U = subspace.build_local_bases(pb, topo, 2)
    x_o, _ = solvers.solve(pb, topo, sup, U, sc.x0, kind="cc", tol=0.0, max_iters=10)
    diag = np.linalg.norm(sc.X.max(0) - sc.X.min(0))
    xs = {}
    for variant in [(0, 0), (1, 0), (1, 1)]:
        x, _ = _run(sc, variant, 10)
        assert np.abs(x - x_o).max() <= 1e-5 * diag, variant
        xs[variant] = x
    step = np.abs(x_o - sc.x0).max()
    assert np.abs(xs[(1, 0)] - xs[(0, 0)]).max() <= 1e-5 * step
    np.testing.assert_array_equal(xs[(1, 0)], xs[(1, 1)])


def test_variant_switch_rejects_bad_values():
    m = cc.Mesh.from_scene(_scene())
    with pytest.raises(cc.CCError):
        m.set_sweep_variant(2, 0)
    with pytest.raises(cc.CCError):
        m.set_sweep_variant(0, -2)
    m.close()
