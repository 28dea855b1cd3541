"""A caller's colouring (cc_set_colors): the Kuhn grid's lattice colouring
(i + j + k) mod 4 gives four colour phases per sweep instead of greedy's
eight.  The GPU's coloured sweeps with it must follow the oracle's sweeps
with the same colouring (float64 to 1e-12, mixed within the mixed
tolerances), and an invalid colouring must be refused."""
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


def _scene(dims=(6, 5, 7)):
    return meshgen.stretch_box(*dims, E=1e5, nu=0.3, factor=1.4, jitter_amount=0.05, seed=6)


def _oracle(sc, dims):
    pb = fem.problem_from_scene(sc)
    topo = topology.Topology(pb.n, pb.tets, pb.free, colors=meshgen.lattice_colors(*dims))
    sup, U = subspace.build_local_bases(pb, topo, 2)
    return pb, topo, sup, U


def test_lattice_coloured_fp64_sweep_matches_the_oracle():
    dims = (6, 5, 7)
    sc = _scene(dims)
    pb, topo, sup, U = _oracle(sc, dims)
    x_o = solvers.sweep(pb, topo, sup, U, sc.x0, None, "cc", "colored")
    m = cc.Mesh.from_scene(sc)
    m.set_colors(meshgen.lattice_colors(*dims))
    assert m.info().num_colors == 4
    m.build_subspace(2)
    xd = cc.to_soa(sc.x0)
    m.sweep(xd, update="cc", schedule="colored", precision="fp64")
    np.testing.assert_allclose(cc.from_soa(xd), x_o, rtol=0, atol=1e-12 * np.abs(x_o).max())
    m.close()


def test_lattice_coloured_mixed_trajectory_matches_the_oracle():
    dims = (6, 5, 7)
    sc = _scene(dims)
    pb, topo, sup, U = _oracle(sc, dims)
    m = cc.Mesh.from_scene(sc)
    m.set_colors(meshgen.lattice_colors(*dims))
    m.build_subspace(2)
    x = sc.x0.copy()
    xd = cc.to_soa(sc.x0)
    for _ in range(20):
        x = solvers.sweep(pb, topo, sup, U, x, None, "cc", "colored")
        m.sweep(xd, update="cc", schedule="colored", precision="mixed")
        E, _, gn = m.energy_grad(xd, precision="fp64", want_grad=False)
        assert E == pytest.approx(pb.energy(x), rel=1e-4)
        assert gn == pytest.approx(np.linalg.norm(pb.gradient(x)[pb.free]), rel=1e-4)
    diag = np.linalg.norm(sc.X.max(0) - sc.X.min(0))
    assert np.abs(cc.from_soa(xd) - x).max() <= 1e-5 * diag
    m.close()


def test_invalid_colourings_are_refused():
    dims = (3, 3, 3)
    sc = _scene(dims)
    m = cc.Mesh.from_scene(sc)
    with pytest.raises(cc.CCError):
        m.set_colors(np.zeros(sc.n, np.int32))          # neighbours alike
    bad = meshgen.lattice_colors(*dims).copy()
    with pytest.raises(cc.CCError):
        m.set_colors(bad, num_colors=3)                  # a colour out of range
    m.set_colors(bad)
    m.close()
