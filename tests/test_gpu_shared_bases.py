"""Shared patch solves (cc_build_subspace on regular grids): vertices whose
patches are translated copies share one dense solve and copy its basis, and
every copy is checked against its own Eq. 5.  The bases must still equal the
oracle's own local-patch solves (Eq. 5 on each vertex's patch) to 1e-10, at
k = 2 on an unjittered box and at k = 3 on an unjittered dynamic cantilever
(the 3-ring, backward-Euler basis of the cantilever workload at a small size),
and the sharing must actually happen there (and not on a jittered mesh)."""
import numpy as np
import pytest

import meshgen
from oracle import fem, subspace, topology

torch = pytest.importorskip("torch")
import paper_2510_12053_gb300 as cc  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def _check_sampled(scene, k, samples=24, seed=5):
    pb = fem.problem_from_scene(scene)
    H0 = pb.hessian(pb.X)
    nb_ptr, nb_idx = topology.vertex_neighbors(pb.n, pb.tets)
    m = cc.Mesh.from_scene(scene)
    m.color()
    m.build_subspace(k)
    info = m.info()
    sp, si, Ug = m.export("sup_ptr"), m.export("sup_idx"), m.export("U").reshape(-1, 3, 3)
    free = np.flatnonzero(pb.free)
    pick = np.unique(free[(meshgen.uniform01(seed, np.arange(samples)) * len(free)).astype(int)])
    for i in pick:
        S = np.array([j for j in topology.k_ring(int(i), k, nb_ptr, nb_idx) if j != i and pb.free[j]])
        np.testing.assert_array_equal(si[sp[i]:sp[i + 1]], S)
        Ui = subspace.local_basis(H0, int(i), S).reshape(-1, 3, 3)
        np.testing.assert_allclose(Ug[sp[i]:sp[i + 1]], Ui, rtol=0, atol=1e-10 * max(1.0, np.abs(Ui).max()))
    m.close()
    return info


def test_regular_box_shares_patch_solves_and_matches_the_oracle():
    # cells of 1/8 (exact in binary): translated patches are bitwise equal
    scene = meshgen.stretch_box(10, 10, 10, E=1e5, nu=0.3, factor=1.2, size=1.25)
    info = _check_sampled(scene, 2)
    assert info.patch_shared > 0
    assert info.patch_solved + info.patch_shared == info.n_free


def test_jittered_box_solves_every_patch():
    scene = meshgen.stretch_box(10, 10, 10, E=1e5, nu=0.3, factor=1.2, size=1.25, jitter_amount=0.05, seed=1)
    info = _check_sampled(scene, 2, samples=8)
    assert info.patch_shared == 0
    assert info.patch_solved == info.n_free


def test_cantilever_three_ring_shared_bases_match_the_oracle():
    scene = meshgen.cantilever(6, 6, 40, cell=1.0 / 64.0, E=1e7, nu=0.45)
    info = _check_sampled(scene, 3, samples=16)
    assert info.support_max > 64      # 3-ring patches: above the shared-memory factor's 192 unknowns
    assert info.patch_shared > 0
