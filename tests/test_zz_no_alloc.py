"""The allocation-free basis builder (cc_build_bases_noalloc).

It exists for callers that must not have device memory allocated on their
behalf (GPU memory owned entirely by their own pool allocator, or loops that
cannot absorb cudaMalloc's implicit synchronisation); it works in a static
16 MiB device array instead.  These tests call it through the C ABI and check
that two calls in a row reproduce the bases of cc_build_subspace (which uses
a cudaMalloc'ed workspace) within the tolerance the other basis tests use,
and that a support too large for the static array, or a max_support smaller
than a listed vertex's support, is rejected before any patch is solved.
"""
import ctypes

import numpy as np
import pytest

import meshgen
from oracle import fem

torch = pytest.importorskip("torch")
import paper_2510_12053_gb300 as cc  # noqa: E402

pytestmark = pytest.mark.gpu


def _inputs():
    scene = meshgen.stretch_box(6, 5, 4, E=1e5, nu=0.3, factor=1.2, jitter_amount=0.05, seed=3)
    m = cc.Mesh.from_scene(scene)
    m.color()
    m.build_subspace(2)
    sp, si, U_ref = m.export("sup_ptr"), m.export("sup_idx"), m.export("U")
    nb_ptr, nb_idx = m.export("nbr_ptr"), m.export("nbr_idx")
    n = scene.n
    # 3x3-block rows of the rest Hessian: 1-ring plus the diagonal, ascending
    H = fem.problem_from_scene(scene).hessian(scene.X).tocsr()
    row_ptr, cols = [0], []
    for j in range(n):
        row = sorted(list(nb_idx[nb_ptr[j]:nb_ptr[j + 1]]) + [j])
        cols.extend(row)
        row_ptr.append(len(cols))
    blocks = np.zeros((len(cols), 3, 3))
    for j in range(n):
        Hj = H[3 * j:3 * j + 3].toarray()
        for p in range(row_ptr[j], row_ptr[j + 1]):
            blocks[p] = Hj[:, 3 * cols[p]:3 * cols[p] + 3]
    verts = np.flatnonzero(scene.pinned == 0).astype(np.int32)
    max_support = int(np.max(np.diff(sp)))
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a, dtype=dt), device="cuda")
    d = dict(H=dev(blocks, np.float64), row_ptr=dev(row_ptr, np.int32), col=dev(cols, np.int32),
             verts=dev(verts, np.int32), sup_ptr=dev(sp, np.int32), sup_idx=dev(si, np.int32))
    m.close()
    return d, U_ref, max_support


def _call(d, max_support, U_out):
    stream = torch.cuda.current_stream().cuda_stream
    return cc.lib().cc_build_bases_noalloc(
        d["H"].data_ptr(), d["row_ptr"].data_ptr(), d["col"].data_ptr(), d["verts"].data_ptr(),
        int(d["verts"].numel()), d["sup_ptr"].data_ptr(), d["sup_idx"].data_ptr(), int(max_support),
        U_out.data_ptr(), ctypes.c_void_p(stream))


def test_noalloc_bases_match_allocating_builder_on_two_calls_in_a_row():
    assert torch.cuda.is_available()
    d, U_ref, max_support = _inputs()
    tol = 1e-10 * max(1.0, float(np.abs(U_ref).max()))
    for call in range(2):
        U_out = torch.zeros(U_ref.size, dtype=torch.float64, device="cuda")
        rc = _call(d, max_support, U_out)
        assert rc == cc.OK, (call, cc.lib().cc_last_error().decode())
        got = U_out.cpu().numpy()
        assert np.abs(got - U_ref).max() <= tol, call


def test_noalloc_rejects_supports_larger_than_its_static_workspace():
    assert torch.cuda.is_available()
    d, U_ref, _ = _inputs()
    U_out = torch.zeros(U_ref.size, dtype=torch.float64, device="cuda")
    rc = _call(d, 483, U_out)
    assert rc == cc.ERR_INVALID_ARG
    assert "16 MiB" in cc.lib().cc_last_error().decode()
    assert float(U_out.abs().max()) == 0.0


def test_noalloc_rejects_an_understated_max_support_before_solving():
    """max_support sizes each vertex's slice of the shared array; a caller
    that understates it (here by one) gets CC_ERR_INVALID_ARG from the support
    check that runs before the patch kernel, so U_out stays untouched."""
    assert torch.cuda.is_available()
    d, U_ref, max_support = _inputs()
    U_out = torch.zeros(U_ref.size, dtype=torch.float64, device="cuda")
    rc = _call(d, max_support - 1, U_out)
    assert rc == cc.ERR_INVALID_ARG
    assert "more than max_support" in cc.lib().cc_last_error().decode()
    torch.cuda.synchronize()
    assert float(U_out.abs().max()) == 0.0
    # the entry point stays usable: the next call with the true maximum succeeds
    rc = _call(d, max_support, U_out)
    assert rc == cc.OK, cc.lib().cc_last_error().decode()
    assert np.abs(U_out.cpu().numpy() - U_ref).max() <= 1e-10 * max(1.0, float(np.abs(U_ref).max()))
