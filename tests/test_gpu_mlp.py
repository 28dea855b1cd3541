"""Learned-subspace MLP on the GPU: the tcgen05 BF16 GEMM against an exact
product of the same BF16 inputs, and (below) the network's gradients against
the FP64 oracle."""
import numpy as np
import pytest

import meshgen

torch = pytest.importorskip("torch")
import paper_2510_12053_gb300 as cc  # noqa: E402

pytestmark = pytest.mark.gpu


def _bf16(rows, cols, seed, ld=None):
    a = meshgen.normal(seed, np.arange(rows * cols)).reshape(rows, cols).astype(np.float32)
    t = torch.zeros((rows, ld or cols), dtype=torch.bfloat16)
    t[:, :cols] = torch.from_numpy(a).to(torch.bfloat16)
    return t


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (300, 256, 320), (1000, 576, 256), (257, 192, 200),
                                   (8192, 256, 576), (64, 128, 1000)])
def test_gemm_bf16_matches_exact_product(M, N, K):
    assert torch.cuda.is_available()
    ld = (K + 7) // 8 * 8
    A = _bf16(M, K, 1 + M, ld)
    B = _bf16(N, K, 2 + N, ld)
    C = cc.gemm_bf16_tn(A.cuda()[:, :K], B.cuda()[:, :K])
    torch.cuda.synchronize()
    ref = A[:, :K].double() @ B[:, :K].double().T
    err = (C.cpu().double() - ref).abs().max().item()
    assert err <= 1e-5 * ref.abs().max().item() + 1e-6, err
