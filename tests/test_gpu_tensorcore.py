"""The tcgen05 BF16 GEMM (tensor-memory accumulators) against float64 numpy on
the same bf16-rounded operands, in all four operand-major combinations."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_06853_b300 as af  # noqa: E402


@pytest.mark.parametrize("a_mn,b_mn", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_gemm_bf16_matches_float64(a_mn, b_mn):
    M, N, K = 256, 384, 192
    dev = torch.device("cuda")
    g = torch.Generator().manual_seed(1 + 2 * a_mn + b_mn)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ref = A.double().numpy() @ B.double().numpy().T
    Ad = (A.t().contiguous() if a_mn else A).to(dev)
    Bd = (B.t().contiguous() if b_mn else B).to(dev)
    D = torch.full((M, N), float("nan"), device=dev)
    err = af.af_gemm_bf16(Ad, Bd, D, a_mn_major=a_mn, b_mn_major=b_mn)
    torch.cuda.synchronize()
    assert int(err) == 0
    out = D.cpu().double().numpy()
    assert np.isfinite(out).all()
    np.testing.assert_allclose(out, ref, rtol=1e-5, atol=1e-4 * np.abs(ref).max())


def test_gemm_rejects_bad_shapes():
    dev = torch.device("cuda")
    A = torch.zeros(100, 64, dtype=torch.bfloat16, device=dev)
    B = torch.zeros(128, 64, dtype=torch.bfloat16, device=dev)
    D = torch.zeros(100, 128, device=dev)
    with pytest.raises(af.AfError) as ei:
        af.af_gemm_bf16(A, B, D)
    assert ei.value.status == af.AF_ERR_SHAPE
