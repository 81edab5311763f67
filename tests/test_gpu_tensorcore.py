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


def test_completion_wait_timeout_is_reported_and_the_context_recovers():
    """The tensor-core kernels wait for their MMAs with a bounded number of tries.  With
    the first wait cut to zero tries (af_set_wait_limit test hook) every wait runs out:
    the GEMM sets its error flag and skips its epilogue, surrogate training returns
    AF_ERR_TIMEOUT, and each kernel still drains its MMAs before freeing tensor memory,
    so the context stays usable and the same GEMM succeeds once the default is back."""
    import synth
    lib = af.load()
    dev = torch.device("cuda")
    g = torch.Generator().manual_seed(3)
    A = torch.randn(128, 64, generator=g).to(torch.bfloat16)
    B = torch.randn(128, 64, generator=g).to(torch.bfloat16)
    ref = A.double().numpy() @ B.double().numpy().T
    Ad, Bd = A.to(dev), B.to(dev)
    D = torch.full((128, 128), float("nan"), device=dev)
    p = synth.config_tiny(n_ang=2, n_rad=2, patch_w=3)
    plan = af.Plan(p)
    iq = torch.from_numpy(synth.simulate(p, 300, seed=5)).to(dev)
    loss = torch.zeros(4, device=dev)
    plan.af_forward(iq, torch.from_numpy(p.initial_slowness()).to(dev), loss)
    torch.cuda.synchronize()
    assert lib.af_set_wait_limit(0) == af.AF_OK
    try:
        err = af.af_gemm_bf16(Ad, Bd, D)
        torch.cuda.synchronize()
        assert int(err) == 1
        assert torch.isnan(D).all()
        with pytest.raises(af.AfError) as ei:
            plan.surrogate_train(n_samples=128 * 32, epochs=1, tiles_per_step=32)
        assert ei.value.status == af.AF_ERR_TIMEOUT
    finally:
        lib.af_set_wait_limit(-1)
    err = af.af_gemm_bf16(Ad, Bd, D)
    torch.cuda.synchronize()
    assert int(err) == 0
    np.testing.assert_allclose(D.cpu().double().numpy(), ref, rtol=1e-5, atol=1e-4 * np.abs(ref).max())
    assert plan.af_sync_status() == af.AF_OK
    plan.close()
