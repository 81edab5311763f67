"""GPU test of af_cmpe_loss_noalloc, the entry point for callers that cannot
allocate device memory while they run (e.g. a real-time pipeline that reserves
its GPU memory at start-up, or a host framework that owns the allocator).

It is called through the C ABI twice in a row on the images of a planned
forward pass and must give the CMPE loss and active-term count of that pass
(loss within the parity tolerance of the other tests), without a plan.  This
file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process."""
import gc

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_06853_b300 as af  # noqa: E402
import synth  # noqa: E402

LOSS_TOL = 1e-4


@pytest.fixture(scope="module")
def planned_forward():
    p = synth.config_tiny()
    psi = synth.simulate(p, 2000, seed=20261205)
    dev = torch.device("cuda")
    plan = af.Plan(p)
    iq = torch.from_numpy(psi).to(dev)
    rng = np.random.default_rng(1)
    s = torch.from_numpy((1.0 / (1540.0 + 15.0 * rng.standard_normal((p.nz, p.nx)))).astype(np.float32)).to(dev)
    loss = torch.zeros(4, device=dev)
    plan.af_forward(iq, s, loss)
    torch.cuda.synchronize()
    _, _, n_active = plan.cmpe()
    return p, plan, plan.images(), float(loss[1]), n_active


def test_noalloc_cmpe_matches_planned_forward_twice(planned_forward):
    p, plan, B, L_ref, M_ref = planned_forward
    assert M_ref > 0
    dev = torch.device("cuda")
    for call in range(2):
        out = torch.full((1,), float("nan"), device=dev)
        n = torch.full((1,), -1, dtype=torch.int32, device=dev)
        af.af_cmpe_loss_noalloc(B, p.nsub, p.n_patch, p.patch_npix, p.rho_thresh, out, n)
        torch.cuda.synchronize()
        assert int(n) == M_ref, call
        assert abs(float(out) - L_ref) <= LOSS_TOL * abs(L_ref), (call, float(out), L_ref)


def test_noalloc_calls_leave_device_memory_unchanged(planned_forward):
    """The point of the entry point: after a first call, further calls change neither
    the device's free memory (cudaMemGetInfo) nor torch's allocated bytes.  Garbage
    left by earlier tests (reference cycles holding device tensors) is collected
    first, and the collector stays off while the calls are measured, so that only
    the entry point can change the counts."""
    p, plan, B, L_ref, M_ref = planned_forward
    dev = torch.device("cuda")
    out = torch.zeros(1, device=dev)
    n = torch.zeros(1, dtype=torch.int32, device=dev)
    af.af_cmpe_loss_noalloc(B, p.nsub, p.n_patch, p.patch_npix, p.rho_thresh, out, n)
    torch.cuda.synchronize()
    gc.collect()
    gc.disable()
    try:
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        for _ in range(5):
            af.af_cmpe_loss_noalloc(B, p.nsub, p.n_patch, p.patch_npix, p.rho_thresh, out, n)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_allocated() == alloc0
    finally:
        gc.enable()


def test_noalloc_after_a_different_call_uses_fresh_scratch(planned_forward):
    """A call on fewer patches gives the loss of those patches and leaves other scratch
    entries behind; the next full call must not be affected by them."""
    p, plan, B, L_ref, M_ref = planned_forward
    dev = torch.device("cuda")
    out = torch.zeros(1, device=dev)
    half = p.n_patch // 2
    af.af_cmpe_loss_noalloc(B[:, : half * p.patch_npix].contiguous(), p.nsub, half, p.patch_npix,
                            p.rho_thresh, out)
    torch.cuda.synchronize()
    # the planned forward's CMPE terms of the first `half` patches
    z, mask, _ = plan.cmpe()
    z, mask = z.cpu().numpy()[:half], mask.cpu().numpy()[:half].astype(bool)
    L_half = np.abs(np.angle(z[mask])).sum() / max(1, int(mask.sum()))
    assert abs(float(out) - L_half) <= LOSS_TOL * abs(L_half)
    af.af_cmpe_loss_noalloc(B, p.nsub, p.n_patch, p.patch_npix, p.rho_thresh, out)
    torch.cuda.synchronize()
    assert abs(float(out) - L_ref) <= LOSS_TOL * abs(L_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(planned_forward):
    p, plan, B, L_ref, M_ref = planned_forward
    out = torch.zeros(1, device=torch.device("cuda"))
    big = torch.zeros((p.nsub * p.nsub, af.AF_NOALLOC_MAX_PATCHES + 1), dtype=torch.complex64, device="cuda")
    with pytest.raises(af.AfError) as ei:
        af.af_cmpe_loss_noalloc(big, p.nsub, af.AF_NOALLOC_MAX_PATCHES + 1, 1, p.rho_thresh, out)
    assert ei.value.status == af.AF_ERR_UNSUPPORTED
    assert "exceeds the fixed scratch" in str(ei.value)
