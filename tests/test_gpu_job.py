"""Autofocus jobs from host memory (af_job_submit): upload, N_i iterations of the
method (Sec. III-A) and read back in one call, with the next job's upload under the
running job's iterations.  Each job must give what the same iterations give through
the device-pointer entry points (af_iterate from the same map, moments at zero)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_06853_b300 as af  # noqa: E402
import synth  # noqa: E402

N_ITER = 4


@pytest.fixture(scope="module")
def job_case():
    p = synth.config_tiny()
    psi_a = synth.simulate(p, 3000, seed=11)
    psi_b = synth.simulate(p, 3000, seed=12)
    rng = np.random.default_rng(5)
    s0 = [(1.0 / (1540.0 + 15.0 * rng.standard_normal((p.nz, p.nx)))).astype(np.float32) for _ in range(3)]
    return p, (psi_a, psi_b), s0


def device_run(p, psi, s0, n_iter, iq_dtype=af.AF_IQ_C64, iq=None, scale=None):
    plan = af.Plan(p, iq_dtype=iq_dtype)
    dev = torch.device("cuda")
    if iq is None:
        iq = torch.from_numpy(psi).to(dev)
    s = torch.from_numpy(s0).to(dev)
    g, m, v = torch.zeros_like(s), torch.zeros_like(s), torch.zeros_like(s)
    loss = torch.zeros(4, device=dev)
    for it in range(1, n_iter + 1):
        plan.af_iterate(iq, s, g, m, v, it, loss, scale)
    torch.cuda.synchronize()
    return s.cpu().numpy(), loss.cpu().numpy()


def assert_same_run(p, s_job, loss_job, s_ref, loss_ref):
    """The same kernels on the same inputs.  The float atomics of the DAS adjoint may
    add dL/dT in another order, and Adam turns a sign change of a near-zero gradient
    into a whole step, so the maps agree to a fraction of a step almost everywhere
    and to two steps at most."""
    step = p.lr * p.c_unit / 1540.0 ** 2                 # one Adam step in slowness
    d = np.abs(s_job.astype(np.float64) - s_ref)
    assert d.max() <= 2.0 * step and np.median(d) <= 0.01 * step
    np.testing.assert_allclose(loss_job, loss_ref, rtol=1e-2)


def test_three_jobs_match_the_device_path(job_case):
    """Three jobs of two acquisitions: every buffer is used twice, the third job's
    upload waits for the first job to finish."""
    p, (psi_a, psi_b), s0 = job_case
    plan = af.Plan(p)
    plan.job_reserve()
    inputs = [(psi_a, s0[0]), (psi_b, s0[1]), (psi_a, s0[2])]
    h_iq = {id(x): torch.from_numpy(x).pin_memory() for x in (psi_a, psi_b)}
    outs = []
    for psi, s_init in inputs:
        h_s = torch.from_numpy(s_init).pin_memory()
        h_out = torch.empty(p.nz, p.nx).pin_memory()
        h_loss = torch.empty(4).pin_memory()
        plan.job_submit(h_iq[id(psi)], h_s, N_ITER, h_out, h_loss)
        outs.append((h_out, h_loss))
    plan.job_wait()
    for (psi, s_init), (h_out, h_loss) in zip(inputs, outs):
        s_ref, loss_ref = device_run(p, psi, s_init, N_ITER)
        assert np.all(np.isfinite(h_out.numpy()))
        assert not np.array_equal(h_out.numpy(), s_init)             # the map moved
        assert_same_run(p, h_out.numpy(), h_loss.numpy(), s_ref, loss_ref)


def test_job_from_pageable_memory_and_16_bit_storage(job_case):
    """Pageable host buffers (copies serialise, results unchanged) and BF16 channel
    data with its per-transmit scale."""
    p, (psi_a, _), s0 = job_case
    r = torch.view_as_real(torch.from_numpy(psi_a))
    scale = r.abs().amax(dim=(1, 2, 3)).clamp_min(1e-30).float().contiguous()
    q = (r / scale[:, None, None, None]).to(torch.bfloat16).contiguous()
    plan = af.Plan(p, iq_dtype=af.AF_IQ_BF16)
    h_out, h_loss = torch.empty(p.nz, p.nx), torch.empty(4)
    plan.job_submit(q, torch.from_numpy(s0[0]), N_ITER, h_out, h_loss, h_iq_scale=scale)
    plan.job_wait()
    s_ref, loss_ref = device_run(p, None, s0[0], N_ITER, af.AF_IQ_BF16, iq=q.cuda(), scale=scale.cuda())
    assert_same_run(p, h_out.numpy(), h_loss.numpy(), s_ref, loss_ref)


def test_job_argument_checks(job_case):
    p, (psi_a, _), s0 = job_case
    plan = af.Plan(p)
    h_iq = torch.from_numpy(psi_a)
    h_s = torch.from_numpy(s0[0])
    with pytest.raises(ValueError, match="bytes"):
        plan.job_submit(h_iq[:-1].contiguous(), h_s, 1)
    with pytest.raises(TypeError):
        plan.job_submit(h_iq.cuda(), h_s, 1)
    with pytest.raises(af.AfError):
        plan.job_submit(h_iq, h_s, 0)
    plan.job_wait()                                       # nothing submitted: returns at once
