"""One plan, several forward + adjoint passes on different slowness maps.

Several kernels keep a device counter in the plan that the kernel itself returns to
zero for its next launch: the delay kernel's item counter, the ray adjoint's block
counter, and the CTA counts of the grid-statistics and CMPE-loss folds (the CTA that
finishes last folds the partial sums).  A counter left non-zero would make the next
launch skip its work and leave the previous results in place.  Without a lens there
is no exit-point solve, so nothing depends on a warm start: every pass of the reused
plan must give exactly the forward results of a fresh plan, and its gradient up to
the order of the DAS adjoint's float atomic adds (Sec. III-A, Eq. 1, 5, 10-12)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2608_06853_b300 as af  # noqa: E402
import synth  # noqa: E402


def speed_map(p, seed, amp):
    """Smooth speed perturbation around 1540 m/s, as slowness (float32)."""
    rng = np.random.default_rng(seed)
    zz, xx = np.meshgrid(np.linspace(0, 1, p.nz), np.linspace(0, 1, p.nx), indexing="ij")
    c = 1540.0 + amp * np.sin(2 * np.pi * (rng.uniform(0.5, 1.5) * xx + rng.uniform(0, 1))) \
        * np.cos(2 * np.pi * rng.uniform(0.5, 1.5) * zz)
    return (1.0 / c).astype(np.float32)


def one_pass(plan, iq, s):
    dev = iq.device
    st = torch.from_numpy(s).to(dev)
    loss = torch.zeros(4, device=dev)
    grad = torch.zeros_like(st)
    plan.af_forward(iq, st, loss)
    plan.af_adjoint(grad)
    torch.cuda.synchronize()
    T, a = plan.delays()
    z, m, n = plan.cmpe()
    return dict(T=T.cpu().numpy(), apod=a.cpu().numpy(), B=plan.images().cpu().numpy(),
                z=z.cpu().numpy(), mask=m.cpu().numpy(), n=n, loss=loss.cpu().numpy(),
                grad=grad.cpu().numpy().astype(np.float64))


def test_reused_plan_matches_fresh_plans():
    p = synth.config_tiny(lens_mode=af.AF_LENS_NONE)
    psi = synth.simulate(p, 1500, seed=31)
    iq = torch.from_numpy(psi).to(torch.device("cuda"))
    maps = [speed_map(p, 1, 30.0), speed_map(p, 2, 45.0), p.initial_slowness(), speed_map(p, 1, 30.0)]
    plan = af.Plan(p)
    prev = None
    for s in maps:
        got = one_pass(plan, iq, s)
        ref = one_pass(af.Plan(p), iq, s)
        for k in ("T", "apod", "B", "z", "mask", "loss"):
            assert np.array_equal(got[k], ref[k]), k
        assert got["n"] == ref["n"]
        g, gr = got["grad"], ref["grad"]
        assert np.linalg.norm(gr) > 0
        assert np.linalg.norm(g - gr) <= 1e-5 * np.linalg.norm(gr)
        if prev is not None:
            assert not np.array_equal(got["loss"], prev["loss"])       # the map changed
            assert not np.array_equal(got["T"], prev["T"])
        prev = got


@pytest.mark.parametrize("lens_mode", [af.AF_LENS_NONE, af.AF_LENS_BENT_RAY])
def test_ray_adjoint_flush_window_does_not_change_the_gradient(lens_mode):
    """The ray adjoint adds its shared-memory integer grids into the global one when
    the rays since the last flush would pass the fixed-point window by their summed
    |dL/dT|; on a small problem that never happens before the end.  Windows of 1,
    0.5 and 0 rays make every CTA flush before each of its blocks after the first:
    the integer sums, hence dL/ds, are unchanged up to the DAS adjoint's float-atomic
    order (Eq. 1 adjoint, Sec. III-A).  The loss may move by rounding only: with the
    lens, later passes start the exit-point solve from the previous angles."""
    p = synth.config_tiny(lens_mode=lens_mode)
    psi = synth.simulate(p, 1500, seed=33)
    iq = torch.from_numpy(psi).to(torch.device("cuda"))
    s = speed_map(p, 3, 40.0)
    plan = af.Plan(p)
    ref = one_pass(plan, iq, s)
    assert np.linalg.norm(ref["grad"]) > 0
    for window in (1.0, 0.5, 0.0):
        plan.set_ray_flush_budget(window)
        got = one_pass(plan, iq, s)
        np.testing.assert_allclose(got["loss"], ref["loss"], rtol=1e-6)
        assert np.linalg.norm(got["grad"] - ref["grad"]) <= 1e-6 * np.linalg.norm(ref["grad"]), window
    with pytest.raises(af.AfError):
        plan.set_ray_flush_budget(-1.0)
    plan.set_ray_flush_budget(1e30)                      # capped at the scale's window
    got = one_pass(plan, iq, s)
    assert np.linalg.norm(got["grad"] - ref["grad"]) <= 1e-6 * np.linalg.norm(ref["grad"])
