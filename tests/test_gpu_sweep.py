"""Global-speed initialisation sweep (Sec. II-C, III-A) with the dynamic CMPE grid,
run on the device by af_sweep, against the oracle, which moves the pixels with its
own implementation of the dynamic grid (or_dynamic_pixels, pinned in the oracle
tests by a point scatterer that stays on its patch centre at every speed)."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2608_06853_b300 as af  # noqa: E402
import synth  # noqa: E402
from paper_2608_06853_b300.sweep import global_speed_sweep  # noqa: E402


@pytest.fixture(scope="module")
def sweep_case():
    p = synth.config_tiny(cover_speeds=(1400.0, 1660.0))
    psi = synth.simulate(p, 20000, seed=20261207)
    return p, psi


def oracle_cmpe(p, psi, c0, pixels):
    q = dataclasses.replace(p, pix_x=pixels[0], pix_z=pixels[1])
    parts, _, _, M = oracle.Oracle(q).loss_grad(psi, np.full((p.nz, p.nx), 1.0 / c0), grad=False)
    return parts[1], M


@pytest.mark.parametrize("dynamic", [True, False])
def test_sweep_matches_oracle_at_every_speed(sweep_case, dynamic):
    p, psi = sweep_case
    plan = af.Plan(p)
    iq = torch.from_numpy(psi).cuda()
    speeds = np.arange(1400.0, 1661.0, 20.0)
    sp, cmpe, active, best = global_speed_sweep(plan, p, iq, speeds, dynamic=dynamic)
    o = oracle.Oracle(p)
    for k, c0 in enumerate(speeds):
        pixels = o.dynamic_pixels(c0, p.c_ref) if dynamic else (p.pix_x, p.pix_z)
        L, M = oracle_cmpe(p, psi, c0, pixels)
        # the correlation masks are decided independently (float vs float64): a few
        # terms within rounding of the threshold may differ
        assert abs(int(active[k]) - M) <= 3, (c0, active[k], M)
        assert cmpe[k] == pytest.approx(L, rel=2e-3), (c0, cmpe[k], L)
    print("dynamic" if dynamic else "static", dict(zip(sp.tolist(), np.round(cmpe, 4).tolist())), "best", best)
    assert speeds[0] < best < speeds[-1]


def test_sweep_restores_the_plan(sweep_case):
    """After a dynamic sweep the plan's own pixels are back: a forward pass gives the
    same loss as before the sweep."""
    p, psi = sweep_case
    plan = af.Plan(p)
    iq = torch.from_numpy(psi).cuda()
    s = torch.from_numpy(p.initial_slowness(1500.0)).cuda()
    l0, l1 = torch.zeros(4, device="cuda"), torch.zeros(4, device="cuda")
    plan.af_forward(iq, s, l0)
    plan.af_sweep(iq, [1420.0, 1500.0, 1640.0], p.c_ref, dynamic=True)
    plan.af_forward(iq, s, l1)
    torch.cuda.synchronize()
    np.testing.assert_allclose(l1.cpu().numpy(), l0.cpu().numpy(), rtol=1e-6)
    # a sweep whose moved pixels leave the grid box is refused on the host
    with pytest.raises(af.AfError) as ei:
        plan.af_sweep(iq, [3000.0], p.c_ref, dynamic=True)
    assert ei.value.status in (af.AF_ERR_ARG, af.AF_ERR_SHAPE)
