"""Global-speed initialisation sweep (Sec. II-C, III-A) with the dynamic CMPE grid."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2608_06853_b300 as af  # noqa: E402
import synth  # noqa: E402
from paper_2608_06853_b300.sweep import dynamic_pixels, global_speed_sweep  # noqa: E402


def test_dynamic_pixels_scale_depth_and_spacing():
    p = synth.config_tiny()
    x0, z0 = dynamic_pixels(p, p.c_ref)
    np.testing.assert_allclose(x0, p.pix_x, atol=1e-7)
    np.testing.assert_allclose(z0, p.pix_z, atol=1e-7)
    x1, z1 = dynamic_pixels(p, 1.1 * p.c_ref)
    d0 = np.hypot(p.pix_x[1] - p.pix_x[0], p.pix_z[1] - p.pix_z[0])
    d1 = np.hypot(x1[1] - x1[0], z1[1] - z1[0])
    assert d1 == pytest.approx(1.1 * d0, rel=1e-5)


def test_sweep_matches_oracle_and_picks_an_interior_speed():
    p = synth.config_tiny(cover_speeds=(1400.0, 1660.0))
    psi = synth.simulate(p, 20000, seed=20261207)
    dev = torch.device("cuda")
    plan = af.Plan(p)
    iq = torch.from_numpy(psi).to(dev)
    speeds = np.arange(1400.0, 1661.0, 20.0)
    sp, cmpe, active, best = global_speed_sweep(plan, p, iq, speeds, dynamic=True)
    _, cmpe_static, _, best_static = global_speed_sweep(plan, p, iq, speeds, dynamic=False)
    print("dynamic", dict(zip(sp.tolist(), np.round(cmpe, 4).tolist())), "best", best)
    print("static ", dict(zip(sp.tolist(), np.round(cmpe_static, 4).tolist())), "best", best_static)
    assert speeds[0] < best < speeds[-1]
    # one sweep point against the oracle on the moved pixels
    import dataclasses
    c0 = float(speeds[4])
    x, z = dynamic_pixels(p, c0)
    q = dataclasses.replace(p, pix_x=x, pix_z=z)
    parts, _, _, _ = oracle.Oracle(q).loss_grad(psi, np.full((p.nz, p.nx), 1.0 / c0), grad=False)
    assert cmpe[4] == pytest.approx(parts[1], rel=2e-3)   # masks decided independently
