"""Image-quality metrics (Sec. III-F) on the GPU against the float64 oracle.

A 32-element acquisition of a two-layer medium with a 4 mm anechoic cyst is
imaged on a dense 48 x 48 polar grid around the cyst.  The GPU's metrics of its
own images must equal the oracle formulas applied to the same images (stage-wise)
and, within the image tolerance, to the oracle's own images; the cyst must show
as a dark target against the speckle (negative contrast, high generalized CNR).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2608_06853_b300 as af
import synth
from oracle import metrics as M

pytestmark = pytest.mark.gpu

CYST_DEPTH, CYST_R = 25e-3, 4e-3


def _case():
    p = synth.config_tiny()
    cx = p.arc_cx
    cz = p.arc_cz + p.lens_radius + CYST_DEPTH
    p.medium.cysts = [(cx, cz, CYST_R)]
    psi = synth.simulate(p, 6000, seed=23)
    q = synth.image_grid_problem(p, 48, 48, (CYST_DEPTH - 10e-3, CYST_DEPTH + 10e-3))
    d = np.hypot(q.pix_x - cx, q.pix_z - cz)
    roi = np.zeros(q.npix, np.uint8)
    roi[d < 0.7 * CYST_R] = 1
    roi[(d > 1.3 * CYST_R) & (d < 2.2 * CYST_R)] = 2
    return p, q, psi, roi


def _forward(q, psi, s):
    dev = torch.device("cuda")
    plan = af.Plan(q)
    iq = torch.from_numpy(psi).to(dev)
    sd = torch.from_numpy(s).to(dev)
    loss = torch.zeros(4, device=dev)
    plan.af_forward(iq, sd, loss)
    torch.cuda.synchronize()
    return plan, sd


def test_image_metrics_match_oracle_and_show_the_cyst():
    p, q, psi, roi = _case()
    assert (roi == 1).sum() > 20 and (roi == 2).sum() > 100
    s = q.initial_slowness(1540.0)
    plan, _ = _forward(q, psi, s)
    m = plan.image_metrics(torch.from_numpy(roi).cuda(), nbins=64)
    B = plan.images().cpu().numpy().astype(np.complex128)
    ref = M.image_metrics(B, q.nsub, q.n_patch, q.patch_npix, roi, nbins=64)
    assert m["n_in"] == (roi == 1).sum() and m["n_out"] == (roi == 2).sum()
    for k in ("cf_mean", "loc", "cmcc", "mean_in", "mean_out", "cnr"):
        assert m[k] == pytest.approx(ref[k], rel=1e-4, abs=1e-6), k
    assert m["contrast_db"] == pytest.approx(ref["contrast_db"], abs=1e-3)
    # a pixel whose envelope lands in the neighbouring bin moves gCNR by 1 / n
    assert abs(m["gcnr"] - ref["gcnr"]) <= 2.0 / min(m["n_in"], m["n_out"])
    # end to end: against the oracle's own images
    o = oracle.Oracle(q)
    _, a_gpu = plan.delays()
    apod = a_gpu.cpu().numpy()
    T, _, _ = o.delays(s.astype(np.float64), apod_in=apod)
    Bo = o.das(psi, T, apod)
    ref2 = M.image_metrics(Bo, q.nsub, q.n_patch, q.patch_npix, roi, nbins=64)
    for k in ("cf_mean", "loc", "cmcc", "cnr"):
        assert m[k] == pytest.approx(ref2[k], rel=1e-3), k
    assert m["contrast_db"] == pytest.approx(ref2["contrast_db"], abs=1e-2)
    # the anechoic cyst against speckle
    assert m["contrast_db"] < -6.0 and m["gcnr"] > 0.5
    assert 0.0 < m["cf_mean"] < 1.0 and -1.0 <= m["loc"] <= 1.0 and 0.0 < m["cmcc"] <= 1.0


def test_speed_mae_matches_oracle():
    p, q, psi, roi = _case()
    rng = np.random.default_rng(2)
    s = (1.0 / (1540.0 + 20.0 * rng.standard_normal((q.nz, q.nx)))).astype(np.float32)
    plan, sd = _forward(q, psi, s)
    c_true = q.medium.speed_at(q.pix_x, q.pix_z).astype(np.float32)
    mae = plan.speed_mae(sd, torch.from_numpy(c_true).cuda())
    o = oracle.Oracle(q)
    c_est = np.array([1.0 / o.bicubic(s.astype(np.float64), x, z) for x, z in zip(q.pix_x, q.pix_z)])
    assert mae == pytest.approx(M.speed_mae(c_est, c_true), rel=1e-5)
    # a uniform map at the top layer's speed: the MAE is the bottom layer's share of the
    # speed difference
    u = q.initial_slowness(1450.0)
    plan2, su = _forward(q, psi, u)
    frac = float(np.mean(np.isclose(c_true, 1570.0)))
    assert plan2.speed_mae(su, torch.from_numpy(c_true).cuda()) == pytest.approx(120.0 * frac, rel=1e-5)


def test_metrics_argument_errors():
    p, q, psi, roi = _case()
    plan = af.Plan(q)
    r = torch.from_numpy(roi).cuda()
    with pytest.raises(af.AfError, match="AF_ERR_STATE"):
        plan.image_metrics(r)
    s = q.initial_slowness(1540.0)
    plan2, _ = _forward(q, psi, s)
    with pytest.raises(af.AfError, match="AF_ERR_ARG"):
        plan2.image_metrics(r, nbins=1)
    assert math.isnan(plan2.image_metrics(torch.zeros_like(r))["contrast_db"])
