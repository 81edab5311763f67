"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Same seeded inputs on both sides.  Where floating point takes a discrete
decision (apodization bit, CMPE correlation mask), the GPU's decision is
injected into the oracle and every disagreement is checked to lie within
rounding distance of the threshold.  Tolerances (stated per test):
delays <= 0.1 ns absolute, images relative L2 <= 1e-4, loss relative <= 1e-4,
gradient relative L2 <= 1e-3.
"""
import dataclasses
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
import paper_2608_06853_b300 as af  # noqa: E402
import synth  # noqa: E402

DELAY_TOL = 1e-10       # s
IMG_TOL = 1e-4          # relative L2
LOSS_TOL = 1e-4         # relative
GRAD_TOL = 1e-3         # relative L2


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def smooth_speed(p, seed, amp=25.0):
    """A smooth random speed map around 1540 m/s (float32 slowness)."""
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((p.nz, p.nx))
    # separable [1 2 1]^3 smoothing
    for _ in range(3):
        f = 0.25 * (np.roll(f, 1, 0) + 2 * f + np.roll(f, -1, 0))
        f = 0.25 * (np.roll(f, 1, 1) + 2 * f + np.roll(f, -1, 1))
    f /= np.abs(f).max()
    return (1.0 / (1540.0 + amp * f)).astype(np.float32)


def layered_speed(p):
    return (1.0 / p.true_speed_grid()).astype(np.float32)


class Run:
    """One forward + adjoint on the GPU with everything copied back to the host."""

    def __init__(self, p, psi, s, iq_dtype=af.AF_IQ_C64):
        dev = torch.device("cuda")
        self.plan = af.Plan(p, iq_dtype=iq_dtype)
        if iq_dtype == af.AF_IQ_C64:
            self.iq = torch.from_numpy(psi).to(dev)
            self.scale = None
        else:
            x = torch.from_numpy(psi).to(dev)
            sc = torch.view_as_real(x).abs().amax(dim=(1, 2, 3)).clamp_min(1e-30)
            q = torch.view_as_real(x) / sc[:, None, None, None]
            q = q.to(torch.bfloat16 if iq_dtype == af.AF_IQ_BF16 else torch.float16).contiguous()
            self.iq, self.scale = q, sc.float().contiguous()
        self.s = torch.from_numpy(s).to(dev)
        self.loss = torch.zeros(4, device=dev)
        self.grad = torch.zeros_like(self.s)
        self.plan.af_forward(self.iq, self.s, self.loss, self.scale)
        self.plan.af_adjoint(self.grad)
        torch.cuda.synchronize()
        T, a = self.plan.delays()
        self.T, self.apod = T.cpu().numpy(), a.cpu().numpy()
        self.phi = self.plan.exit_angles().cpu().numpy().astype(np.float64)
        self.B = self.plan.images().cpu().numpy().astype(np.complex128)
        z, m, n = self.plan.cmpe()
        self.z, self.mask, self.n_active = z.cpu().numpy(), m.cpu().numpy(), n
        self.G = self.plan.image_grad().cpu().numpy().astype(np.complex128)
        self.gdel = self.plan.delay_grad().cpu().numpy().astype(np.float64)
        self.L = self.loss.cpu().numpy().astype(np.float64)
        self.dLds = self.grad.cpu().numpy().astype(np.float64)
        self.counters = self.plan.counters()


def check_apod_disagreements(o, p, run):
    """Apodization bits may differ only where |x'| is within rounding of the cone edge."""
    _, apod_or, _ = o.delays(np.full((p.nz, p.nx), 1 / 1540.0))
    diff = np.argwhere(apod_or != run.apod)
    th = o.element_angles()
    for e, k in diff[:200]:
        c, s_ = math.cos(th[e]), math.sin(th[e])
        dx, dz = p.pix_x[k] - p.elem_x[e], p.pix_z[k] - p.elem_z[e]
        xp, zp = c * dx - s_ * dz, s_ * dx + c * dz
        lim = zp / (2 * p.fnum) if p.apod_mode == 0 else 0.5 * p.fnum * zp
        assert abs(abs(xp) - lim) < 1e-6 * max(abs(zp), 1e-3), (e, k)
    return len(diff)


def check_mask_disagreements(rho_or, mask_gpu, thresh):
    diff = rho_or.ravel()[(rho_or >= thresh).ravel() != (mask_gpu.ravel() == 1)]
    assert np.all(np.abs(diff - thresh) < 1e-4), diff
    return diff.size


# ------------------------------------------------------------------ fixtures
@pytest.fixture(scope="module")
def tiny_case():
    p = synth.config_tiny()
    psi = synth.simulate(p, 2000, seed=20261202)
    return p, psi


def ray_only(p):
    """The same problem with the regularisers off (w1 = w2 = 0): dL/ds is then the ray
    adjoint alone.  With Table II's weights the regulariser gradient is thousands of
    times larger than the ray part and would hide an error in it."""
    return dataclasses.replace(p, w1=0.0, w2=0.0)


def full_parity(p, psi, s, iq_dtype=af.AF_IQ_C64):
    run = Run(p, psi, s, iq_dtype)
    o = oracle.Oracle(p)
    sd = s.astype(np.float64)
    T, apod, phi = o.delays(sd, apod_in=run.apod)
    parts, g, mask, M = o.loss_grad(psi, sd, apod_in=run.apod, mask_in=run.mask)
    B = o.das(psi, T, run.apod)
    _, z, rho, _, _ = o.cmpe(B)
    return run, o, dict(T=T, phi=phi, parts=parts, grad=g, B=B, z=z, rho=rho, M=M)


# ------------------------------------------------------------------ tests
@pytest.mark.parametrize("speed", ["uniform", "smooth", "layered"])
def test_tiny_forward_adjoint_parity(tiny_case, speed):
    p, psi = tiny_case
    s = {"uniform": p.initial_slowness(), "smooth": smooth_speed(p, 1),
         "layered": layered_speed(p)}[speed]
    run, o, ref = full_parity(p, psi, s)
    on = run.apod == 1
    assert on.sum() > 0
    # one-way delays (0.1 ns) and exit angles
    err_T = np.abs(run.T - ref["T"])[on]
    assert err_T.max() <= DELAY_TOL, err_T.max()
    assert np.abs(run.phi - ref["phi"])[on].max() < 2e-5
    # images
    assert rel_l2(run.B, ref["B"]) <= IMG_TOL
    # CMPE decisions and loss
    check_mask_disagreements(ref["rho"], run.mask, p.rho_thresh)
    assert run.n_active == ref["M"]
    for k in range(4):
        assert abs(run.L[k] - ref["parts"][k]) <= LOSS_TOL * max(abs(ref["parts"][k]), 1e-12), k
    # gradient
    assert rel_l2(run.dLds, ref["grad"]) <= GRAD_TOL
    check_apod_disagreements(o, p, run)


def test_tiny_stagewise_adjoint(tiny_case):
    """Each adjoint stage on the GPU's own inputs: CMPE -> dL/dB, DAS -> dL/dT, rays -> dL/ds."""
    p, psi = tiny_case
    s = smooth_speed(p, 2)
    run = Run(p, psi, s)
    o = oracle.Oracle(p)
    G = o.cmpe_adjoint(run.B, run.z.astype(np.complex128), run.mask, run.n_active)
    assert rel_l2(run.G, G) <= 1e-4
    gT = o.das_adjoint(psi, run.T, run.apod, run.G)
    assert rel_l2(run.gdel, gT) <= 1e-4
    ray = o.ray_adjoint(s.astype(np.float64), run.phi, run.apod, run.gdel)
    reg = o.regularizer_grad(s.astype(np.float64))
    assert rel_l2(run.dLds, ray + reg) <= 1e-4
    # the ray adjoint alone (regularisers off), on that run's own dL/dT
    r0 = Run(ray_only(p), psi, s)
    ray0 = o.ray_adjoint(s.astype(np.float64), r0.phi, r0.apod, r0.gdel)
    assert np.linalg.norm(ray0) > 0
    assert rel_l2(r0.dLds, ray0) <= 1e-4


def test_adam_step_parity(tiny_case):
    p, psi = tiny_case
    s = smooth_speed(p, 3)
    run = Run(p, psi, s)
    dev = torch.device("cuda")
    rng = np.random.default_rng(5)
    m0 = (1e-3 * rng.standard_normal(s.shape)).astype(np.float32)
    v0 = (1e-6 * rng.random(s.shape)).astype(np.float32)
    sg, mg, vg = (torch.from_numpy(x.copy()).to(dev) for x in (s, m0, v0))
    run.plan.af_step(run.grad, sg, mg, vg, 3)
    o = oracle.Oracle(p)
    s1, m1, v1 = o.adam(s, run.dLds, m0, v0, 3, p.lr, p.beta1, p.beta2, p.eps, p.c_unit)
    np.testing.assert_allclose(sg.cpu().numpy(), s1, rtol=1e-6)
    np.testing.assert_allclose(mg.cpu().numpy(), m1, rtol=1e-5, atol=1e-12)
    np.testing.assert_allclose(vg.cpu().numpy(), v1, rtol=1e-5, atol=1e-18)


def test_plain_gradient_step_parity(tiny_case):
    """Eq. 9 as printed (AF_OPT_GD): one gradient step of c in km/s, against the oracle."""
    p, psi = tiny_case
    q = dataclasses.replace(p, optimizer=af.AF_OPT_GD, lr=0.02)
    s = smooth_speed(q, 3)
    run = Run(q, psi, s)
    sg = torch.from_numpy(s.copy()).cuda()
    run.plan.af_step(run.grad, sg, None, None, 1)
    s1 = oracle.Oracle(q).gd(s, run.dLds, q.lr, q.c_unit)
    np.testing.assert_allclose(sg.cpu().numpy(), s1, rtol=1e-6)
    assert np.abs(s1 - s).max() > 0


def test_ragged_and_variant_shapes():
    """Pixel count not a multiple of 32, no lens, sub_width 1, 2, 8 and 16, printed Eq. 4; one
    CTA's pixels spread over the whole depth range; an odd trace length; samples
    outside the trace for some pixels; the Eq. 6 conventional lens model and non-zero
    t_ttp / t0."""
    cases = [
        dict(n_ang=3, n_rad=3, patch_w=3),                      # 81 pixels
        dict(n_ang=1, n_rad=8, patch_w=5),                      # 200 pixels over 8-50 mm depth
        dict(n_ang=3, n_rad=3, patch_w=3, ns=1023),             # 1023 samples per trace
        # a third of the pixels need samples past the end of a 600-sample trace, or
        # (first sample at 20 us) before its start: their warps gather with range
        # checks, the others without
        dict(n_ang=3, n_rad=3, patch_w=3, ns=600),
        dict(n_ang=3, n_rad=3, patch_w=3, t0=2.0e-5),
        # Eq. 6 conventional model: straight rays from the elements plus one scalar
        # offset (lens correction + envelope peak) on every round trip; and the
        # bent-ray model with an envelope offset and a late first sample
        dict(n_ang=3, n_rad=3, patch_w=3, lens_mode=1, t_ttp=1.1e-6),
        dict(n_ang=3, n_rad=3, patch_w=3, t_ttp=3.5e-7, t0=2.0e-6),
        dict(n_ang=5, n_rad=2, patch_w=5, lens_mode=1),         # straight rays, 250 pixels
        dict(n_ang=2, n_rad=3, patch_w=3, sub_width=2),         # 16 subapertures
        dict(n_ang=2, n_rad=2, patch_w=4, sub_width=8),         # 4 subapertures
        dict(n_ang=2, n_rad=2, patch_w=3, sub_width=1),         # 32 one-element subapertures, 1024 images
        dict(n_ang=2, n_rad=2, patch_w=3, sub_width=16),        # 2 subapertures: images only, no CMPE pair
        dict(n_ang=3, n_rad=2, patch_w=3, apod_mode=1, hyper=dict(synth.TABLE2["phantom_c5"], fnum=3.0)),
    ]
    for kw in cases:
        p = synth.config_tiny(**kw)
        psi = synth.simulate(p, 500, seed=7)
        run, o, ref = full_parity(p, psi, smooth_speed(p, 4))
        on = run.apod == 1
        if on.any():
            assert np.abs(run.T - ref["T"])[on].max() <= DELAY_TOL, kw
        assert rel_l2(run.B, ref["B"]) <= IMG_TOL, kw
        assert abs(run.L[0] - ref["parts"][0]) <= LOSS_TOL * max(abs(ref["parts"][0]), 1e-12), kw
        assert rel_l2(run.dLds, ref["grad"]) <= GRAD_TOL, kw


@pytest.mark.parametrize("lens_mode", [af.AF_LENS_PLANAR, af.AF_LENS_NONE])
def test_linear_array_parity(lens_mode):
    """Linear array (L12-3v lens of Table I): the bent-ray model with a flat lens, and
    the Eq. 6 conventional model (straight rays + the scalar t_ttp), every stage
    against the oracle."""
    p = synth.config_linear_tiny(lens_mode=lens_mode)
    psi = synth.simulate(p, 800, seed=17)
    run, o, ref = full_parity(p, psi, smooth_speed(p, 6))
    on = run.apod == 1
    assert on.any()
    assert np.abs(run.T - ref["T"])[on].max() <= DELAY_TOL
    if lens_mode == af.AF_LENS_PLANAR:
        np.testing.assert_allclose(run.phi[on], ref["phi"][on], rtol=0, atol=5e-8)   # exit x (m)
    assert rel_l2(run.B, ref["B"]) <= IMG_TOL
    assert abs(run.L[0] - ref["parts"][0]) <= LOSS_TOL * max(abs(ref["parts"][0]), 1e-12)
    assert rel_l2(run.dLds, ref["grad"]) <= GRAD_TOL
    assert run.plan.counters()["fp64_solves"] == 0


def test_large_grid_fallback_layouts():
    """A 176 x 176 grid: the paired slowness grid of the delay kernel and the two
    bank-skewed copies of the ray adjoint no longer fit in shared memory, so the
    scalar-tap delay kernel and the single-copy ray adjoint run; both against the
    oracle.  The ray adjoint is checked with the regularisers off: on this fine grid
    a few second differences of Eq. 11 sit within float rounding of the deadzone
    threshold, so the float kernel and the float64 oracle take different sign
    decisions there (a decision, not an arithmetic error), and the regulariser
    gradient is ~1e4 times the ray part."""
    p = ray_only(synth.config_tiny(n_ang=4, n_rad=4, patch_w=5, nx=176, nz=176))
    psi = synth.simulate(p, 600, seed=19)
    s = smooth_speed(p, 8)
    run = Run(p, psi, s)
    o = oracle.Oracle(p)
    T, _, _ = o.delays(s.astype(np.float64), apod_in=run.apod)
    on = run.apod == 1
    assert np.abs(run.T - T)[on].max() <= DELAY_TOL
    assert rel_l2(run.B, o.das(psi, T, run.apod)) <= IMG_TOL
    ray = o.ray_adjoint(s.astype(np.float64), run.phi, run.apod, run.gdel)
    assert np.linalg.norm(ray) > 0
    assert rel_l2(run.dLds, ray) <= 1e-4


@pytest.mark.parametrize("nx,nz", [(128, 128), (128, 136)])
def test_ray_adjoint_launch_shapes(nx, nz):
    """The ray adjoint's two-copy layouts against the oracle. On a 128 x 128 grid
    the two copies (165 KB) leave room for the 24-warp CTA's item tables. On a
    128 x 136 grid (179 KB) they do not, and the 16-warp CTA runs. The 128-wide
    grids also take the delay kernel's compile-time pitch. The regularisers are off,
    so that dL/ds is the ray part alone."""
    p = ray_only(synth.config_tiny(n_ang=4, n_rad=4, patch_w=5, nx=nx, nz=nz))
    psi = synth.simulate(p, 600, seed=23)
    s = smooth_speed(p, 8)
    run = Run(p, psi, s)
    o = oracle.Oracle(p)
    T, _, _ = o.delays(s.astype(np.float64), apod_in=run.apod)
    on = run.apod == 1
    assert np.abs(run.T - T)[on].max() <= DELAY_TOL
    ray = o.ray_adjoint(s.astype(np.float64), run.phi, run.apod, run.gdel)
    assert np.linalg.norm(ray) > 0
    assert rel_l2(run.dLds, ray) <= 1e-4


def test_degenerate_cases():
    """No patches: loss and gradient are the regulariser's; < 3 subapertures: no CMPE terms."""
    base = synth.config_tiny(n_ang=2, n_rad=2, patch_w=3)
    psi = synth.simulate(base, 200, seed=8)
    s = smooth_speed(base, 5, amp=60.0)
    empty = dataclasses.replace(base, n_patch=0, pix_x=np.zeros(0), pix_z=np.zeros(0))
    run = Run(empty, psi, s)
    o = oracle.Oracle(empty)
    rtv, rsv = o.regularizers(s.astype(np.float64))
    assert run.L[1] == 0.0
    assert run.L[0] == pytest.approx(empty.w1 * rtv + empty.w2 * rsv, rel=1e-4)
    assert rel_l2(run.dLds, o.regularizer_grad(s.astype(np.float64))) <= 1e-4
    few = dataclasses.replace(base, sub_width=16)
    run2 = Run(few, psi, s)
    assert run2.L[1] == 0.0 and run2.counters["npair"] == 0


@pytest.mark.parametrize("dtype", [af.AF_IQ_BF16, af.AF_IQ_F16])
def test_half_precision_storage_error_is_small(tiny_case, dtype):
    """16-bit channel data with a per-transmit scale: error vs the FP64 oracle is reported
    and bounded by the storage rounding (bf16: 2^-8, f16: 2^-11 relative)."""
    p, psi = tiny_case
    s = smooth_speed(p, 6)
    run, o, ref = full_parity(p, psi, s, iq_dtype=dtype)
    e_img = rel_l2(run.B, ref["B"])
    e_loss = abs(run.L[0] - ref["parts"][0]) / abs(ref["parts"][0])
    bound = 2 ** -8 if dtype == af.AF_IQ_BF16 else 2 ** -11
    print(f"dtype {dtype}: image rel L2 {e_img:.2e}, loss rel {e_loss:.2e}")
    assert e_img < bound
    assert e_loss < 20 * bound


def test_autograd_function_matches_adjoint(tiny_case):
    p, psi = tiny_case
    dev = torch.device("cuda")
    plan = af.Plan(p)
    iq = torch.from_numpy(psi).to(dev)
    s = torch.from_numpy(smooth_speed(p, 7)).to(dev).requires_grad_(True)
    L = af.AutofocusLoss.apply(s, plan, iq, None)
    (2.0 * L).backward()
    loss = torch.zeros(4, device=dev)
    g = torch.zeros_like(s)
    plan.af_forward(iq, s.detach(), loss, None)
    plan.af_adjoint(g)
    # float atomics make the two adjoint runs differ in the last bits only
    torch.testing.assert_close(s.grad, 2.0 * g, rtol=1e-4, atol=1e-6 * float(g.abs().max()))
    assert float(L.detach()) == pytest.approx(float(loss[0]))


def test_error_statuses():
    p = synth.config_tiny(n_ang=2, n_rad=2, patch_w=3)
    dev = torch.device("cuda")
    plan = af.Plan(p)
    g = torch.zeros((p.nz, p.nx), device=dev)
    with pytest.raises(af.AfError) as ei:
        plan.af_adjoint(g)
    assert ei.value.status == af.AF_ERR_STATE
    iq = torch.zeros((p.ne, p.ne, p.ns), dtype=torch.complex64, device=dev)
    s = torch.full((p.nz, p.nx), 1 / 1540.0, device=dev)
    s[3, 4] = float("nan")
    loss = torch.zeros(4, device=dev)
    plan.af_forward(iq, s, loss)
    assert plan.af_sync_status() == af.AF_ERR_NUMERIC
    assert plan.af_sync_status() == af.AF_OK          # flag cleared once reported
    plan16 = af.Plan(p, iq_dtype=af.AF_IQ_BF16)
    with pytest.raises(af.AfError) as ei:
        plan16.af_forward(iq, s, loss, None)
    assert ei.value.status == af.AF_ERR_DTYPE


def autofocus_mae(p, psi, lens_mode, iters=100):
    """MAE of Eq. 13 over the image points before and after `iters` Adam iterations from
    a uniform 1540 m/s map, with the given lens model; also the CMPE history."""
    q = dataclasses.replace(p, lens_mode=lens_mode)
    dev = torch.device("cuda")
    plan = af.Plan(q)
    iq = torch.from_numpy(psi).to(dev)
    s = torch.from_numpy(q.initial_slowness()).to(dev)
    m, v, g = torch.zeros_like(s), torch.zeros_like(s), torch.zeros_like(s)
    loss = torch.zeros(4, device=dev)
    c_true = torch.from_numpy(q.medium.speed_at(q.pix_x, q.pix_z).astype(np.float32)).to(dev)
    mae0 = plan.speed_mae(s, c_true)
    cmpe = []
    for it in range(1, iters + 1):
        plan.af_iterate(iq, s, g, m, v, it, loss)
        cmpe.append(float(loss[1]))
    assert plan.af_sync_status() == af.AF_OK
    c = 1.0 / s.cpu().numpy()
    assert np.isfinite(c).all() and c.min() > 1300 and c.max() < 1800
    return mae0, plan.speed_mae(s, c_true), cmpe


def test_autofocus_lowers_mae_and_lens_model_beats_no_lens():
    """100 Adam iterations (Eq. 9) with Table II's phantom C5-2v column on the two-layer
    medium, starting from a uniform 1540 m/s map: the sound-speed MAE of Eq. 13 over the
    image points falls, and with the bent-ray lens model (Eq. 7-8) it ends below the MAE of
    the model without the lens (Sec. IV: lens correction lowers the MAE).  Under the
    reading of Eq. 9-11 in km/s the oracle gives 42.4 -> 41.5 m/s (no lens: 42.2 m/s)."""
    column = "phantom_c5"
    p = synth.config_tiny(hyper=synth.TABLE2[column])
    psi = synth.simulate(p, 2000, seed=20261202)
    mae0, mae, cmpe = autofocus_mae(p, psi, af.AF_LENS_BENT_RAY)
    mae0_n, mae_n, _ = autofocus_mae(p, psi, af.AF_LENS_NONE)
    print(f"{column}: CMPE {cmpe[0]:.4f} -> {cmpe[-1]:.4f}; MAE {mae0:.2f} -> {mae:.2f} m/s "
          f"(no lens: {mae_n:.2f} m/s)")
    assert mae0 == pytest.approx(mae0_n)
    assert mae < mae0
    assert mae < mae_n
    assert min(cmpe[-10:]) < cmpe[0]


def test_full_size_eq9_with_the_in_vivo_column_lowers_mae_and_beats_no_lens(full_case):
    """The 128-element workload with Table II's in vivo C5-2v column as printed
    (LR 0.05) and Eq. 9 as printed (the plain gradient step on c in km/s): 100
    iterations from a uniform 1540 m/s map keep the map within 1300-1800 m/s, lower the
    MAE of Eq. 13 over the image points, and end below the MAE of the model without the
    lens.  (With Adam, whose steps do not shrink with the gradient, the same learning
    rate moves every node by 50 m/s per step and the map leaves the speed range.)"""
    p, psi = full_case
    q = dataclasses.replace(p, lr=synth.TABLE2["invivo_c5"]["lr"], optimizer=af.AF_OPT_GD)
    mae0, mae, cmpe = autofocus_mae(q, psi, af.AF_LENS_BENT_RAY)
    _, mae_n, _ = autofocus_mae(q, psi, af.AF_LENS_NONE)
    print(f"full size, Eq. 9 as printed, in vivo LR: CMPE {cmpe[0]:.4f} -> {cmpe[-1]:.4f}; "
          f"MAE {mae0:.2f} -> {mae:.2f} m/s (no lens: {mae_n:.2f} m/s)")
    assert mae < mae0
    assert mae < mae_n


# ------------------------------------------------------------------ full size
@pytest.fixture(scope="module")
def full_case():
    """The benchmark's workload: 10 scatterers per resolution cell (about 7e5), echoes
    simulated by the input generator's GPU kernels."""
    p = synth.config_full()
    psi = synth.simulate_gpu(p, synth.speckle_count(p), seed=20261203).cpu().numpy()
    torch.cuda.empty_cache()
    return p, psi


@pytest.mark.parametrize("dtype", [af.AF_IQ_C64, af.AF_IQ_BF16, af.AF_IQ_F16])
def test_full_size_end_to_end_parity(full_case, dtype):
    """The whole forward and adjoint at full size (128 x 128 x 3072 channel data, 400
    patches of 9 x 9, 128^2 grid, a layered map) against the oracle run end to end on the
    same inputs (OpenMP build of the oracle source), with the GPU's apodization bits and
    CMPE mask injected.  Float32 channel data: loss of Eq. 12 within 1e-4, dL/ds within
    1e-3 (relative L2).  Bf16 and f16 storage with a per-transmit scale: the errors of
    images, loss and gradient against the same float64 reference are printed and bounded
    by the storage rounding (2^-8, 2^-11)."""
    p, psi = full_case
    s = layered_speed(p)
    run = Run(p, psi, s, iq_dtype=dtype)
    o = oracle.Oracle(p, parallel=True)
    sd = s.astype(np.float64)
    parts, g, _, M = o.loss_grad(psi, sd, apod_in=run.apod, mask_in=run.mask)
    assert M == run.n_active > 0
    T, _, _ = o.delays(sd, apod_in=run.apod)
    e_img = rel_l2(run.B, o.das(psi, T, run.apod))
    e_loss = abs(run.L[0] - parts[0]) / abs(parts[0])
    e_grad = rel_l2(run.dLds, g)
    name = {af.AF_IQ_C64: "float32", af.AF_IQ_BF16: "bf16", af.AF_IQ_F16: "f16"}[dtype]
    print(f"full size, {name} channel data vs float64 oracle: images {e_img:.2e}, loss {e_loss:.2e}, "
          f"dL/ds {e_grad:.2e} (rel L2); active CMPE terms {M}")
    if dtype == af.AF_IQ_C64:
        assert e_img <= IMG_TOL
        assert e_loss <= LOSS_TOL
        assert e_grad <= GRAD_TOL
    else:
        unit = 2 ** -8 if dtype == af.AF_IQ_BF16 else 2 ** -11
        assert e_img < unit
        assert e_loss < 20 * unit
        assert e_grad < 0.1


def test_full_size_sampled_parity(full_case):
    """128 x 128 x 3072 acquisition, 400 patches of 9 x 9, 128^2 grid, in the launch
    configuration of the benchmark.  The oracle checks sampled outputs: delays of random
    (element, pixel) pairs, images, CMPE terms and dL/dT of sampled patches, and every
    adjoint stage on the GPU's own intermediate values."""
    p, psi = full_case
    s = layered_speed(p)
    run = Run(p, psi, s)
    o_full = oracle.Oracle(p, parallel=True)
    sd = s.astype(np.float64)
    sbar = 1.0 / o_full.mean_speed(sd)
    rng = np.random.default_rng(11)
    # delays of 3000 random apodized pairs
    ee, kk = np.nonzero(run.apod)
    pick = rng.choice(len(ee), 3000, replace=False)
    errs = []
    for q in pick:
        e, k = int(ee[q]), int(kk[q])
        phi, tl, qx, qz, _ = o_full.exit_point(e, p.pix_x[k], p.pix_z[k], sbar)
        T = tl + o_full.ray_time(sd, qx, qz, p.pix_x[k], p.pix_z[k])
        errs.append(abs(T - run.T[e, k]))
    assert max(errs) <= DELAY_TOL, max(errs)
    # sampled patches as a sub-problem: per-pixel images and per-patch CMPE terms
    patches = np.sort(rng.choice(p.n_patch, 6, replace=False))
    pix = np.concatenate([np.arange(P * p.patch_npix, (P + 1) * p.patch_npix) for P in patches])
    sub = dataclasses.replace(p, n_patch=len(patches), pix_x=p.pix_x[pix], pix_z=p.pix_z[pix])
    o = oracle.Oracle(sub)
    T, _, _ = o.delays(sd, apod_in=run.apod[:, pix])
    B = o.das(psi, T, run.apod[:, pix])
    assert rel_l2(run.B[:, pix], B) <= IMG_TOL
    _, z, rho, _, _ = o.cmpe(B)
    np.testing.assert_allclose(run.z[patches], z, rtol=1e-4, atol=1e-4 * np.abs(z).max())
    check_mask_disagreements(rho, run.mask[patches], p.rho_thresh)
    # adjoint stages on the GPU's own inputs
    G = o_full.cmpe_adjoint(run.B, run.z.astype(np.complex128), run.mask, run.n_active)
    assert rel_l2(run.G, G) <= 1e-4
    gT = o.das_adjoint(psi, run.T[:, pix], run.apod[:, pix], run.G[:, pix])
    assert rel_l2(run.gdel[:, pix], gT) <= 1e-4
    ray = o_full.ray_adjoint(sd, run.phi, run.apod, run.gdel)
    reg = o_full.regularizer_grad(sd)
    assert rel_l2(run.dLds, ray + reg) <= 1e-4
    # the ray adjoint alone in the benchmark's launch shape (regularisers off); its
    # dL/dT equals this run's up to the order of the DAS adjoint's float atomics
    r0 = Run(ray_only(p), psi, s)
    assert rel_l2(r0.gdel, run.gdel) <= 1e-5
    assert rel_l2(r0.dLds, ray) <= 1e-4
    # loss assembled from the oracle's terms with the GPU mask
    L_or = float(np.sum(np.abs(np.angle(run.z.astype(np.complex128)))[run.mask == 1])) / max(run.n_active, 1)
    assert abs(run.L[1] - L_or) <= LOSS_TOL * L_or
    rtv, rsv = o_full.regularizers(sd)
    assert run.L[2] == pytest.approx(rtv, rel=1e-4)
    assert run.L[3] == pytest.approx(rsv, rel=1e-4, abs=1e-9)


def test_bmode_and_integrated_cmpe_images(tiny_case):
    """Full-aperture envelope |sum B| and integrated CMPE against the oracle's images; a
    point scatterer at the true speed is the brightest pixel of its patch with zero
    integrated phase error."""
    p, psi = tiny_case
    run = Run(p, psi, smooth_speed(p, 9))
    b, c = run.plan.bmode()
    b, c = b.cpu().numpy(), c.cpu().numpy()
    o = oracle.Oracle(p)
    T, _, _ = o.delays(smooth_speed(p, 9).astype(np.float64), apod_in=run.apod)
    B = o.das(psi, T, run.apod)
    np.testing.assert_allclose(b, np.abs(B.sum(0)), rtol=2e-4, atol=1e-4 * np.abs(B.sum(0)).max())
    pr = o.pairs()
    ref_c = np.abs(np.angle(B[pr[:, 0]] * np.conj(B[pr[:, 1]]))).sum(0)
    # phases of near-zero cross products are ill-conditioned: compare where they are not
    mag = np.abs(B[pr[:, 0]] * np.conj(B[pr[:, 1]])).min(0)
    ok = mag > 1e-3 * mag.max()
    np.testing.assert_allclose(c[ok], ref_c[ok], rtol=1e-3, atol=1e-3)
    # point scatterer
    q = synth.config_tiny(n_ang=3, n_rad=3, patch_w=3)
    q.medium = synth.Medium(speeds=[1540.0])
    P = 4
    centre = P * q.patch_npix + q.patch_npix // 2
    T1 = synth.oneway_times(q, np.array([q.pix_x[centre]]), np.array([q.pix_z[centre]]))
    psi1 = synth.echoes(q, T1, np.array([1.0]))
    run1 = Run(q, psi1, q.initial_slowness(1540.0))
    b1, c1 = run1.plan.bmode()
    b1, c1 = b1.cpu().numpy(), c1.cpu().numpy()
    patch = slice(P * q.patch_npix, (P + 1) * q.patch_npix)
    assert int(np.argmax(b1[patch])) == q.patch_npix // 2
    assert c1[centre] < 1e-3


def test_seeded_random_configurations():
    """Sixteen seeded random small problems drawn over element count, subaperture width
    (1-8), patch layout and width, trace length (some traces end before the deepest
    pixels), grid size, depth range, lens model (bent ray or Eq. 6), f-number rule,
    t0 and t_ttp: delays, images, loss and dL/ds (regularisers off, so the ray
    adjoint is not hidden) against the oracle at the usual tolerances."""
    rng = np.random.default_rng(20261204)
    ran = 0
    for case in range(16):
        ne = int(rng.choice([16, 24, 32, 40]))
        sub = int(rng.choice([w for w in (1, 2, 4, 8) if ne % w == 0 and ne // w >= 2]))
        d0 = float(rng.uniform(6e-3, 15e-3))
        kw = dict(ne=ne, sub_width=sub, n_ang=int(rng.integers(1, 5)), n_rad=int(rng.integers(1, 5)),
                  patch_w=int(rng.integers(2, 7)), ns=int(rng.integers(600, 1400)),
                  nx=int(rng.integers(8, 41)), nz=int(rng.integers(8, 41)),
                  depth_min=d0, depth_max=d0 + float(rng.uniform(5e-3, 40e-3)),
                  lens_mode=int(rng.choice([0, 0, 1])), apod_mode=int(rng.integers(0, 2)),
                  t0=float(rng.choice([0.0, 2e-6])), t_ttp=float(rng.choice([0.0, 5e-7])))
        p = ray_only(synth.config_tiny(**kw))
        if af.check_config(p) != af.AF_OK:
            continue
        psi = synth.simulate(p, 400, seed=100 + case)
        run, o, ref = full_parity(p, psi, smooth_speed(p, 30 + case))
        on = run.apod == 1
        if on.any():
            assert np.abs(run.T - ref["T"])[on].max() <= DELAY_TOL, kw
        assert rel_l2(run.B, ref["B"]) <= IMG_TOL, kw
        assert abs(run.L[0] - ref["parts"][0]) <= LOSS_TOL * max(abs(ref["parts"][0]), 1e-12), kw
        assert rel_l2(run.dLds, ref["grad"]) <= GRAD_TOL, kw
        ran += 1
    assert ran >= 12


@pytest.mark.parametrize("lens_mode", [af.AF_LENS_PLANAR, af.AF_LENS_NONE])
def test_seeded_random_linear_configurations(lens_mode):
    """Six seeded random linear-array problems per lens model (the flat-lens bent ray
    of Eq. 8, and the Eq. 6 straight ray with t_ttp): element count, subaperture
    width, patch layout, trace length, grid and depth drawn at random; delays,
    images, loss and dL/ds (regularisers off) against the oracle."""
    rng = np.random.default_rng(20261205 + lens_mode)
    ran = 0
    for case in range(6):
        ne = int(rng.choice([16, 24, 32]))
        sub = int(rng.choice([w for w in (1, 2, 4, 8) if ne % w == 0 and ne // w >= 2]))
        d0 = float(rng.uniform(3e-3, 8e-3))
        kw = dict(ne=ne, sub_width=sub, lens_mode=lens_mode, n_lat=int(rng.integers(1, 5)),
                  n_ax=int(rng.integers(1, 5)), patch_w=int(rng.integers(2, 7)), ns=int(rng.integers(500, 1100)),
                  nx=int(rng.integers(8, 33)), nz=int(rng.integers(8, 33)),
                  depth_min=d0, depth_max=d0 + float(rng.uniform(4e-3, 16e-3)))
        p = ray_only(synth.config_linear_tiny(**kw))
        if af.check_config(p) != af.AF_OK:
            continue
        psi = synth.simulate(p, 400, seed=200 + case)
        run, o, ref = full_parity(p, psi, smooth_speed(p, 50 + case))
        on = run.apod == 1
        if on.any():
            assert np.abs(run.T - ref["T"])[on].max() <= DELAY_TOL, kw
        assert rel_l2(run.B, ref["B"]) <= IMG_TOL, kw
        assert abs(run.L[0] - ref["parts"][0]) <= LOSS_TOL * max(abs(ref["parts"][0]), 1e-12), kw
        assert rel_l2(run.dLds, ref["grad"]) <= GRAD_TOL, kw
        ran += 1
    assert ran >= 4
