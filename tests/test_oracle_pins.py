"""Pins of the FP64 oracle to the paper and to mathematics (CPU only).

Each test checks the oracle against something other than itself: a closed
form, an invariant, a brute-force search, finite differences, or a special
case that reduces to a textbook result.  A plausible slip in the oracle (a
dropped term, a wrong sign, a transposed operand, a wrong index) fails at
least one of them.
"""
import dataclasses
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small(**over):
    kw = dict(n_ang=3, n_rad=3, patch_w=3)
    kw.update(over)
    return synth.config_tiny(**kw)


# ---------------------------------------------------------------- geometry
def test_table_values_match_paper():
    """Table I/II values as printed in the paper drive the configs."""
    t2 = json.load(open(os.path.join(GOLDEN, "table2_hyperparameters.json")))
    for col in ("phantom_l12", "phantom_c5", "invivo_c5"):
        for k, v in t2[col].items():
            assert synth.TABLE2[col][k] == pytest.approx(v, rel=0, abs=0), (col, k)
    t1 = json.load(open(os.path.join(GOLDEN, "table1_lens_calibration.json")))
    assert t1["C5-2v (Phantoms)"]["c_lens"] == 999.4
    # the linear-array configuration uses the L12-3v lens of Table I
    pl = synth.config_linear_tiny()
    assert pl.c_lens == pytest.approx(t1["L12-3v"]["c_lens"], rel=1e-7)
    assert pl.d_lens == pytest.approx(t1["L12-3v"]["d_lens_mm"] * 1e-3, rel=1e-7)
    assert pl.t_ttp == pytest.approx(t1["L12-3v"]["t_ttp_ns"] * 1e-9, rel=1e-7)


def test_eq3_orientation_exact_on_uniform_arc(tiny):
    """Eq. 3 central difference on a uniform arc equals the polar angle exactly."""
    o = oracle.Oracle(tiny)
    th = o.element_angles()
    ref = np.arctan2(tiny.elem_x - tiny.arc_cx, tiny.elem_z - tiny.arc_cz)
    # element positions are float32-rounded, so agreement is to ~1e-7 rad
    np.testing.assert_allclose(th, ref, atol=2e-6)
    # exact arc in float64
    R = 0.04
    a = (np.arange(9) - 4) * 0.01
    ex, ez = R * np.sin(a), R * np.cos(a) - R
    th2 = np.empty(9)
    o.lib.or_element_angles(9, oracle._d(ex), oracle._d(ez), oracle._d(th2))
    np.testing.assert_allclose(th2, a, atol=1e-14)


def test_eq4_apodization_cone():
    """Eq. 2+4: a pixel on the element normal is inside, one beyond the f-number cone is out;
    the printed form (F/2) z' gives the narrower cone."""
    p = small()
    o = oracle.Oracle(p)
    e = 5
    th = o.element_angles()[e]
    n = np.array([math.sin(th), math.cos(th)])
    t = np.array([math.cos(th), -math.sin(th)])
    r0 = np.array([p.elem_x[e], p.elem_z[e]])
    zp = 0.02
    half = zp / (2 * p.fnum)
    inside = r0 + zp * n + 0.99 * half * t
    outside = r0 + zp * n + 1.01 * half * t
    assert o.apod(e, *inside) == 1
    assert o.apod(e, *outside) == 0
    assert o.apod(e, *(r0 - zp * n)) == 0           # behind the element
    pp = small(apod_mode=1)
    op = oracle.Oracle(pp)
    narrow = r0 + zp * n + 1.01 * (0.5 * pp.fnum * zp) * t
    assert op.apod(e, *narrow) == 0
    assert op.apod(e, *(r0 + zp * n + 0.99 * (0.5 * pp.fnum * zp) * t)) == 1


# ---------------------------------------------------------------- lens (Eq. 8)
def _brute_exit(p, e, x, z, sbar, n=1_000_001):
    """Dense search over the lens surface with positions computed directly."""
    the = math.atan2(p.elem_x[e] - p.arc_cx, p.elem_z[e] - p.arc_cz)
    thp = math.atan2(x - p.arc_cx, z - p.arc_cz)
    lo, hi = min(the, thp) - 0.05, max(the, thp) + 0.05
    phi = np.linspace(lo, hi, n)
    RL = p.lens_radius
    qx = p.arc_cx + RL * np.sin(phi)
    qz = p.arc_cz + RL * np.cos(phi)
    T = np.hypot(qx - p.elem_x[e], qz - p.elem_z[e]) / p.c_lens + np.hypot(x - qx, z - qz) * sbar
    k = int(np.argmin(T))
    # refine on a finer grid around the best sample
    phi2 = np.linspace(phi[max(k - 1, 0)], phi[min(k + 1, n - 1)], 200_001)
    qx = p.arc_cx + RL * np.sin(phi2)
    qz = p.arc_cz + RL * np.cos(phi2)
    T2 = np.hypot(qx - p.elem_x[e], qz - p.elem_z[e]) / p.c_lens + np.hypot(x - qx, z - qz) * sbar
    k2 = int(np.argmin(T2))
    return phi2[k2], T2[k2]


def test_exit_point_matches_brute_force_and_snell():
    p = synth.config_full()
    o = oracle.Oracle(p)
    rng = np.random.default_rng(3)
    sbar = 1.0 / 1480.0
    for _ in range(12):
        e = int(rng.integers(p.ne))
        k = int(rng.integers(p.npix))
        x, z = p.pix_x[k], p.pix_z[k]
        phi, tl, qx, qz, it = o.exit_point(e, x, z, sbar)
        assert it > 0
        T = tl + math.hypot(x - qx, z - qz) * sbar
        bphi, bT = _brute_exit(p, e, x, z, sbar)
        assert T <= bT * (1 + 1e-14)
        assert abs(T - bT) <= 1e-12 * bT
        assert abs(phi - bphi) < 1e-6
        # Snell's law at q: sin(theta_lens) / c_lens = sin(theta_tissue) / c_med
        nrm = np.array([qx - p.arc_cx, qz - p.arc_cz]) / p.lens_radius
        a = np.array([qx - p.elem_x[e], qz - p.elem_z[e]])
        b = np.array([x - qx, z - qz])
        sl = (a[0] * nrm[1] - a[1] * nrm[0]) / np.linalg.norm(a)
        st = (b[0] * nrm[1] - b[1] * nrm[0]) / np.linalg.norm(b)
        assert abs(sl / p.c_lens - st * sbar) < 1e-12 * sbar


def test_exit_straight_line_when_lens_matches_medium():
    """c_lens = c_med: the Fermat path is the straight line, T = |r_e - r| / c."""
    c = 1500.0
    p = small(c_lens=c)
    o = oracle.Oracle(p)
    for e in (0, 7, 31):
        for k in (0, 40, 80):
            x, z = p.pix_x[k], p.pix_z[k]
            phi, tl, qx, qz, _ = o.exit_point(e, x, z, 1.0 / c)
            T = tl + math.hypot(x - qx, z - qz) / c
            assert T == pytest.approx(math.hypot(x - p.elem_x[e], z - p.elem_z[e]) / c, rel=1e-14)


# ---------------------------------------------------------------- flat lens (linear array)
def _brute_exit_flat(p, e, x, z, sbar, n=1_000_001):
    """Dense search along the lens line z = lens_z."""
    xe, ze = p.elem_x[e], p.elem_z[e]
    lo, hi = min(xe, x) - 1e-3, max(xe, x) + 1e-3
    u = np.linspace(lo, hi, n)
    T = np.hypot(u - xe, p.lens_z - ze) / p.c_lens + np.hypot(x - u, z - p.lens_z) * sbar
    k = int(np.argmin(T))
    u2 = np.linspace(u[max(k - 1, 0)], u[min(k + 1, n - 1)], 200_001)
    T2 = np.hypot(u2 - xe, p.lens_z - ze) / p.c_lens + np.hypot(x - u2, z - p.lens_z) * sbar
    k2 = int(np.argmin(T2))
    return u2[k2], T2[k2]


def test_flat_lens_exit_matches_brute_force_and_snell():
    """Eq. 8 with a flat lens: the exit point minimises the two-leg time (dense search)
    and satisfies Snell's law about the lens normal (the z axis)."""
    p = synth.config_linear_tiny()
    o = oracle.Oracle(p)
    rng = np.random.default_rng(5)
    sbar = 1.0 / 1530.0
    for _ in range(12):
        e = int(rng.integers(p.ne))
        k = int(rng.integers(p.npix))
        x, z = p.pix_x[k], p.pix_z[k]
        u, tl, qx, qz, it = o.exit_point(e, x, z, sbar)
        assert it > 0 and qz == p.lens_z and qx == u
        T = tl + math.hypot(x - qx, z - qz) * sbar
        bu, bT = _brute_exit_flat(p, e, x, z, sbar)
        assert T <= bT * (1 + 1e-14)
        assert abs(T - bT) <= 1e-12 * bT
        assert abs(u - bu) < 1e-8
        sl = (qx - p.elem_x[e]) / math.hypot(qx - p.elem_x[e], qz - p.elem_z[e])
        st = (x - qx) / math.hypot(x - qx, z - qz)
        assert abs(sl / p.c_lens - st * sbar) < 1e-12 * sbar


def test_flat_lens_closed_forms():
    """A pixel straight below the element exits at the element's foot with
    T_lens = h1 / c_lens; with c_lens = c_med the path is the straight line."""
    p = synth.config_linear_tiny()
    o = oracle.Oracle(p)
    h1 = p.lens_z - p.elem_z[3]
    u, tl, qx, qz, _ = o.exit_point(3, p.elem_x[3], p.lens_z + 7e-3, 1.0 / 1540.0)
    assert u == p.elem_x[3] and tl == pytest.approx(h1 / p.c_lens, rel=1e-15)
    c = 1500.0
    pc = synth.config_linear_tiny(c_lens=c)
    oc = oracle.Oracle(pc)
    for e in (0, 9, 31):
        for k in (0, 150, 399):
            x, z = pc.pix_x[k], pc.pix_z[k]
            _, tl, qx, qz, _ = oc.exit_point(e, x, z, 1.0 / c)
            T = tl + math.hypot(x - qx, z - qz) / c
            assert T == pytest.approx(math.hypot(x - pc.elem_x[e], z - pc.elem_z[e]) / c, rel=1e-14)


@pytest.mark.parametrize("linear", [False, True])
def test_homogeneous_delays_match_independent_simulator(linear):
    """Uniform medium: the oracle's one-way delays (Newton exit point, Eq. 1 ray sum on a
    uniform grid) equal the simulator's (golden-section exit point, exact segment
    time), for the curved and the flat lens."""
    c = 1530.0
    p = synth.config_linear_tiny() if linear else small()
    s = np.full((p.nz, p.nx), 1.0 / c)
    T, _, _ = oracle.Oracle(p).delays(s)
    Ts = synth.oneway_times(p, p.pix_x, p.pix_z, synth.Medium(speeds=[c]))
    np.testing.assert_allclose(T, Ts, rtol=1e-11, atol=0)


def test_zero_thickness_lens_reduces_to_straight_ray():
    p0 = small(d_lens=0.0)
    pn = dataclasses.replace(p0, lens_mode=1)
    s = p0.initial_slowness(1470.0).astype(np.float64)
    T0, _, _ = oracle.Oracle(p0).delays(s)
    Tn, _, _ = oracle.Oracle(pn).delays(s)
    # float32-rounded element positions sit within 1e-8 m of the arc: <= 1e-8 / c_lens
    np.testing.assert_allclose(T0, Tn, rtol=0, atol=1e-8 / p0.c_lens)


def test_homogeneous_delay_is_distance_over_speed():
    """Uniform s: the ray sum is L*s exactly, so T = T_lens + |q - r| / c;
    without a lens T = |r_e - r| / c."""
    pn = small(lens_mode=1)
    c = 1530.0
    s = pn.initial_slowness(c).astype(np.float64)
    s[:] = 1.0 / c
    T, _, _ = oracle.Oracle(pn).delays(s)
    D = np.hypot(pn.pix_x[None, :] - pn.elem_x[:, None], pn.pix_z[None, :] - pn.elem_z[:, None])
    np.testing.assert_allclose(T, D / c, rtol=1e-14)
    p = small()
    o = oracle.Oracle(p)
    T, _, phi = o.delays(s)
    for e in (3, 20):
        for k in (5, 33):
            tl, qx, qz = o.exit_from_angle(e, phi[e, k])
            assert T[e, k] == pytest.approx(tl + math.hypot(p.pix_x[k] - qx, p.pix_z[k] - qz) / c,
                                            rel=1e-14)


# ---------------------------------------------------------------- bicubic + ray sum (Eq. 1)
def test_keys_weights_partition_and_interpolation():
    o = oracle.Oracle(small())
    for t in (0.0, 0.13, 0.5, 0.999):
        w = o.keys_weights(t)
        assert w.sum() == pytest.approx(1.0, abs=1e-15)
        # reproduces linear and quadratic functions sampled at -1, 0, 1, 2
        xs = np.array([-1.0, 0.0, 1.0, 2.0])
        assert (w * xs).sum() == pytest.approx(t, abs=1e-15)
        assert (w * xs ** 2).sum() == pytest.approx(t * t, abs=1e-14)
    np.testing.assert_allclose(o.keys_weights(0.0), [0, 1, 0, 0], atol=0)


def _grid_xy(p):
    gx = p.x0 + p.dx * np.arange(p.nx)
    gz = p.z0 + p.dz * np.arange(p.nz)
    return np.meshgrid(gx, gz)


def test_bicubic_reproduces_quadratic_field_interior():
    p = small()
    o = oracle.Oracle(p)
    X, Z = _grid_xy(p)
    f = lambda x, z: 1e-3 + 0.02 * x - 0.013 * z + 0.7 * x * z + 0.4 * x * x - 0.3 * z * z
    s = f(X, Z)
    rng = np.random.default_rng(0)
    for _ in range(50):
        x = p.x0 + p.dx * rng.uniform(1.0, p.nx - 2.0)
        z = p.z0 + p.dz * rng.uniform(1.0, p.nz - 2.0)
        assert o.bicubic(s, x, z) == pytest.approx(f(x, z), abs=1e-15)


def test_ray_sum_linear_field_closed_form():
    """Mean of N+1 equally spaced samples of a linear field is its midpoint value."""
    p = small()
    o = oracle.Oracle(p)
    X, Z = _grid_xy(p)
    a, bx, bz = 6.4e-4, 1e-3, -2e-3
    s = a + bx * X + bz * Z
    rng = np.random.default_rng(1)
    for _ in range(20):
        qx, x = p.x0 + p.dx * rng.uniform(1, p.nx - 2, 2)
        qz, z = p.z0 + p.dz * rng.uniform(1, p.nz - 2, 2)
        L = math.hypot(x - qx, z - qz)
        ref = L * (a + bx * 0.5 * (qx + x) + bz * 0.5 * (qz + z))
        assert o.ray_time(s, qx, qz, x, z) == pytest.approx(ref, rel=1e-13)


def test_layered_vertical_ray_matches_sum_of_thicknesses():
    """Fine grid of a two-layer medium: vertical ray time ~ sum h_k / c_k (interpolation error only)."""
    p = small(nx=64, nz=400)
    o = oracle.Oracle(p)
    X, Z = _grid_xy(p)
    zi = 0.015
    s = np.where(Z < zi, 1 / 1450.0, 1 / 1570.0)
    z0, z1 = 0.002, 0.045
    x = 0.0
    ref = (zi - z0) / 1450.0 + (z1 - zi) / 1570.0
    p2 = dataclasses.replace(p, nseg=4000)
    t = oracle.Oracle(p2).ray_time(s, x, z0, x, z1)
    # the bicubic smears the step over ~2 cells: error <= jump * 2 dz
    assert abs(t - ref) < abs(1 / 1450.0 - 1 / 1570.0) * 2 * p.dz


# ---------------------------------------------------------------- DAS (Eq. 5) + CMPE
def _point_problem(c=1540.0, **over):
    p = small(**over)
    p.medium = synth.Medium(speeds=[c])
    return p


def _point_data(p, x, z, amp=1.0):
    T = synth.oneway_times(p, np.array([x]), np.array([z]))
    return synth.echoes(p, T, np.array([amp]))


def test_point_scatterer_focuses_with_zero_phase_error():
    """Homogeneous medium at the true speed: every subaperture image is real-positive at the
    scatterer, so a one-pixel patch on it has zero CMPE; the 3x3 patch around it has a
    CMPE far below the one seen at a 3 % speed error."""
    c = 1540.0
    p = _point_problem(c)
    o = oracle.Oracle(p)
    P = 4                                                  # centre patch of the 3x3 grid
    centre = P * p.patch_npix + p.patch_npix // 2
    x, z = p.pix_x[centre], p.pix_z[centre]
    psi = _point_data(p, x, z)
    s = np.full((p.nz, p.nx), 1.0 / c)
    T, apod, _ = o.delays(s)
    B = o.das(psi, T, apod)
    Bc = B[:, centre]
    live = np.abs(Bc) > 1e-3 * np.abs(Bc).max()
    assert live.sum() > 0.5 * len(Bc)
    assert np.all(np.abs(np.angle(Bc[live])) < 1e-7)
    assert np.all(Bc[live].real > 0)
    # focus: the compounded image peaks at the scatterer among the patch pixels
    tot = np.abs(B.sum(0))[P * p.patch_npix:(P + 1) * p.patch_npix]
    assert int(np.argmax(tot)) == p.patch_npix // 2
    # one-pixel patch on the scatterer: exactly zero phase error
    p1 = dataclasses.replace(p, n_patch=1, patch_npix=1, pix_x=np.array([x]), pix_z=np.array([z]))
    o1 = oracle.Oracle(p1)
    T1, a1, _ = o1.delays(s)
    L1, z1, r1, m1, M1 = o1.cmpe(o1.das(psi, T1, a1))
    assert M1 > 0 and L1 < 1e-7
    # 3x3 patch: true speed vs 3 % off
    L, zc, rho, mask, M = o.cmpe(B, mask_in=np.ones((p.n_patch, o.npair), np.uint8))
    err_true = np.abs(np.angle(zc[P])).mean()
    s_bad = np.full((p.nz, p.nx), 1.0 / (1.03 * c))
    Tb, apb, _ = o.delays(s_bad)
    Bb = o.das(psi, Tb, apb)
    Lb, zb, rb, mb, Mb = o.cmpe(Bb, mask_in=np.ones_like(mask))
    err_bad = np.abs(np.angle(zb[P])).mean()
    assert err_bad > 1e-2
    assert err_true < 0.05 * err_bad


def test_reciprocity_and_global_phase_invariance(tiny):
    o = oracle.Oracle(tiny)
    psi = synth.simulate(tiny, 300, seed=5)
    assert np.array_equal(psi, psi.transpose(1, 0, 2))
    s = tiny.initial_slowness().astype(np.float64)
    T, apod, _ = o.delays(s)
    B = o.das(psi, T, apod)
    n = o.nsub
    Bm = B.reshape(n, n, -1)
    np.testing.assert_allclose(Bm, Bm.transpose(1, 0, 2), rtol=1e-12, atol=1e-12 * np.abs(B).max())
    rot = np.exp(1j * 0.7).astype(np.complex64)
    B2 = o.das(psi * rot, T, apod)
    L1, z1, r1, m1, M1 = o.cmpe(B)
    L2, z2, r2, m2, M2 = o.cmpe(B2, mask_in=m1)
    assert L2 == pytest.approx(L1, rel=1e-5)   # psi*rot is rounded to complex64
    np.testing.assert_allclose(r2, r1, atol=1e-5)


def test_das_single_constant_trace_closed_form():
    """Psi_{t,r} = const for one pair only: B = const * exp(j 2 pi fd tau) in that block."""
    p = small(n_ang=1, n_rad=1, patch_w=1)
    o = oracle.Oracle(p)
    psi = np.zeros((p.ne, p.ne, p.ns), np.complex64)
    t, r = 9, 22
    psi[t, r, :] = 0.5 - 0.25j
    s = np.full((p.nz, p.nx), 1 / 1500.0)
    T, apod, _ = o.delays(s)
    B = o.das(psi, T, apod)
    tau = T[t, 0] + T[r, 0] + p.t_ttp
    b = (t // p.sub_width) * o.nsub + r // p.sub_width
    ref = (0.5 - 0.25j) * np.exp(2j * np.pi * p.fd * tau) * apod[t, 0] * apod[r, 0]
    assert abs(B[b, 0] - ref) < 1e-12
    others = np.delete(B[:, 0], b)
    assert np.all(others == 0)


def test_cmpe_closed_form_phase_shift():
    """B2 = B1 exp(j a) on a patch: z = exp(-j a) sum|B1|^2, rho = 1, loss = |a|."""
    p = small(n_ang=1, n_rad=1, patch_w=3)
    o = oracle.Oracle(p)
    rng = np.random.default_rng(2)
    nb, npix = o.nsub ** 2, p.npix
    B = rng.standard_normal((nb, npix)) + 1j * rng.standard_normal((nb, npix))
    pairs = o.pairs()
    a = 0.37
    # make only the first pair fully correlated
    B[pairs[0, 1]] = B[pairs[0, 0]] * np.exp(1j * a)
    L, z, rho, mask, M = o.cmpe(B)
    assert rho[0, 0] == pytest.approx(1.0, abs=1e-14)
    assert np.angle(z[0, 0]) == pytest.approx(-a, abs=1e-14)
    only = np.zeros_like(mask)
    only[0, 0] = 1
    L1, *_ = o.cmpe(B, mask_in=only)
    assert L1 == pytest.approx(a, abs=1e-14)


def test_cmpe_pairs_are_common_midpoint_and_skip_reciprocal():
    p = small()
    o = oracle.Oracle(p)
    n = o.nsub
    pr = o.pairs()
    assert len(pr) == (n - 1) * (n - 2)
    for b1, b2 in pr:
        i1, j1 = divmod(int(b1), n)
        i2, j2 = divmod(int(b2), n)
        assert i1 + j1 == i2 + j2 and i2 == i1 + 1
        assert not (i2 == j1 and j2 == i1)


# ---------------------------------------------------------------- regularisers (Eq. 10-11)
def test_regularizers_closed_form_linear_and_quadratic_speed():
    """Eq. 10-11 on fields with a known derivative, with c in km/s and positions in mm
    (the reading of "physical units" used throughout): a lateral gradient of 20 m/s per
    mm is 0.02 km/s per mm, 0.01 above Table II's kappa; an axial curvature of 10 m/s
    per mm^2 is 0.01 km/s per mm^2, 0.009 above kappa^(2) = 0.001."""
    p = small()
    assert p.c_unit == 1000.0
    o = oracle.Oracle(p)
    X, Z = _grid_xy(p)
    gam = 20.0                                   # m/s per mm along x
    c = 1500.0 + gam * (X - p.x0) * 1e3
    rtv, rsv = o.regularizers(1.0 / c)
    nt = (p.nx - 1) * p.nz + p.nx * (p.nz - 1)
    assert rtv == pytest.approx((p.nx - 1) * p.nz * (gam / 1000.0 - p.kx1) / nt, rel=1e-9)
    assert rsv == pytest.approx(0.0, abs=1e-9)
    beta = 5.0                                   # c = c0 + beta z^2 (z in mm): d2c/dz2 = 2 beta
    c2 = 1500.0 + beta * ((Z - p.z0) * 1e3) ** 2
    rtv2, rsv2 = o.regularizers(1.0 / c2)
    ns_ = (p.nx - 2) * p.nz + p.nx * (p.nz - 2)
    assert rsv2 == pytest.approx(p.nx * (p.nz - 2) * (2 * beta / 1000.0 - p.kz2) / ns_, rel=1e-7)
    # a gradient inside the deadzone (5 m/s per mm < 10 m/s per mm) costs nothing
    rtv3, _ = o.regularizers(1.0 / (1500.0 + 5.0 * (X - p.x0) * 1e3))
    assert rtv3 == 0.0


def test_mean_speed_is_the_mean_of_c_on_a_two_valued_map():
    """c_med of Sec. III-A is the mean sound speed of the grid: on a map with n1 nodes at
    c1 and n2 at c2 it is (n1 c1 + n2 c2) / n, which differs from the harmonic mean and
    from 1 / mean(s)."""
    p = small(nx=7, nz=5)
    o = oracle.Oracle(p)
    c = np.full((p.nz, p.nx), 1450.0)
    c[:2, :] = 1600.0
    c[4, 5] = 1600.0
    n1, n2 = int((c == 1600.0).sum()), int((c == 1450.0).sum())
    cmed = o.mean_speed(1.0 / c)
    assert cmed == pytest.approx((n1 * 1600.0 + n2 * 1450.0) / (n1 + n2), rel=1e-14)
    harmonic = (n1 + n2) / (n1 / 1600.0 + n2 / 1450.0)
    assert abs(cmed - harmonic) > 1.0


def test_regularizer_gradient_matches_finite_differences():
    p = small(nx=7, nz=6)
    o = oracle.Oracle(p)
    rng = np.random.default_rng(4)
    s = 1.0 / (1500.0 + 30.0 * rng.standard_normal((p.nz, p.nx)))
    g = o.regularizer_grad(s)

    def R(sv):
        a, b = o.regularizers(sv)
        return p.w1 * a + p.w2 * b

    for k in rng.choice(s.size, 12, replace=False):
        h = 1e-9 * s.flat[k]
        sp, sm = s.copy(), s.copy()
        sp.flat[k] += h
        sm.flat[k] -= h
        fd = (R(sp) - R(sm)) / (2 * h)
        assert g.flat[k] == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.abs(g).max())


# ---------------------------------------------------------------- adjoint (Fig. 1g)
def test_cmpe_adjoint_matches_finite_differences():
    p = small(n_ang=1, n_rad=2, patch_w=3)
    o = oracle.Oracle(p)
    rng = np.random.default_rng(7)
    nb, npix = o.nsub ** 2, p.npix
    B = rng.standard_normal((nb, npix)) + 1j * rng.standard_normal((nb, npix))
    ones = np.ones((p.n_patch, o.npair), np.uint8)
    L, z, rho, mask, M = o.cmpe(B, mask_in=ones)
    G = o.cmpe_adjoint(B, z, ones, M)
    for _ in range(15):
        b, q = int(rng.integers(nb)), int(rng.integers(npix))
        for d, part in ((1e-7, "re"), (1e-7j, "im")):
            Bp, Bm = B.copy(), B.copy()
            Bp[b, q] += d
            Bm[b, q] -= d
            fd = (o.cmpe(Bp, mask_in=ones)[0] - o.cmpe(Bm, mask_in=ones)[0]) / 2e-7
            an = G[b, q].real if part == "re" else G[b, q].imag
            assert an == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_ray_adjoint_dot_product(tiny):
    """<A v, w> = <v, A^T w> for the linear map s -> ray sums (exit angles frozen)."""
    o = oracle.Oracle(tiny)
    rng = np.random.default_rng(8)
    s0 = tiny.initial_slowness().astype(np.float64)
    T0, apod, phi = o.delays(s0)
    v = 1e-5 * rng.standard_normal(s0.shape)
    Tv, _, _ = o.delays(s0 + v, apod_in=apod, phi_in=phi)
    Av = Tv - T0
    w = rng.standard_normal(T0.shape) * apod
    ATw = o.ray_adjoint(s0, phi, apod, w)
    lhs = float((Av * w).sum())
    rhs = float((v * ATw).sum())
    assert lhs == pytest.approx(rhs, rel=1e-9)


def test_full_gradient_matches_central_differences():
    """dL/ds of Eq. 12 vs central differences, with apodization, CMPE mask and exit
    angles frozen (the constants of the adjoint)."""
    p = small(n_ang=2, n_rad=2, patch_w=3, nx=8, nz=8)
    o = oracle.Oracle(p)
    psi = synth.simulate(p, 400, seed=11)
    rng = np.random.default_rng(9)
    s = (1.0 / (1510.0 + 20.0 * rng.standard_normal((p.nz, p.nx))))
    parts, g, mask, M = o.loss_grad(psi, s)
    _, apod, phi = o.delays(s)
    assert M > 0

    def loss(sv):
        return o.loss_grad(psi, sv, apod_in=apod, mask_in=mask, phi_in=phi, grad=False)[0][0]

    checked = 0
    for k in np.argsort(-np.abs(g).ravel())[:10]:
        h = 1e-8 * s.flat[k]
        sp, sm = s.copy(), s.copy()
        sp.flat[k] += h
        sm.flat[k] -= h
        fd = (loss(sp) - loss(sm)) / (2 * h)
        assert g.flat[k] == pytest.approx(fd, rel=1e-5), k
        checked += 1
    assert checked == 10


# ---------------------------------------------------------------- optimiser (Eq. 9)
def test_adam_first_step_is_signed_learning_rate():
    """Step 1 of Adam on c (km/s): m_hat = g_c, v_hat = g_c^2, so c moves by
    -lr * g_c / (|g_c| + eps), g_c = dL/dc = -dL/ds * 1000 s^2 (Eq. 9 up to the step
    normalisation)."""
    o = oracle.Oracle(small())
    s = 1.0 / np.array([1540.0, 1450.0, 1600.0, 1500.0, 1540.0])
    g = np.array([3.0, -2.0, 1e-3, -5e4, 0.0])
    lr = 0.01
    s1, m, v = o.adam(s, g, np.zeros(5), np.zeros(5), 1, lr)
    gc = -g * 1000.0 * s * s
    dc = 1e-3 / s1 - 1e-3 / s                    # km/s
    np.testing.assert_allclose(dc, -lr * gc / (np.abs(gc) + 1e-8), rtol=1e-9, atol=1e-13)
    # a positive dL/ds (slower is worse) raises the speed by lr km/s = 10 m/s
    assert 1.0 / s1[0] - 1540.0 == pytest.approx(10.0, rel=1e-4)   # eps = 1e-8 vs |g_c| ~ 1e-3
    # beta1 = beta2 = 0 keeps it a sign step at every iteration
    s2, _, _ = o.adam(s1, -g, m, v, 2, lr, beta1=0.0, beta2=0.0)
    gc1 = g * 1000.0 * s1 * s1
    np.testing.assert_allclose(1e-3 / s2 - 1e-3 / s1, -lr * gc1 / (np.abs(gc1) + 1e-8), rtol=1e-9, atol=1e-13)


def test_plain_gradient_step_of_eq9_lands_on_the_minimum_of_a_quadratic():
    """Eq. 9 as printed, c <- c - lr dL/dc with c in km/s: for L = k/2 (c - c*)^2 one step
    of lr = 1/k lands on c* exactly; the gradient is handed over as dL/ds, so a wrong sign
    or unit in the chain rule c = 1/(1000 s) misses c*."""
    o = oracle.Oracle(small())
    c_star = np.array([1.45, 1.56, 1.60, 1.52])               # km/s
    c0 = np.array([1.54, 1.50, 1.55, 1.52])
    k = 3.0
    s0 = 1e-3 / c0
    dLdc = k * (c0 - c_star)
    dLds = dLdc * (-1e-3 / s0 ** 2)                     # c = 1e-3 / s: dc/ds = -1e-3 / s^2
    s1 = o.gd(s0, dLds, 1.0 / k)
    np.testing.assert_allclose(1e-3 / s1, c_star, rtol=1e-13)


# ---------------------------------------------------------------- MLP reference
def test_mlp_oracle_gradient_matches_finite_differences():
    from oracle import mlp_oracle as mo
    rng = np.random.default_rng(12)
    p = mo.init(3) + 0.01 * rng.standard_normal(mo.NPARAM)
    X = rng.uniform(-1, 1, (16, 4))
    Y = rng.uniform(-1, 1, (16, 2))
    L, g = mo.forward_backward(p, X, Y)
    for k in rng.choice(mo.NPARAM, 25, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (mo.forward_backward(pp, X, Y)[0] - mo.forward_backward(pm, X, Y)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_mlp_oracle_closed_forms():
    """Zero weights: output = b4, loss = mean squared error, d loss / d b4 = 2 mean(err);
    bf16 rounding keeps exactly representable values and rounds 1 + 2^-9 to 1."""
    from oracle import mlp_oracle as mo
    d = {n: np.zeros(s) for n, s in mo.SIZES}
    d["b4"] = np.array([0.3, -0.2])
    X = np.ones((8, 4))
    Y = np.zeros((8, 2))
    L, g = mo.forward_backward(mo.pack(d), X, Y)
    assert L == pytest.approx(0.3 ** 2 + 0.2 ** 2)
    gb4 = mo.unpack(g)["b4"]
    np.testing.assert_allclose(gb4, [0.6, -0.4])
    assert mo.bf16(np.array([1.0 + 2 ** -9]))[0] == 1.0
    assert mo.bf16(np.array([0.75]))[0] == 0.75


# ---------------------------------------------------------------- image metrics (Sec. III-F)
def test_metrics_closed_forms():
    """Coherence factor, lag-one coherence, contrast, CNR and gCNR on inputs whose
    values are known in closed form."""
    from oracle import metrics as M
    n, P = 8, 5
    same = np.ones((n, P), complex) * (0.3 + 0.4j)
    assert np.allclose(M.coherence_factor(same), 1.0)                 # coherent channels
    spread = np.exp(2j * np.pi * np.arange(n) / n)[:, None] * np.ones(P)
    assert np.allclose(M.coherence_factor(spread), 0.0, atol=1e-15)   # phases cancel
    one = np.zeros((n, P), complex)
    one[3] = 2.0
    assert np.allclose(M.coherence_factor(one), 1.0 / n)              # a single channel
    sel = np.ones(P, bool)
    assert M.lag_one_coherence(same, sel) == pytest.approx(1.0)
    alt = ((-1.0) ** np.arange(n))[:, None] * np.ones(P)
    assert M.lag_one_coherence(alt.astype(complex), sel) == pytest.approx(-1.0)
    env = np.array([1.0, 3.0, 9.0, 11.0, 5.0])
    roi = np.array([1, 1, 2, 2, 0])
    c, cnr, g, mi, mo = M.contrast_cnr_gcnr(env, roi)
    assert c == pytest.approx(20 * math.log10(2.0 / 10.0), rel=1e-14)
    assert cnr == pytest.approx(8.0 / math.sqrt(2.0), rel=1e-14)
    assert g == pytest.approx(1.0) and (mi, mo) == (2.0, 10.0)        # disjoint histograms
    env2 = np.array([1.0, 2.0, 1.0, 2.0])
    assert M.contrast_cnr_gcnr(env2, np.array([1, 1, 2, 2]))[2] == pytest.approx(0.0)   # identical
    assert M.speed_mae([1500.0, 1520.0], [1510.0, 1510.0]) == pytest.approx(10.0)


def test_cmcc_matches_cmpe_correlations():
    """The mean common-midpoint correlation equals the mean of the C oracle's CMPE
    correlation coefficients (an independent implementation of the same sums); images
    identical along each common-midpoint pair give 1."""
    from oracle import metrics as M
    p = small()
    o = oracle.Oracle(p)
    rng = np.random.default_rng(4)
    B = rng.standard_normal((p.nsub ** 2, p.npix)) + 1j * rng.standard_normal((p.nsub ** 2, p.npix))
    _, _, rho, _, _ = o.cmpe(B)
    assert M.cmcc(B, p.nsub, p.n_patch, p.patch_npix) == pytest.approx(rho.mean(), rel=1e-12)
    # images that depend only on i + j (the common midpoint) are identical in each pair
    C = np.empty_like(B)
    for i in range(p.nsub):
        for j in range(p.nsub):
            C[i * p.nsub + j] = B[(i + j) % B.shape[0]]
    assert M.cmcc(C, p.nsub, p.n_patch, p.patch_npix) == pytest.approx(1.0, rel=1e-12)


# ---------------------------------------------------------------- all-core build
def test_openmp_build_matches_single_thread():
    """The OpenMP build of the same oracle source (used for full-size checks and the
    all-core CPU baseline) gives the single-threaded loss, images and mask bit for bit;
    only the ray adjoint's per-node sums are reduced in another order."""
    p = small(n_ang=3, n_rad=3, patch_w=3)
    psi = synth.simulate(p, 600, seed=21)
    s = 1.0 / (1540.0 + 20.0 * np.random.default_rng(3).standard_normal((p.nz, p.nx)))
    serial = oracle.Oracle(p)
    par = oracle.Oracle(p, parallel=True)
    a, b = serial.loss_grad(psi, s), par.loss_grad(psi, s)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2]) and a[3] == b[3]
    assert np.linalg.norm(a[1] - b[1]) <= 1e-12 * np.linalg.norm(a[1])
    T, apod, _ = serial.delays(s)
    T2, apod2, _ = par.delays(s)
    assert np.array_equal(T, T2) and np.array_equal(apod, apod2)
    assert np.array_equal(serial.das(psi, T, apod), par.das(psi, T, apod))
    assert oracle.omp_threads() >= 1


# ---------------------------------------------------------------- dynamic sweep grid (Sec. III-A)
def test_dynamic_grid_closed_form():
    """At speed c0 a patch's depth below the lens and its pixel offsets are multiplied
    by c0 / c_ref, its direction from the lens centre is kept; c0 = c_ref is the
    identity."""
    p = small(n_ang=3, n_rad=2, patch_w=3)
    o = oracle.Oracle(p)
    x1, z1 = o.dynamic_pixels(1540.0, 1540.0)
    np.testing.assert_allclose(x1, p.pix_x, atol=1e-15)
    np.testing.assert_allclose(z1, p.pix_z, atol=1e-15)
    k = 1.1
    x, z = o.dynamic_pixels(1.1 * 1540.0, 1540.0)
    n = p.patch_npix
    for P in range(p.n_patch):
        sl = slice(P * n, (P + 1) * n)
        c0 = np.array([p.pix_x[sl].mean(), p.pix_z[sl].mean()])
        c1 = np.array([x[sl].mean(), z[sl].mean()])
        v0, v1 = c0 - [p.arc_cx, p.arc_cz], c1 - [p.arc_cx, p.arc_cz]
        assert np.linalg.norm(v1) - p.lens_radius == pytest.approx(k * (np.linalg.norm(v0) - p.lens_radius),
                                                                   rel=1e-12)
        assert v0[0] * v1[1] - v0[1] * v1[0] == pytest.approx(0.0, abs=1e-15)     # same direction
        np.testing.assert_allclose(x[sl] - c1[0], k * (p.pix_x[sl] - c0[0]), atol=1e-15)
        np.testing.assert_allclose(z[sl] - c1[1], k * (p.pix_z[sl] - c0[1]), atol=1e-15)


def test_dynamic_grid_keeps_a_point_scatterer_on_its_patch_centre():
    """What the dynamic grid is for: beamformed at a wrong uniform speed c0, a point
    scatterer sitting on a patch's centre pixel (at the reference speed) still peaks on
    that patch's centre pixel when the patch moves with the dynamic grid, because its
    echo's apparent depth below the lens scales with c0; on the static grid it peaks
    elsewhere in the patch."""
    p = synth.config_tiny(n_ang=1, n_rad=1, patch_w=9, depth_min=20e-3)
    c_true = 1500.0
    p.medium = synth.Medium(speeds=[c_true])
    centre = p.patch_npix // 2
    T1 = synth.oneway_times(p, np.array([p.pix_x[centre]]), np.array([p.pix_z[centre]]))
    psi = synth.echoes(p, T1, np.array([1.0]))
    o = oracle.Oracle(p)
    for c0 in (0.95 * c_true, 1.05 * c_true):
        s = np.full((p.nz, p.nx), 1.0 / c0)
        peaks = {}
        for name, (x, z) in (("dynamic", o.dynamic_pixels(c0, c_true)), ("static", (p.pix_x, p.pix_z))):
            q = dataclasses.replace(p, pix_x=np.asarray(x), pix_z=np.asarray(z))
            oq = oracle.Oracle(q)
            T, apod, _ = oq.delays(s)
            peaks[name] = int(np.argmax(np.abs(oq.das(psi, T, apod).sum(0))))
        assert peaks["dynamic"] == centre, (c0, peaks)
        assert peaks["static"] != centre, (c0, peaks)
