"""Seeded synthetic problems and acquisitions (input generator).

This module builds the inputs that both the CUDA library and the oracle
consume: the geometry of a curvilinear array with a lens, the image patches,
the slowness grid, the hyperparameters of the paper's Table II, and demodulated
full-synthetic-aperture channel data simulated from point scatterers in a
layered medium.  It holds none of the autofocusing method's arithmetic.

Every geometric quantity is rounded to the nearest float32 value (and kept as
float64), so that a float32 device copy and the float64 oracle see exactly the
same positions.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_GPU_LIB_PATH = os.path.join(_HERE, "libsynth_gpu.so")
_lib = None
_gpu_lib = None

C_REF = 1540.0  # beamforming reference speed (m/s); lambda/2 pixel spacing uses it
C_UNIT = 1000.0  # Eq. 9-11 take the sound speed in km/s (Table II's LR and kappa values)


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so (OpenMP, portable x86-64 code)."""
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-shared", "-fPIC", "-o", _LIB_PATH, src, "-lm"])
    return _LIB_PATH


def build_gpu(force: bool = False) -> str:
    """Compile synth_gpu.cu (the GPU echo simulator) into libsynth_gpu.so for sm_103a."""
    src = os.path.join(_HERE, "synth_gpu.cu")
    if force or not os.path.exists(_GPU_LIB_PATH) or os.path.getmtime(_GPU_LIB_PATH) < os.path.getmtime(src):
        nvcc = os.environ.get("NVCC", "nvcc")
        subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
                               "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-o", _GPU_LIB_PATH, src])
    return _GPU_LIB_PATH


class _Medium(ctypes.Structure):
    _fields_ = [("n_if", ctypes.c_int),
                ("base", ctypes.c_double * 8), ("amp", ctypes.c_double * 8),
                ("period", ctypes.c_double * 8), ("phase", ctypes.c_double * 8),
                ("slow", ctypes.c_double * 9)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.sy_oneway_times.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        ctypes.POINTER(_Medium), ctypes.c_int, dp, dp, dp]
        lib.sy_echoes.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.POINTER(ctypes.c_float)]
        lib.sy_segment_time.argtypes = [ctypes.POINTER(_Medium), ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double]
        lib.sy_segment_time.restype = ctypes.c_double
        lib.sy_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _load_gpu():
    global _gpu_lib
    if _gpu_lib is None:
        build_gpu()
        lib = ctypes.CDLL(_GPU_LIB_PATH)
        vp, d, i, ll = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_longlong
        lib.sy_gpu_oneway_times.argtypes = [i, vp, vp, d, d, d, d, d, i, ctypes.POINTER(_Medium), ll, vp, vp, vp]
        lib.sy_gpu_oneway_times.restype = i
        lib.sy_gpu_echoes.argtypes = [i, ll, vp, vp, i, d, d, d, d, d, vp]
        lib.sy_gpu_echoes.restype = i
        _gpu_lib = lib
    return _gpu_lib


def f32(x):
    """Round to the nearest float32 value, returned as float64."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclasses.dataclass
class Medium:
    """True layered medium: interface i at z = base + amp sin(2 pi x / period + phase)."""
    speeds: list
    base: list = dataclasses.field(default_factory=list)
    amp: list = dataclasses.field(default_factory=list)
    period: list = dataclasses.field(default_factory=list)
    phase: list = dataclasses.field(default_factory=list)
    cysts: list = dataclasses.field(default_factory=list)   # (x, z, radius): no scatterers inside

    def to_c(self) -> _Medium:
        m = _Medium()
        m.n_if = len(self.base)
        for i in range(m.n_if):
            m.base[i] = self.base[i]
            m.amp[i] = self.amp[i]
            m.period[i] = self.period[i] if self.period[i] else 1.0
            m.phase[i] = self.phase[i]
        for i, c in enumerate(self.speeds):
            m.slow[i] = 1.0 / c
        return m

    def speed_at(self, x, z):
        x = np.asarray(x, np.float64)
        z = np.asarray(z, np.float64)
        layer = np.zeros(np.broadcast(x, z).shape, np.int64)
        for i in range(len(self.base)):
            zi = self.base[i] + self.amp[i] * np.sin(2 * np.pi * x / (self.period[i] or 1.0) + self.phase[i])
            layer = np.where(z > zi, i + 1, layer)
        return np.asarray(self.speeds, np.float64)[layer]


@dataclasses.dataclass
class Problem:
    """Everything an autofocus run needs besides the channel data and the slowness map."""
    name: str
    # array and lens (Sec. II-A, II-B, III-B; Table I)
    elem_x: np.ndarray
    elem_z: np.ndarray
    arc_cx: float
    arc_cz: float
    arc_radius: float
    d_lens: float
    c_lens: float
    t_ttp: float
    lens_mode: int            # 0 bent-ray (curved lens), 1 no lens, 2 bent-ray (flat lens)
    # apodization (Eq. 4)
    fnum: float
    apod_mode: int            # 0 |x'| <= z'/(2F), 1 printed (F/2) z'
    # image patches (patch-major pixels)
    n_patch: int
    patch_npix: int
    pix_x: np.ndarray
    pix_z: np.ndarray
    # slowness grid (Sec. III-A)
    nx: int
    nz: int
    x0: float
    z0: float
    dx: float
    dz: float
    nseg: int
    # channel data
    ns: int
    fs: float
    fd: float
    fc: float
    t0: float
    sub_width: int
    # Table II
    rho_thresh: float
    w1: float
    kx1: float
    kz1: float
    w2: float
    kx2: float
    kz2: float
    lr: float
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8
    c_ref: float = C_REF      # reference speed of the patch geometry (lambda/2 pixels)
    c_unit: float = C_UNIT    # m/s per unit of the speed that Eq. 9-11 act on (km/s)
    optimizer: int = 0        # update of Eq. 9: 0 Adam on c, 1 the plain gradient step as printed
    medium: Optional[Medium] = None
    sector_half_angle: float = 0.0    # curved array: sector half angle; linear: half width (m)
    depth_range: tuple = (0.0, 0.0)
    lens_z: float = 0.0       # flat lens (lens_mode 2): outer surface z = lens_z

    @property
    def ne(self) -> int:
        return int(self.elem_x.shape[0])

    @property
    def npix(self) -> int:
        return int(self.n_patch * self.patch_npix)

    @property
    def nsub(self) -> int:
        return self.ne // self.sub_width

    @property
    def lens_radius(self) -> float:
        return float(f32(self.arc_radius + self.d_lens))

    def initial_slowness(self, c: float = C_REF) -> np.ndarray:
        """Uniform slowness grid [nz][nx] (float32) at speed c."""
        return np.full((self.nz, self.nx), 1.0 / c, dtype=np.float32)

    def true_speed_grid(self) -> np.ndarray:
        gx = self.x0 + self.dx * np.arange(self.nx)
        gz = self.z0 + self.dz * np.arange(self.nz)
        X, Z = np.meshgrid(gx, gz)
        return self.medium.speed_at(X, Z)


# Table II (phantom L12-3v, phantom C5-2v and in vivo C5-2v columns)
TABLE2 = {
    "phantom_l12": dict(lr=0.0030, w1=7.0, kx1=0.0010, kz1=0.0200, w2=0.0, kx2=0.0,
                        kz2=0.0, rho_thresh=0.9, fnum=0.75, nseg=32),
    "phantom_c5": dict(lr=0.0030, w1=10.0, kx1=0.0100, kz1=0.0100, w2=100.0, kx2=0.0010,
                       kz2=0.0010, rho_thresh=0.9, fnum=0.5, nseg=32),
    "invivo_c5": dict(lr=0.0500, w1=100.0, kx1=0.0100, kz1=0.0100, w2=100.0, kx2=0.0020,
                      kz2=0.0020, rho_thresh=0.9, fnum=0.4, nseg=64),
}


def curvilinear_problem(name: str, *, ne: int, radius: float, pitch: float, fc: float,
                        d_lens: float, c_lens: float, ns: int, fs: float, nx: int, nz: int,
                        n_ang: int, n_rad: int, patch_w: int, depth_min: float, depth_max: float,
                        sub_width: int, hyper: dict, medium: Optional[Medium] = None,
                        t_ttp: float = 0.0, t0: float = 0.0, lens_mode: int = 0,
                        apod_mode: int = 0, sector_frac: float = 0.8,
                        grid_margin: float = 2e-3, cover_speeds: Optional[tuple] = None) -> Problem:
    """Curvilinear array on an arc of `radius` about (0, -radius) (apex at the origin),
    a concentric lens shell of thickness d_lens, and a regular polar grid of square
    patches of patch_w x patch_w pixels at lambda/2 (lambda at 1540 m/s)."""
    th = (np.arange(ne) - (ne - 1) / 2.0) * pitch / radius
    ex = f32(radius * np.sin(th))
    ez = f32(radius * np.cos(th) - radius)
    cx, cz = 0.0, float(f32(-radius))
    RL = radius + d_lens
    half = sector_frac * abs(th[-1]) if ne > 1 else 0.2
    ang = np.linspace(-half, half, n_ang) if n_ang > 1 else np.zeros(1)
    rad = RL + (np.linspace(depth_min, depth_max, n_rad) if n_rad > 1 else np.array([depth_min]))
    step = C_REF / fc / 2.0
    h = (patch_w - 1) / 2.0
    px, pz = [], []
    for r in rad:
        for a in ang:
            ur = np.array([np.sin(a), np.cos(a)])       # radial unit vector
            ut = np.array([np.cos(a), -np.sin(a)])      # tangential unit vector
            c = np.array([cx, cz]) + r * ur
            for b in range(patch_w):
                for k in range(patch_w):
                    q = c + (k - h) * step * ut + (b - h) * step * ur
                    px.append(q[0])
                    pz.append(q[1])
    px = f32(np.array(px))
    pz = f32(np.array(pz))
    # grid box also covering the patches as moved by a global-speed sweep over
    # cover_speeds (depths below the lens and in-patch offsets scaled by c / C_REF)
    bx, bz = [px], [pz]
    if cover_speeds is not None:
        qx = px.reshape(n_ang * n_rad, patch_w * patch_w)
        qz = pz.reshape(n_ang * n_rad, patch_w * patch_w)
        ccx, ccz = qx.mean(1, keepdims=True), qz.mean(1, keepdims=True)
        rho = np.hypot(ccx - cx, ccz - cz)
        for c in cover_speeds:
            k = c / C_REF
            r2 = RL + (rho - RL) * k
            bx.append((cx + r2 * (ccx - cx) / rho + k * (qx - ccx)).ravel())
            bz.append((cz + r2 * (ccz - cz) / rho + k * (qz - ccz)).ravel())
    bx, bz = np.concatenate(bx), np.concatenate(bz)
    # grid: bounding box of the lens surface over the aperture and every pixel
    lens_th = np.linspace(th[0], th[-1], 64) if ne > 1 else np.zeros(1)
    lx = cx + RL * np.sin(lens_th)
    lz = cz + RL * np.cos(lens_th)
    xmin = min(bx.min(), lx.min(), ex.min()) - grid_margin
    xmax = max(bx.max(), lx.max(), ex.max()) + grid_margin
    zmin = min(bz.min(), lz.min(), ez.min()) - grid_margin
    zmax = max(bz.max(), lz.max()) + grid_margin
    dx = float(f32((xmax - xmin) / (nx - 1)))
    dz = float(f32((zmax - zmin) / (nz - 1)))
    return Problem(
        name=name, elem_x=ex, elem_z=ez, arc_cx=cx, arc_cz=cz, arc_radius=float(f32(radius)),
        d_lens=float(f32(d_lens)), c_lens=float(f32(c_lens)), t_ttp=float(f32(t_ttp)),
        lens_mode=lens_mode, fnum=float(f32(hyper["fnum"])), apod_mode=apod_mode,
        n_patch=n_ang * n_rad, patch_npix=patch_w * patch_w, pix_x=px, pix_z=pz,
        nx=nx, nz=nz, x0=float(f32(xmin)), z0=float(f32(zmin)), dx=dx, dz=dz,
        nseg=int(hyper["nseg"]), ns=ns, fs=float(f32(fs)), fd=float(f32(fc)), fc=fc,
        t0=float(f32(t0)), sub_width=sub_width, rho_thresh=float(f32(hyper["rho_thresh"])),
        w1=hyper["w1"], kx1=hyper["kx1"], kz1=hyper["kz1"], w2=hyper["w2"],
        kx2=hyper["kx2"], kz2=hyper["kz2"], lr=hyper["lr"], medium=medium,
        sector_half_angle=float(half), depth_range=(depth_min, depth_max))


def linear_problem(name: str, *, ne: int, pitch: float, fc: float, d_lens: float, c_lens: float,
                   ns: int, fs: float, nx: int, nz: int, n_lat: int, n_ax: int, patch_w: int,
                   depth_min: float, depth_max: float, sub_width: int, hyper: dict,
                   medium: Optional[Medium] = None, t_ttp: float = 0.0, t0: float = 0.0,
                   lens_mode: int = 2, apod_mode: int = 0, lat_frac: float = 0.8,
                   grid_margin: float = 1e-3) -> Problem:
    """Linear array on z = 0 (elements along x), a flat lens whose outer surface is the
    line z = d_lens, and a rectangular grid of square patches of patch_w x patch_w
    pixels at lambda/2 (lambda at 1540 m/s) below the lens."""
    ex = f32((np.arange(ne) - (ne - 1) / 2.0) * pitch)
    ez = f32(np.zeros(ne))
    lz = float(f32(d_lens))
    half = lat_frac * abs(float(ex[-1])) if ne > 1 else 1e-3
    lat = np.linspace(-half, half, n_lat) if n_lat > 1 else np.zeros(1)
    ax = lz + (np.linspace(depth_min, depth_max, n_ax) if n_ax > 1 else np.array([depth_min]))
    step = C_REF / fc / 2.0
    h = (patch_w - 1) / 2.0
    px, pz = [], []
    for zc in ax:
        for xc in lat:
            for b in range(patch_w):
                for k in range(patch_w):
                    px.append(xc + (k - h) * step)
                    pz.append(zc + (b - h) * step)
    px = f32(np.array(px))
    pz = f32(np.array(pz))
    # grid: bounding box of the lens line over the aperture and every pixel
    xmin = min(px.min(), ex.min()) - grid_margin
    xmax = max(px.max(), ex.max()) + grid_margin
    zmin = min(ez.min(), lz) - grid_margin
    zmax = pz.max() + grid_margin
    dx = float(f32((xmax - xmin) / (nx - 1)))
    dz = float(f32((zmax - zmin) / (nz - 1)))
    return Problem(
        name=name, elem_x=ex, elem_z=ez, arc_cx=0.0, arc_cz=0.0, arc_radius=0.0,
        d_lens=float(f32(d_lens)), c_lens=float(f32(c_lens)), t_ttp=float(f32(t_ttp)),
        lens_mode=lens_mode, fnum=float(f32(hyper["fnum"])), apod_mode=apod_mode,
        n_patch=n_lat * n_ax, patch_npix=patch_w * patch_w, pix_x=px, pix_z=pz,
        nx=nx, nz=nz, x0=float(f32(xmin)), z0=float(f32(zmin)), dx=dx, dz=dz,
        nseg=int(hyper["nseg"]), ns=ns, fs=float(f32(fs)), fd=float(f32(fc)), fc=fc,
        t0=float(f32(t0)), sub_width=sub_width, rho_thresh=float(f32(hyper["rho_thresh"])),
        w1=hyper["w1"], kx1=hyper["kx1"], kz1=hyper["kz1"], w2=hyper["w2"],
        kx2=hyper["kx2"], kz2=hyper["kz2"], lr=hyper["lr"], medium=medium,
        sector_half_angle=float(half), depth_range=(depth_min, depth_max), lens_z=lz)


def config_linear_tiny(**over) -> Problem:
    """32-element, 0.2 mm-pitch linear array at 6 MHz with the L12-3v lens of Table I
    (0.67 mm at 1049.4 m/s, t_ttp 578.3 ns); 32 x 32 x 1024 samples at 24 MHz; 16 x 16
    grid; 16 patches of 5 x 5 pixels from 4 to 20 mm below the lens; Table II L12-3v
    column; two-layer medium (6 mm at 1575 m/s over 1516 m/s, a tissue layer on a
    phantom)."""
    kw = dict(ne=32, pitch=0.2e-3, fc=6e6, d_lens=0.67e-3, c_lens=1049.4, t_ttp=578.3e-9,
              ns=1024, fs=24e6, nx=16, nz=16, n_lat=4, n_ax=4, patch_w=5,
              depth_min=4e-3, depth_max=20e-3, sub_width=4, hyper=TABLE2["phantom_l12"],
              medium=Medium(speeds=[1575.0, 1516.0], base=[6.67e-3], amp=[0.0], period=[0.0],
                            phase=[0.0]))
    kw.update(over)
    return linear_problem("l32_fsa1024", **kw)


def image_grid_problem(problem: Problem, n_lat: int, n_ax: int, depth: tuple,
                       half: Optional[float] = None) -> Problem:
    """The same curvilinear acquisition imaged on a dense polar grid: n_ax depths
    below the lens (depth[0]..depth[1]) by n_lat angles (+-half, default 0.9 of the
    sector), one patch per depth row (patch-major pixels).  The slowness grid is
    unchanged, so the pixels must lie inside its box."""
    RL = problem.lens_radius
    half = 0.9 * problem.sector_half_angle if half is None else half
    ang = np.linspace(-half, half, n_lat)
    rad = RL + np.linspace(depth[0], depth[1], n_ax)
    px = problem.arc_cx + rad[:, None] * np.sin(ang)[None, :]
    pz = problem.arc_cz + rad[:, None] * np.cos(ang)[None, :]
    return dataclasses.replace(problem, n_patch=n_ax, patch_npix=n_lat, pix_x=f32(px.ravel()),
                               pix_z=f32(pz.ravel()))


def config_tiny(**over) -> Problem:
    """32-element, 40 mm-radius, 0.4 mm-pitch, 3 MHz array; 1.0 mm lens at 1000 m/s;
    32 x 32 x 1024 samples at 12 MHz; 16 x 16 grid; 64 patches of 5 x 5 pixels;
    two-layer medium (15 mm at 1450 m/s over 1570 m/s)."""
    kw = dict(ne=32, radius=40e-3, pitch=0.4e-3, fc=3e6, d_lens=1.0e-3, c_lens=1000.0,
              ns=1024, fs=12e6, nx=16, nz=16, n_ang=8, n_rad=8, patch_w=5,
              depth_min=8e-3, depth_max=50e-3, sub_width=4, hyper=TABLE2["phantom_c5"],
              medium=Medium(speeds=[1450.0, 1570.0], base=[15e-3], amp=[0.0], period=[0.0],
                            phase=[0.0]))
    kw.update(over)
    return curvilinear_problem("c32_fsa1024", **kw)


def config_full(seed: int = 20261204, **over) -> Problem:
    """128-element, 60 mm-radius, 0.35 mm-pitch, 3.5 MHz array; 1.2 mm lens at 1000 m/s;
    128 x 128 x 3072 samples at 14 MHz; 128 x 128 grid; 400 patches of 9 x 9 pixels;
    skin 3 mm (1600) / fat 10-25 mm (1440) with a 3 mm wavy lower interface / liver
    (1560) with two 8 mm anechoic cysts."""
    rng = np.random.default_rng(seed)
    h_fat = rng.uniform(10e-3, 25e-3)
    ph = rng.uniform(0, 2 * np.pi)
    medium = Medium(speeds=[1600.0, 1440.0, 1560.0], base=[3e-3, 3e-3 + h_fat],
                    amp=[0.0, 3e-3], period=[0.0, 20e-3], phase=[0.0, ph])
    # Table II in vivo column, except the learning rate of the default Adam update: 0.05
    # km/s moves every node by 50 m/s per Adam step and the map leaves the speed range
    # within a few iterations, so the C5-2v phantom value (0.003, 3 m/s per step) is used.
    # Eq. 9 as printed (optimizer=1, a plain gradient step) runs the in vivo value.
    hyper = dict(TABLE2["invivo_c5"], lr=TABLE2["phantom_c5"]["lr"])
    kw = dict(ne=128, radius=60e-3, pitch=0.35e-3, fc=3.5e6, d_lens=1.2e-3, c_lens=1000.0,
              ns=3072, fs=14e6, nx=128, nz=128, n_ang=20, n_rad=20, patch_w=9,
              depth_min=10e-3, depth_max=140e-3, sub_width=8, hyper=hyper,
              medium=medium)
    kw.update(over)
    p = curvilinear_problem("c128_fsa3072", **kw)
    # cysts: 8 mm diameter, seeded positions in the liver inside the sector
    cysts = []
    for _ in range(2):
        a = rng.uniform(-0.6, 0.6) * p.sector_half_angle
        d = rng.uniform(max(40e-3, 3e-3 + h_fat + 10e-3), 120e-3)
        r = p.lens_radius + d
        cysts.append((p.arc_cx + r * math.sin(a), p.arc_cz + r * math.cos(a), 4e-3))
    medium.cysts = cysts
    return p


def pulse_sigma(fc: float, frac_bw: float = 0.7) -> float:
    """Std of the Gaussian envelope whose -6 dB bandwidth is frac_bw * fc."""
    sigma_f = frac_bw * fc / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    return 1.0 / (2.0 * math.pi * sigma_f)


def sector_scatterers(problem: Problem, n: int, seed: int, depth=(2e-3, None),
                      half_angle: Optional[float] = None):
    """n scatterers uniform in area over the imaging sector, N(0,1) amplitudes,
    none inside the medium's cysts."""
    rng = np.random.default_rng(seed)
    d0 = depth[0]
    d1 = depth[1] if depth[1] is not None else problem.depth_range[1] + 10e-3
    if problem.arc_radius == 0.0:
        # linear array: a rectangle below the lens, 15 % wider than the patches
        half = 1.15 * problem.sector_half_angle + 2e-3
        x = rng.uniform(-half, half, n)
        z = rng.uniform(problem.lens_z + d0, problem.lens_z + d1, n)
    else:
        RL = problem.lens_radius
        half = half_angle if half_angle is not None else 1.15 * problem.sector_half_angle
        r = np.sqrt(rng.uniform((RL + d0) ** 2, (RL + d1) ** 2, n))
        a = rng.uniform(-half, half, n)
        x = problem.arc_cx + r * np.sin(a)
        z = problem.arc_cz + r * np.cos(a)
    amp = rng.standard_normal(n)
    keep = np.ones(n, bool)
    if problem.medium is not None:
        for (cxs, czs, rad) in problem.medium.cysts:
            keep &= (x - cxs) ** 2 + (z - czs) ** 2 > rad ** 2
    return x[keep], z[keep], amp[keep]


def oneway_times(problem: Problem, kx: np.ndarray, kz: np.ndarray,
                 medium: Optional[Medium] = None) -> np.ndarray:
    """True one-way times [ne][nk] element -> scatterer through lens and medium."""
    lib = _load()
    med = (medium or problem.medium or Medium(speeds=[C_REF])).to_c()
    kx = np.ascontiguousarray(kx, np.float64)
    kz = np.ascontiguousarray(kz, np.float64)
    ex = np.ascontiguousarray(problem.elem_x, np.float64)
    ez = np.ascontiguousarray(problem.elem_z, np.float64)
    T = np.empty((problem.ne, kx.shape[0]), np.float64)
    kind = {0: 1, 1: 0, 2: 2}[int(problem.lens_mode)]     # curved lens / none / flat lens
    lib.sy_oneway_times(problem.ne, _dp(ex), _dp(ez), problem.arc_cx, problem.arc_cz,
                        problem.lens_radius, problem.lens_z, problem.c_lens, kind, ctypes.byref(med),
                        kx.shape[0], _dp(kx), _dp(kz), _dp(T))
    return T


def echoes(problem: Problem, T: np.ndarray, amp: np.ndarray, sigma: Optional[float] = None) -> np.ndarray:
    """Demodulated FSA data Psi[t][r][n] (complex64) for one-way times T[e][k]."""
    lib = _load()
    T = np.ascontiguousarray(T, np.float64)
    amp = np.ascontiguousarray(amp, np.float64)
    sig = pulse_sigma(problem.fc) if sigma is None else sigma
    out = np.empty((problem.ne, problem.ne, problem.ns), np.complex64)
    lib.sy_echoes(problem.ne, T.shape[1], _dp(T), _dp(amp), problem.ns, problem.fs, problem.fd,
                  problem.t0, problem.t_ttp, sig,
                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return out


def simulate(problem: Problem, n_scatterers: int, seed: int,
             medium: Optional[Medium] = None) -> np.ndarray:
    """Speckle acquisition: n_scatterers random scatterers in the (true) medium."""
    x, z, a = sector_scatterers(problem, n_scatterers, seed)
    T = oneway_times(problem, x, z, medium)
    return echoes(problem, T, a)


def oneway_times_gpu(problem: Problem, kx, kz, medium: Optional[Medium] = None):
    """The true one-way times of `oneway_times`, computed on the current CUDA device in
    float64; returns a torch tensor [ne][nk] (float64, device)."""
    import torch
    lib = _load_gpu()
    dev = torch.device("cuda")
    med = (medium or problem.medium or Medium(speeds=[C_REF])).to_c()
    ex = torch.as_tensor(np.asarray(problem.elem_x, np.float64), device=dev)
    ez = torch.as_tensor(np.asarray(problem.elem_z, np.float64), device=dev)
    kxd = torch.as_tensor(np.asarray(kx, np.float64), device=dev)
    kzd = torch.as_tensor(np.asarray(kz, np.float64), device=dev)
    T = torch.empty((problem.ne, kxd.shape[0]), dtype=torch.float64, device=dev)
    kind = {0: 1, 1: 0, 2: 2}[int(problem.lens_mode)]
    torch.cuda.synchronize()
    rc = lib.sy_gpu_oneway_times(problem.ne, ex.data_ptr(), ez.data_ptr(), problem.arc_cx, problem.arc_cz,
                                 problem.lens_radius, problem.lens_z, problem.c_lens, kind, ctypes.byref(med),
                                 kxd.shape[0], kxd.data_ptr(), kzd.data_ptr(), T.data_ptr())
    if rc != 0:
        raise RuntimeError(f"sy_gpu_oneway_times failed ({rc})")
    return T


def echoes_gpu(problem: Problem, T, amp, sigma: Optional[float] = None):
    """`echoes` on the current CUDA device: T [ne][nk] float64 torch tensor (device),
    amp [nk]; returns Psi [ne][ne][ns] complex64 (device)."""
    import torch
    lib = _load_gpu()
    dev = torch.device("cuda")
    ampd = torch.as_tensor(np.asarray(amp, np.float64), device=dev)
    T = T.contiguous()
    sig = pulse_sigma(problem.fc) if sigma is None else sigma
    out = torch.empty((problem.ne, problem.ne, problem.ns), dtype=torch.complex64, device=dev)
    torch.cuda.synchronize()
    rc = lib.sy_gpu_echoes(problem.ne, T.shape[1], T.data_ptr(), ampd.data_ptr(), problem.ns, problem.fs,
                           problem.fd, problem.t0, problem.t_ttp, sig, out.data_ptr())
    if rc != 0:
        raise RuntimeError(f"sy_gpu_echoes failed ({rc})")
    return out


def speckle_count(problem: Problem, per_cell: float = 10.0, depth=(2e-3, None)) -> int:
    """Scatterers for `per_cell` per resolution cell (lambda^2, lambda = c_ref / fc) over
    the area `sector_scatterers` draws from (curved arrays)."""
    RL = problem.lens_radius
    d1 = depth[1] if depth[1] is not None else problem.depth_range[1] + 10e-3
    half = 1.15 * problem.sector_half_angle
    area = half * ((RL + d1) ** 2 - (RL + depth[0]) ** 2)
    lam = C_REF / problem.fc
    return int(round(per_cell * area / lam ** 2))


def simulate_gpu(problem: Problem, n_scatterers: int, seed: int, medium: Optional[Medium] = None):
    """`simulate` on the current CUDA device (same scatterers, same physics); returns
    Psi as a complex64 torch tensor on the device."""
    x, z, a = sector_scatterers(problem, n_scatterers, seed)
    T = oneway_times_gpu(problem, x, z, medium)
    psi = echoes_gpu(problem, T, a)
    del T
    return psi


def segment_time(medium: Medium, ax, az, bx, bz) -> float:
    lib = _load()
    m = medium.to_c()
    return lib.sy_segment_time(ctypes.byref(m), ax, az, bx, bz)


def threads() -> int:
    return _load().sy_threads()


def config_batch_member(k: int, seed: int = 20261206, **over) -> Problem:
    """Member k of the batched workload: seeded uneven sizes (96-192 elements in
    steps of 16, 2048-4096 samples, 80-160 mm deepest patch, 64^2-128^2 grid) with a
    layered medium drawn like the full-size one."""
    rng = np.random.default_rng(seed + 7919 * k)
    ne = int(rng.choice(np.arange(96, 193, 16)))
    ns = int(rng.integers(2048, 4097) // 64 * 64)
    depth = float(rng.uniform(80e-3, 160e-3))
    ng = int(rng.choice([64, 80, 96, 112, 128]))
    fs = 14e6
    # keep the deepest round trip inside the record
    depth = min(depth, 0.9 * ns / fs * 1540.0 / 2.0 - 5e-3)
    h_fat = rng.uniform(10e-3, 25e-3)
    medium = Medium(speeds=[1600.0, 1440.0, 1560.0], base=[3e-3, 3e-3 + h_fat], amp=[0.0, 3e-3],
                    period=[0.0, 20e-3], phase=[0.0, rng.uniform(0, 2 * np.pi)])
    hyper = dict(TABLE2["invivo_c5"], lr=TABLE2["phantom_c5"]["lr"])
    kw = dict(ne=ne, radius=60e-3, pitch=0.35e-3, fc=3.5e6, d_lens=1.2e-3, c_lens=1000.0, ns=ns, fs=fs,
              nx=ng, nz=ng, n_ang=20, n_rad=20, patch_w=9, depth_min=10e-3, depth_max=depth,
              sub_width=8, hyper=hyper, medium=medium)
    kw.update(over)
    return curvilinear_problem(f"batch{k}_ne{ne}_ns{ns}", **kw)
