"""FP64 CPU oracle (ctypes wrapper around af_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg, never by the library.  The wrapper only
marshals arrays; every step of the computation is in af_oracle.c.

A `problem` argument is any object with the attributes of `synth.Problem`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_OMP_LIB_PATH = os.path.join(_HERE, "liboracle_omp.so")
_libs = {}


def _compile(out: str, extra: list, force: bool) -> str:
    src = os.path.join(_HERE, "af_oracle.c")
    hdr = os.path.join(_HERE, "af_oracle.h")
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
    if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
        subprocess.check_call(["gcc", "-O2", "-std=c99", *extra, "-shared", "-fPIC", "-o", out, src, "-lm"])
    return out


def build(force: bool = False) -> str:
    """Compile af_oracle.c twice: plain -O2, IEEE arithmetic, one thread (the parity
    judge), and the same source with -fopenmp (all host cores; for full-size checks and
    the benchmark's all-core CPU baseline).  Returns the single-threaded library."""
    _compile(_OMP_LIB_PATH, ["-fopenmp"], force)
    return _compile(_LIB_PATH, ["-Wno-unknown-pragmas"], force)


def omp_threads() -> int:
    """Threads the OpenMP build uses (OMP_NUM_THREADS, else the host's cores)."""
    lib = _load(True)
    return int(lib.or_omp_threads())


_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_ip = ctypes.POINTER(ctypes.c_int)


class Geom(ctypes.Structure):
    _fields_ = [
        ("ne", ctypes.c_int), ("ex", _dp), ("ez", _dp),
        ("lens_mode", ctypes.c_int), ("arc_cx", ctypes.c_double), ("arc_cz", ctypes.c_double),
        ("lens_radius", ctypes.c_double), ("c_lens", ctypes.c_double), ("t_ttp", ctypes.c_double),
        ("lens_z", ctypes.c_double),
        ("apod_mode", ctypes.c_int), ("fnum", ctypes.c_double),
        ("n_patch", ctypes.c_int), ("patch_npix", ctypes.c_int), ("px", _dp), ("pz", _dp),
        ("nx", ctypes.c_int), ("nz", ctypes.c_int), ("x0", ctypes.c_double), ("z0", ctypes.c_double),
        ("dx", ctypes.c_double), ("dz", ctypes.c_double), ("nseg", ctypes.c_int),
        ("ns", ctypes.c_int), ("fs", ctypes.c_double), ("fd", ctypes.c_double), ("t0", ctypes.c_double),
        ("sub_width", ctypes.c_int), ("rho_thresh", ctypes.c_double),
        ("w1", ctypes.c_double), ("kx1", ctypes.c_double), ("kz1", ctypes.c_double),
        ("w2", ctypes.c_double), ("kx2", ctypes.c_double), ("kz2", ctypes.c_double),
        ("c_unit", ctypes.c_double),
    ]


def _load(parallel: bool = False):
    if parallel not in _libs:
        build()
        lib = ctypes.CDLL(_OMP_LIB_PATH if parallel else _LIB_PATH)
        G = ctypes.POINTER(Geom)
        sig = {
            "or_element_angles": (None, [ctypes.c_int, _dp, _dp, _dp]),
            "or_apod": (ctypes.c_int, [G, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_double]),
            "or_mean_speed": (ctypes.c_double, [G, _dp]),
            "or_exit_point": (ctypes.c_int, [G, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, _dp, _dp, _dp, _dp]),
            "or_exit_from_angle": (None, [G, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]),
            "or_keys_weights": (None, [ctypes.c_double, _dp]),
            "or_bicubic": (ctypes.c_double, [G, _dp, ctypes.c_double, ctypes.c_double]),
            "or_ray_time": (ctypes.c_double, [G, _dp, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double]),
            "or_delays": (None, [G, _dp, _u8p, _dp, _dp, _u8p, _dp]),
            "or_das": (None, [G, _fp, _dp, _u8p, _dp]),
            "or_cmpe_pairs": (ctypes.c_int, [G, _ip]),
            "or_cmpe": (ctypes.c_double, [G, _dp, _u8p, _dp, _dp, _u8p, _ip]),
            "or_regularizers": (None, [G, _dp, _dp, _dp]),
            "or_regularizer_grad": (None, [G, _dp, _dp]),
            "or_cmpe_adjoint": (None, [G, _dp, _dp, _u8p, ctypes.c_int, _dp]),
            "or_das_adjoint": (None, [G, _fp, _dp, _u8p, _dp, _dp]),
            "or_ray_adjoint": (None, [G, _dp, _dp, _u8p, _dp, _dp]),
            "or_loss_grad": (ctypes.c_double, [G, _fp, _dp, _u8p, _u8p, _dp, _dp, _dp, _u8p, _ip]),
            "or_dynamic_pixels": (None, [G, ctypes.c_double, ctypes.c_double, _dp, _dp]),
            "or_gd": (None, [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double]),
            "or_adam": (None, [ctypes.c_int, _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
        }
        sig["or_omp_threads"] = (ctypes.c_int, [])
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _libs[parallel] = lib
    return _libs[parallel]


def _d(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _u8(a):
    return None if a is None else a.ctypes.data_as(_u8p)


class Oracle:
    """Holds the C geometry struct (and keeps its arrays alive).  parallel=True runs
    the OpenMP build of the same source on all host cores."""

    def __init__(self, problem, parallel: bool = False):
        self.lib = _load(parallel)
        p = problem
        self.p = p
        self._ex = np.ascontiguousarray(p.elem_x, np.float64)
        self._ez = np.ascontiguousarray(p.elem_z, np.float64)
        self._px = np.ascontiguousarray(p.pix_x, np.float64)
        self._pz = np.ascontiguousarray(p.pix_z, np.float64)
        g = Geom()
        g.ne = self._ex.shape[0]
        g.ex, g.ez = _d(self._ex), _d(self._ez)
        g.lens_mode = int(p.lens_mode)
        g.arc_cx, g.arc_cz = p.arc_cx, p.arc_cz
        g.lens_radius = p.lens_radius
        g.c_lens, g.t_ttp = p.c_lens, p.t_ttp
        g.lens_z = getattr(p, "lens_z", 0.0)
        g.apod_mode, g.fnum = int(p.apod_mode), p.fnum
        g.n_patch, g.patch_npix = int(p.n_patch), int(p.patch_npix)
        g.px, g.pz = _d(self._px), _d(self._pz)
        g.nx, g.nz = int(p.nx), int(p.nz)
        g.x0, g.z0, g.dx, g.dz = p.x0, p.z0, p.dx, p.dz
        g.nseg = int(p.nseg)
        g.ns, g.fs, g.fd, g.t0 = int(p.ns), p.fs, p.fd, p.t0
        g.sub_width = int(p.sub_width)
        g.rho_thresh = p.rho_thresh
        g.w1, g.kx1, g.kz1 = p.w1, p.kx1, p.kz1
        g.w2, g.kx2, g.kz2 = p.w2, p.kx2, p.kz2
        g.c_unit = p.c_unit
        self.g = g
        self.gp = ctypes.byref(g)
        self.ne = g.ne
        self.npix = g.n_patch * g.patch_npix
        self.nsub = g.ne // g.sub_width if g.sub_width > 0 else 0
        self.npair = self.lib.or_cmpe_pairs(self.gp, None)

    # --- geometry -------------------------------------------------------
    def element_angles(self):
        th = np.empty(self.ne)
        self.lib.or_element_angles(self.ne, _d(self._ex), _d(self._ez), _d(th))
        return th

    def apod(self, e, x, z):
        th = self.element_angles()
        return self.lib.or_apod(self.gp, _d(th), e, x, z)

    def mean_speed(self, s):
        s = np.ascontiguousarray(s, np.float64)
        return self.lib.or_mean_speed(self.gp, _d(s))

    def exit_point(self, e, x, z, sbar):
        out = [ctypes.c_double() for _ in range(4)]
        it = self.lib.or_exit_point(self.gp, e, x, z, sbar, *[ctypes.byref(o) for o in out])
        phi, tl, qx, qz = (o.value for o in out)
        return phi, tl, qx, qz, it

    def exit_from_angle(self, e, phi):
        out = [ctypes.c_double() for _ in range(3)]
        self.lib.or_exit_from_angle(self.gp, e, phi, *[ctypes.byref(o) for o in out])
        return tuple(o.value for o in out)

    def dynamic_pixels(self, c0, c_ref):
        """Pixel positions of the dynamic sweep grid at speed c0 (Sec. III-A)."""
        x = np.empty(self.npix)
        z = np.empty(self.npix)
        self.lib.or_dynamic_pixels(self.gp, c0, c_ref, _d(x), _d(z))
        return x, z

    def keys_weights(self, t):
        w = np.empty(4)
        self.lib.or_keys_weights(t, _d(w))
        return w

    def bicubic(self, s, x, z):
        s = np.ascontiguousarray(s, np.float64)
        return self.lib.or_bicubic(self.gp, _d(s), x, z)

    def ray_time(self, s, qx, qz, x, z):
        s = np.ascontiguousarray(s, np.float64)
        return self.lib.or_ray_time(self.gp, _d(s), qx, qz, x, z)

    # --- pipeline stages ---------------------------------------------------
    def delays(self, s, apod_in=None, phi_in=None):
        s = np.ascontiguousarray(s, np.float64)
        T = np.empty((self.ne, self.npix))
        apod = np.empty((self.ne, self.npix), np.uint8)
        phi = np.empty((self.ne, self.npix))
        ai = None if apod_in is None else np.ascontiguousarray(apod_in, np.uint8)
        pi = None if phi_in is None else np.ascontiguousarray(phi_in, np.float64)
        self.lib.or_delays(self.gp, _d(s), _u8(ai), _d(pi), _d(T), _u8(apod), _d(phi))
        return T, apod, phi

    def das(self, psi, T, apod):
        psi = np.ascontiguousarray(psi, np.complex64)
        T = np.ascontiguousarray(T, np.float64)
        apod = np.ascontiguousarray(apod, np.uint8)
        B = np.empty((self.nsub * self.nsub, self.npix, 2))
        self.lib.or_das(self.gp, psi.ctypes.data_as(_fp), _d(T), _u8(apod), _d(B))
        return B[..., 0] + 1j * B[..., 1]

    def pairs(self):
        out = np.empty((max(self.npair, 1), 2), np.int32)
        self.lib.or_cmpe_pairs(self.gp, out.ctypes.data_as(_ip))
        return out[: self.npair]

    def cmpe(self, B, mask_in=None):
        Bd = np.ascontiguousarray(np.stack([B.real, B.imag], -1), np.float64)
        nzp = max(self.g.n_patch * self.npair, 1)
        z = np.empty((nzp, 2))
        rho = np.empty(nzp)
        mask = np.empty(nzp, np.uint8)
        M = ctypes.c_int()
        mi = None if mask_in is None else np.ascontiguousarray(mask_in, np.uint8).ravel()
        L = self.lib.or_cmpe(self.gp, _d(Bd), _u8(mi), _d(z), _d(rho), _u8(mask), ctypes.byref(M))
        n = self.g.n_patch * self.npair
        shape = (self.g.n_patch, self.npair)
        return (L, (z[:n, 0] + 1j * z[:n, 1]).reshape(shape), rho[:n].reshape(shape),
                mask[:n].reshape(shape), M.value)

    def regularizers(self, s):
        s = np.ascontiguousarray(s, np.float64)
        a, b = ctypes.c_double(), ctypes.c_double()
        self.lib.or_regularizers(self.gp, _d(s), ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def regularizer_grad(self, s):
        s = np.ascontiguousarray(s, np.float64)
        g = np.zeros(s.shape)
        self.lib.or_regularizer_grad(self.gp, _d(s), _d(g))
        return g

    def cmpe_adjoint(self, B, z, mask, M):
        Bd = np.ascontiguousarray(np.stack([B.real, B.imag], -1), np.float64)
        zd = np.ascontiguousarray(np.stack([z.real, z.imag], -1), np.float64)
        G = np.empty(Bd.shape)
        self.lib.or_cmpe_adjoint(self.gp, _d(Bd), _d(zd), _u8(np.ascontiguousarray(mask, np.uint8)),
                                 int(M), _d(G))
        return G[..., 0] + 1j * G[..., 1]

    def das_adjoint(self, psi, T, apod, G):
        psi = np.ascontiguousarray(psi, np.complex64)
        Gd = np.ascontiguousarray(np.stack([G.real, G.imag], -1), np.float64)
        gT = np.empty((self.ne, self.npix))
        self.lib.or_das_adjoint(self.gp, psi.ctypes.data_as(_fp), _d(np.ascontiguousarray(T)),
                                _u8(np.ascontiguousarray(apod, np.uint8)), _d(Gd), _d(gT))
        return gT

    def ray_adjoint(self, s, phi, apod, gT):
        s = np.ascontiguousarray(s, np.float64)
        grad = np.zeros(s.shape)
        self.lib.or_ray_adjoint(self.gp, _d(s), _d(np.ascontiguousarray(phi, np.float64)),
                                _u8(None if apod is None else np.ascontiguousarray(apod, np.uint8)),
                                _d(np.ascontiguousarray(gT, np.float64)), _d(grad))
        return grad

    def loss_grad(self, psi, s, apod_in=None, mask_in=None, phi_in=None, grad=True):
        """Eq. 12 loss parts {L, L_CMPE, R_TV, R_SV}, dL/ds (or None), CMPE mask, M."""
        psi = np.ascontiguousarray(psi, np.complex64)
        s = np.ascontiguousarray(s, np.float64)
        parts = np.empty(4)
        g = np.zeros(s.shape) if grad else None
        nzp = max(self.g.n_patch * self.npair, 1)
        mask = np.empty(nzp, np.uint8)
        M = ctypes.c_int()
        ai = None if apod_in is None else np.ascontiguousarray(apod_in, np.uint8)
        mi = None if mask_in is None else np.ascontiguousarray(mask_in, np.uint8).ravel()
        pi = None if phi_in is None else np.ascontiguousarray(phi_in, np.float64)
        self.lib.or_loss_grad(self.gp, psi.ctypes.data_as(_fp), _d(s), _u8(ai), _u8(mi), _d(pi),
                              _d(g), _d(parts), _u8(mask), ctypes.byref(M))
        n = self.g.n_patch * self.npair
        return parts, g, mask[:n].reshape(self.g.n_patch, self.npair), M.value

    def gd(self, s, grad, lr, c_unit=1000.0):
        """Eq. 9 as printed on c in units of c_unit m/s; returns the new slowness."""
        s = np.array(s, np.float64)
        self.lib.or_gd(s.size, _d(s), _d(np.ascontiguousarray(grad, np.float64)), lr, c_unit)
        return s

    def adam(self, s, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, c_unit=1000.0):
        s = np.array(s, np.float64)
        m = np.array(m, np.float64)
        v = np.array(v, np.float64)
        self.lib.or_adam(s.size, _d(s), _d(np.ascontiguousarray(grad, np.float64)), _d(m), _d(v),
                         step, lr, beta1, beta2, eps, c_unit)
        return s, m, v
