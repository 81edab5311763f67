"""B300 (sm_103a) lens-aware differentiable-beamforming autofocus.

Thin ctypes binding of the C ABI in include/af.h (libaf.so, built in-tree by
`paper_2608_06853_b300.build.build()`).  The binding only marshals arguments:
every step of the hot path runs in the library's CUDA kernels.  PyTorch
provides device memory and streams.  There is no CPU fallback: if libaf.so is
missing or no CUDA device is present, the calls raise.

Main entry points (same names as the C ABI):
    Plan(problem, iq_dtype=AF_IQ_C64, stream=None)
    plan.af_forward(iq, s, loss, iq_scale=None)   -> loss[4] = {L, L_CMPE, R_TV, R_SV}
    plan.af_adjoint(grad)                          -> dL/ds
    plan.af_step(grad, s, m, v, step)              -> Adam update (Eq. 9)
    plan.af_iterate(iq, s, grad, m, v, step, loss, iq_scale=None)
    AutofocusLoss.apply(s, plan, iq, iq_scale)     -> torch.autograd.Function

A `problem` is any object with the attributes of the library's problem
description (elem_x, elem_z, arc_cx, ..., see `ProblemFields`).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaf.so")

AF_OK, AF_ERR_ARG, AF_ERR_SHAPE, AF_ERR_DTYPE, AF_ERR_CUDA = 0, 1, 2, 3, 4
AF_ERR_NUMERIC, AF_ERR_TIMEOUT, AF_ERR_UNSUPPORTED, AF_ERR_STATE = 5, 6, 7, 8
AF_IQ_C64, AF_IQ_BF16, AF_IQ_F16 = 0, 1, 2
AF_LENS_BENT_RAY, AF_LENS_NONE, AF_LENS_PLANAR = 0, 1, 2
AF_APOD_FNUMBER, AF_APOD_PRINTED = 0, 1
AF_OPT_ADAM, AF_OPT_GD = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)


class AfConfig(ctypes.Structure):
    """Mirror of af_config (include/af.h)."""
    _fields_ = [
        ("n_elem", ctypes.c_int), ("elem_x", _dp), ("elem_z", _dp),
        ("lens_mode", ctypes.c_int), ("arc_cx", ctypes.c_double), ("arc_cz", ctypes.c_double),
        ("lens_radius", ctypes.c_double), ("c_lens", ctypes.c_double), ("t_ttp", ctypes.c_double),
        ("lens_z", ctypes.c_double),
        ("apod_mode", ctypes.c_int), ("fnum", ctypes.c_double),
        ("n_patch", ctypes.c_int), ("patch_npix", ctypes.c_int), ("pix_x", _dp), ("pix_z", _dp),
        ("nx", ctypes.c_int), ("nz", ctypes.c_int), ("x0", ctypes.c_double), ("z0", ctypes.c_double),
        ("dx", ctypes.c_double), ("dz", ctypes.c_double), ("nseg", ctypes.c_int),
        ("n_samp", ctypes.c_int), ("fs", ctypes.c_double), ("fd", ctypes.c_double),
        ("t0", ctypes.c_double), ("iq_dtype", ctypes.c_int), ("sub_width", ctypes.c_int),
        ("rho_thresh", ctypes.c_double),
        ("w1", ctypes.c_double), ("kx1", ctypes.c_double), ("kz1", ctypes.c_double),
        ("w2", ctypes.c_double), ("kx2", ctypes.c_double), ("kz2", ctypes.c_double),
        ("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
        ("eps", ctypes.c_double), ("c_unit", ctypes.c_double), ("optimizer", ctypes.c_int),
    ]


ProblemFields = ("elem_x", "elem_z", "lens_mode", "arc_cx", "arc_cz", "lens_radius", "c_lens",
                 "t_ttp", "apod_mode", "fnum", "n_patch", "patch_npix", "pix_x", "pix_z", "nx",
                 "nz", "x0", "z0", "dx", "dz", "nseg", "ns", "fs", "fd", "t0", "sub_width",
                 "rho_thresh", "w1", "kx1", "kz1", "w2", "kx2", "kz2", "lr", "beta1", "beta2",
                 "eps", "c_unit", "optimizer")

_lib = None

_VP = ctypes.c_void_p
_PA = ctypes.POINTER(ctypes.c_void_p)   # host array of device pointers


class AfMetrics(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("cf_mean", "loc", "cmcc", "contrast_db", "cnr", "gcnr",
                                                "mean_in", "mean_out")] + \
               [("n_in", ctypes.c_longlong), ("n_out", ctypes.c_longlong)]


# name -> (restype, argtypes) of every exported entry point of include/af.h
_SIGNATURES = {
    "af_check_config": (ctypes.c_int, [ctypes.POINTER(AfConfig)]),
    "af_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(AfConfig), ctypes.POINTER(ctypes.c_size_t)]),
    "af_plan": (ctypes.c_int, [ctypes.POINTER(AfConfig), _VP, ctypes.POINTER(_VP)]),
    "af_forward": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "af_adjoint": (ctypes.c_int, [_VP, _VP]),
    "af_step": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_int]),
    "af_iterate": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_int, _VP]),
    "af_destroy": (ctypes.c_int, [_VP]),
    "af_job_reserve": (ctypes.c_int, [_VP]),
    "af_job_submit": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, _VP, _VP]),
    "af_job_wait": (ctypes.c_int, [_VP]),
    "af_batch_plan": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.POINTER(AfConfig)), _VP,
                                      ctypes.POINTER(_VP)]),
    "af_batch_plan_of": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(_VP)]),
    "af_batch_iterate": (ctypes.c_int, [_VP, _PA, _PA, _PA, _PA, _PA, _PA, ctypes.c_int, _PA]),
    "af_batch_capture": (ctypes.c_int, [_VP, _PA, _PA, _PA, _PA, _PA, _PA, _PA, ctypes.c_int, ctypes.c_int]),
    "af_batch_launch": (ctypes.c_int, [_VP]),
    "af_batch_destroy": (ctypes.c_int, [_VP]),
    "af_sync_status": (ctypes.c_int, [_VP]),
    "af_sweep": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_double,
                                 ctypes.c_int, _VP, _VP]),
    "af_set_pixels": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "af_get_delays": (ctypes.c_int, [_VP, _VP, _VP]),
    "af_get_exit_angles": (ctypes.c_int, [_VP, _VP]),
    "af_get_images": (ctypes.c_int, [_VP, _VP]),
    "af_get_cmpe": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(ctypes.c_int)]),
    "af_get_image_grad": (ctypes.c_int, [_VP, _VP]),
    "af_cmpe_totals": (ctypes.c_int, [_VP, _VP]),
    "af_set_cmpe_totals": (ctypes.c_int, [_VP, _VP, _VP]),
    "af_get_bmode": (ctypes.c_int, [_VP, _VP, _VP]),
    "af_image_metrics": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.POINTER(AfMetrics)]),
    "af_speed_mae": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(ctypes.c_double)]),
    "af_get_delay_grad": (ctypes.c_int, [_VP, _VP]),
    "af_get_counters": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_longlong)]),
    "af_cmpe_loss_noalloc": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             _VP, _VP, _VP]),
    "af_surrogate_train": (ctypes.c_int, [_VP, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                           ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_double)]),
    "af_surrogate_enable": (ctypes.c_int, [_VP, ctypes.c_int]),
    "af_surrogate_eval": (ctypes.c_int, [_VP, ctypes.c_float, _VP, _VP]),
    "af_surrogate_params": (ctypes.c_int, [_VP, _VP, ctypes.c_int]),
    "af_surrogate_grad": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, ctypes.POINTER(ctypes.c_float)]),
    "af_gemm_bf16": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, _VP, _VP]),
    "af_set_wait_limit": (ctypes.c_int, [ctypes.c_int]),
    "af_set_ray_flush_budget": (ctypes.c_int, [_VP, ctypes.c_double]),
    "af_fp32_lane_rate": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_double)]),
    "af_set_timing": (ctypes.c_int, [_VP, ctypes.c_int]),
    "af_get_stage_times": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int)]),
    "af_last_error": (ctypes.c_char_p, []),
    "af_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}


class AfError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        name = lib.af_status_string(status).decode()
        msg = lib.af_last_error().decode()
        super().__init__(f"{where}: {name}: {msg}")
        self.status = status


def load():
    """Load libaf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2608_06853_b300.build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(status: int, where: str):
    if status != AF_OK:
        raise AfError(status, where)


def make_config(problem, iq_dtype: int = AF_IQ_C64):
    """af_config for a problem description; returns (config, arrays kept alive)."""
    keep = []

    def arr(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(_dp)

    c = AfConfig()
    c.n_elem = int(len(problem.elem_x))
    c.elem_x, c.elem_z = arr(problem.elem_x), arr(problem.elem_z)
    c.lens_mode = int(problem.lens_mode)
    c.arc_cx, c.arc_cz = float(problem.arc_cx), float(problem.arc_cz)
    c.lens_radius, c.c_lens, c.t_ttp = float(problem.lens_radius), float(problem.c_lens), float(problem.t_ttp)
    c.lens_z = float(getattr(problem, "lens_z", 0.0))
    c.apod_mode, c.fnum = int(problem.apod_mode), float(problem.fnum)
    c.n_patch, c.patch_npix = int(problem.n_patch), int(problem.patch_npix)
    c.pix_x, c.pix_z = arr(problem.pix_x), arr(problem.pix_z)
    c.nx, c.nz = int(problem.nx), int(problem.nz)
    c.x0, c.z0, c.dx, c.dz = float(problem.x0), float(problem.z0), float(problem.dx), float(problem.dz)
    c.nseg = int(problem.nseg)
    c.n_samp, c.fs, c.fd, c.t0 = int(problem.ns), float(problem.fs), float(problem.fd), float(problem.t0)
    c.iq_dtype = int(iq_dtype)
    c.sub_width = int(problem.sub_width)
    c.rho_thresh = float(problem.rho_thresh)
    c.w1, c.kx1, c.kz1 = float(problem.w1), float(problem.kx1), float(problem.kz1)
    c.w2, c.kx2, c.kz2 = float(problem.w2), float(problem.kx2), float(problem.kz2)
    c.lr, c.beta1, c.beta2 = float(problem.lr), float(problem.beta1), float(problem.beta2)
    c.eps, c.c_unit = float(problem.eps), float(problem.c_unit)
    c.optimizer = int(getattr(problem, "optimizer", AF_OPT_ADAM))
    return c, keep


def check_config(problem, iq_dtype: int = AF_IQ_C64) -> int:
    """Host-only validation (no CUDA call); returns the af_status code."""
    c, keep = make_config(problem, iq_dtype)
    return load().af_check_config(ctypes.byref(c))


def _ptr(t):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("device tensors only (torch.Tensor on cuda)")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(t, dtype, nbytes: int, what: str):
    """Address of a host tensor of exactly nbytes bytes (contiguous, given dtype)."""
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{what}: host tensors only (torch.Tensor on the CPU)")
    if not t.is_contiguous():
        raise ValueError(f"{what}: tensor must be contiguous")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise ValueError(f"{what}: dtype {t.dtype}")
    if t.numel() * t.element_size() != nbytes:
        raise ValueError(f"{what}: {t.numel() * t.element_size()} bytes, expected {nbytes}")
    return ctypes.c_void_p(t.data_ptr())


def iq_view(iq):
    """The raw storage of channel data: complex64 tensors are passed as interleaved float32."""
    import torch
    if iq.dtype == torch.complex64:
        return torch.view_as_real(iq)
    return iq


AF_NOALLOC_MAX_PATCHES = 16384


def af_cmpe_loss_noalloc(B, nsub: int, n_patch: int, patch_npix: int, rho_thresh: float, loss,
                         n_active=None, stream=None):
    """L_CMPE of images B ([nsub*nsub][npix] complex64 or [..][npix][2] float32, device) into
    loss[0], without any device allocation by the library (see include/af.h).

    The library reads nsub*nsub*n_patch*patch_npix complex values from B and writes
    loss[0] (and n_active[0]) on the device that is current when it is called, so the
    arguments are checked here first: shapes, dtypes and contiguity (ValueError), then
    that every tensor is on the current CUDA device."""
    import torch
    nsub, n_patch, patch_npix = int(nsub), int(n_patch), int(patch_npix)
    if B.dtype == torch.complex64:
        n_values = B.numel()
    elif B.dtype == torch.float32 and B.dim() >= 1 and B.shape[-1] == 2:
        n_values = B.numel() // 2
    else:
        raise ValueError("B must be complex64, or float32 with a last dimension of 2")
    if n_values != nsub * nsub * n_patch * patch_npix:
        raise ValueError(f"B holds {n_values} complex values, expected nsub^2 * n_patch * patch_npix = "
                         f"{nsub * nsub * n_patch * patch_npix}")
    if not B.is_contiguous():
        raise ValueError("B must be contiguous")
    if loss.dtype != torch.float32 or loss.numel() < 1 or not loss.is_contiguous():
        raise ValueError("loss must be a contiguous float32 tensor with at least one element")
    if n_active is not None and (n_active.dtype != torch.int32 or n_active.numel() < 1):
        raise ValueError("n_active must be an int32 tensor with at least one element, or None")
    tensors = [B, loss] + ([n_active] if n_active is not None else [])
    if not all(t.is_cuda for t in tensors):
        raise ValueError("B, loss and n_active must be CUDA tensors")
    cur = torch.cuda.current_device()
    if any(t.device.index != cur for t in tensors):
        raise ValueError(f"B, loss and n_active must be on the current CUDA device (cuda:{cur})")
    Bv = torch.view_as_real(B) if B.dtype == torch.complex64 else B
    h = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    _check(load().af_cmpe_loss_noalloc(_ptr(Bv), nsub, n_patch, patch_npix,
                                       float(rho_thresh), _ptr(loss), _ptr(n_active), h),
           "af_cmpe_loss_noalloc")
    return loss


def fp32_lane_rate(stream=None) -> float:
    """Measured FP32 lane-operations per second of the current device (af_fp32_lane_rate)."""
    import torch
    sink = torch.zeros(1, device=torch.device("cuda", torch.cuda.current_device()))
    h = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    rate = ctypes.c_double()
    _check(load().af_fp32_lane_rate(_ptr(sink), h, ctypes.byref(rate)), "af_fp32_lane_rate")
    return rate.value


def af_gemm_bf16(A, B, D, a_mn_major=False, b_mn_major=False, err=None, stream=None):
    """D = A B^T on the tensor cores (see include/af.h).  A: bf16 [M][K] or [K][M];
    B: bf16 [N][K] or [K][N]; D: float32 [M][N]."""
    import torch
    M, N = D.shape
    K = A.shape[0] if a_mn_major else A.shape[1]
    if err is None:
        err = torch.zeros(1, dtype=torch.int32, device=D.device)
    h = ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    _check(load().af_gemm_bf16(_ptr(A), _ptr(B), _ptr(D), M, N, K, int(bool(a_mn_major)),
                               int(bool(b_mn_major)), _ptr(err), h), "af_gemm_bf16")
    return err


class Plan:
    """An af_plan_t: device geometry and workspaces for one problem on one stream."""

    def __init__(self, problem, iq_dtype: int = AF_IQ_C64, stream=None):
        import torch
        self._describe(problem, iq_dtype, stream if stream is not None else torch.cuda.current_stream())
        cfg, keep = make_config(problem, iq_dtype)
        h = ctypes.c_void_p()
        _check(self.lib.af_plan(ctypes.byref(cfg), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
               "af_plan")
        self.handle = h
        self._owner = None

    def _describe(self, problem, iq_dtype, stream):
        self.lib = load()
        self.problem = problem
        self.iq_dtype = iq_dtype
        self.ne = int(len(problem.elem_x))
        self.npix = int(problem.n_patch) * int(problem.patch_npix)
        self.nsub = self.ne // int(problem.sub_width)
        self.npair = (self.nsub - 1) * (self.nsub - 2) if self.nsub >= 3 else 0
        self.nx, self.nz = int(problem.nx), int(problem.nz)
        self.stream = stream

    @classmethod
    def batch_member(cls, batch, k: int, problem, iq_dtype: int, stream):
        """Member k of an af_batch_t (af_batch_plan_of): the batch owns the plan,
        this object keeps the batch alive and never destroys the plan."""
        self = cls.__new__(cls)
        self._describe(problem, iq_dtype, stream)
        h = ctypes.c_void_p()
        _check(self.lib.af_batch_plan_of(batch.handle, int(k), ctypes.byref(h)), "af_batch_plan_of")
        self.handle = h
        self._owner = batch
        return self

    def close(self):
        if getattr(self, "handle", None):
            if getattr(self, "_owner", None) is None:
                self.lib.af_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- the four calls of one iteration ----
    def af_forward(self, iq, s, loss, iq_scale=None):
        _check(self.lib.af_forward(self.handle, _ptr(iq_view(iq)), _ptr(iq_scale), _ptr(s), _ptr(loss)),
               "af_forward")
        return loss

    def af_adjoint(self, grad):
        _check(self.lib.af_adjoint(self.handle, _ptr(grad)), "af_adjoint")
        return grad

    def af_step(self, grad, s, m, v, step: int):
        _check(self.lib.af_step(self.handle, _ptr(grad), _ptr(s), _ptr(m), _ptr(v), int(step)), "af_step")

    def af_iterate(self, iq, s, grad, m, v, step: int, loss, iq_scale=None):
        _check(self.lib.af_iterate(self.handle, _ptr(iq_view(iq)), _ptr(iq_scale), _ptr(s), _ptr(grad),
                                   _ptr(m), _ptr(v), int(step), _ptr(loss)), "af_iterate")
        return loss

    def af_sync_status(self) -> int:
        return self.lib.af_sync_status(self.handle)

    # ---- autofocus jobs from host memory ----
    def job_reserve(self):
        """Device buffers, copy stream and events of af_job_submit (af_job_reserve)."""
        _check(self.lib.af_job_reserve(self.handle), "af_job_reserve")

    def job_submit(self, h_iq, h_s0, n_iter: int, h_s_out=None, h_loss=None, h_iq_scale=None):
        """Enqueue one job: upload of h_iq and h_s0 (host tensors, pinned for overlap),
        n_iter iterations, read back into h_s_out ([nz][nx] float32) and h_loss ([4]
        float32).  The host tensors are kept alive until job_wait."""
        import torch
        ns = int(self.problem.ns)
        ebytes = 8 if self.iq_dtype == AF_IQ_C64 else 4
        iq_dt = (torch.complex64, torch.float32) if self.iq_dtype == AF_IQ_C64 else (torch.bfloat16, torch.float16)
        ng = self.nx * self.nz
        args = [_hptr(h_iq, iq_dt, self.ne * self.ne * ns * ebytes, "h_iq"),
                None if h_iq_scale is None else _hptr(h_iq_scale, torch.float32, 4 * self.ne, "h_iq_scale"),
                _hptr(h_s0, torch.float32, 4 * ng, "h_s0"), int(n_iter),
                None if h_s_out is None else _hptr(h_s_out, torch.float32, 4 * ng, "h_s_out"),
                None if h_loss is None else _hptr(h_loss, torch.float32, 16, "h_loss")]
        self._job_refs = getattr(self, "_job_refs", []) + [h_iq, h_iq_scale, h_s0, h_s_out, h_loss]
        _check(self.lib.af_job_submit(self.handle, *args), "af_job_submit")

    def job_wait(self):
        """Wait for every submitted job (af_job_wait); raises on an error status."""
        st = self.lib.af_job_wait(self.handle)
        self._job_refs = []
        _check(st, "af_job_wait")

    def af_sweep(self, iq, speeds, c_ref, dynamic=True, iq_scale=None):
        """L_CMPE and active terms of uniform maps at each speed (af_sweep); returns
        (cmpe [n] float32, active [n] int32) device tensors, queued on the plan's stream."""
        import torch
        sp = np.ascontiguousarray(speeds, np.float64)
        cm = torch.empty(len(sp), dtype=torch.float32, device=self._dev())
        act = torch.empty(len(sp), dtype=torch.int32, device=self._dev())
        _check(self.lib.af_sweep(self.handle, _ptr(iq_view(iq)), _ptr(iq_scale),
                                 sp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(sp), float(c_ref),
                                 1 if dynamic else 0, _ptr(cm), _ptr(act)), "af_sweep")
        return cm, act

    def af_set_pixels(self, pix_x, pix_z):
        x = np.ascontiguousarray(pix_x, np.float64)
        z = np.ascontiguousarray(pix_z, np.float64)
        _check(self.lib.af_set_pixels(self.handle, x.ctypes.data_as(_dp), z.ctypes.data_as(_dp)), "af_set_pixels")

    # ---- introspection ----
    def _dev(self):
        import torch
        return torch.device("cuda", torch.cuda.current_device())

    def delays(self):
        """(T [ne][npix] float64 seconds, apod [ne][npix] uint8) of the last forward."""
        import torch
        T = torch.empty((self.ne, self.npix), dtype=torch.float64, device=self._dev())
        a = torch.empty((self.ne, self.npix), dtype=torch.uint8, device=self._dev())
        _check(self.lib.af_get_delays(self.handle, _ptr(T), _ptr(a)), "af_get_delays")
        return T, a

    def exit_angles(self):
        import torch
        phi = torch.empty((self.ne, self.npix), dtype=torch.float32, device=self._dev())
        _check(self.lib.af_get_exit_angles(self.handle, _ptr(phi)), "af_get_exit_angles")
        return phi

    def images(self):
        """B [nsub*nsub][npix] complex64."""
        import torch
        B = torch.empty((self.nsub * self.nsub, self.npix, 2), dtype=torch.float32, device=self._dev())
        _check(self.lib.af_get_images(self.handle, _ptr(B)), "af_get_images")
        return torch.view_as_complex(B)

    def cmpe(self):
        """(z [n_patch][npair] complex64, mask [n_patch][npair] uint8, n_active)."""
        import torch
        P = int(self.problem.n_patch)
        z = torch.empty((P, max(self.npair, 1), 2), dtype=torch.float32, device=self._dev())
        m = torch.empty((P, max(self.npair, 1)), dtype=torch.uint8, device=self._dev())
        n = ctypes.c_int()
        _check(self.lib.af_get_cmpe(self.handle, _ptr(z), _ptr(m), ctypes.byref(n)), "af_get_cmpe")
        return torch.view_as_complex(z)[:, : self.npair], m[:, : self.npair], n.value

    def bmode(self):
        """(|sum_ij B_ij| [npix], integrated CMPE image [npix]) of the last forward."""
        import torch
        b = torch.empty(self.npix, dtype=torch.float32, device=self._dev())
        c = torch.empty_like(b)
        _check(self.lib.af_get_bmode(self.handle, _ptr(b), _ptr(c)), "af_get_bmode")
        return b, c

    def image_metrics(self, roi, nbins: int = 256):
        """Metrics of the last forward (af_image_metrics): roi [npix] uint8 tensor on the
        device, 1 target, 2 background.  Returns a dict."""
        m = AfMetrics()
        _check(self.lib.af_image_metrics(self.handle, _ptr(roi), int(nbins), ctypes.byref(m)),
               "af_image_metrics")
        return {name: getattr(m, name) for name, _ in AfMetrics._fields_}

    def speed_mae(self, s, c_true):
        """Mean |1 / bicubic(s) - c_true| over the plan's pixels (af_speed_mae)."""
        out = ctypes.c_double()
        _check(self.lib.af_speed_mae(self.handle, _ptr(s), _ptr(c_true), ctypes.byref(out)), "af_speed_mae")
        return out.value

    def cmpe_totals(self, out=None):
        """{sum of |arg z| over active CMPE terms, their number} of the last forward, as a
        float64 device tensor [2] (af_cmpe_totals; asynchronous on the plan's stream)."""
        import torch
        out = torch.empty(2, dtype=torch.float64, device=self._dev()) if out is None else out
        _check(self.lib.af_cmpe_totals(self.handle, _ptr(out)), "af_cmpe_totals")
        return out

    def set_cmpe_totals(self, totals, loss=None):
        """Use CMPE totals summed over several plans (af_set_cmpe_totals)."""
        _check(self.lib.af_set_cmpe_totals(self.handle, _ptr(totals), _ptr(loss)), "af_set_cmpe_totals")

    def image_grad(self):
        """dL/dB [nsub*nsub][npix] complex64 of the last adjoint."""
        import torch
        G = torch.empty((self.nsub * self.nsub, self.npix, 2), dtype=torch.float32, device=self._dev())
        _check(self.lib.af_get_image_grad(self.handle, _ptr(G)), "af_get_image_grad")
        return torch.view_as_complex(G)

    def delay_grad(self):
        import torch
        g = torch.empty((self.ne, self.npix), dtype=torch.float32, device=self._dev())
        _check(self.lib.af_get_delay_grad(self.handle, _ptr(g)), "af_get_delay_grad")
        return g

    STAGES = ("grid_stats", "delays", "das_forward", "cmpe_forward", "cmpe_adjoint",
              "das_adjoint", "ray_adjoint", "adam", "surrogate")

    def set_timing(self, enable: bool):
        _check(self.lib.af_set_timing(self.handle, 1 if enable else 0), "af_set_timing")

    def set_ray_flush_budget(self, rays: float):
        """Flush window of the ray adjoint's fixed-point grids, in rays of the largest
        |dL/dT| (capped at the window the fixed-point scale is sized for)."""
        _check(self.lib.af_set_ray_flush_budget(self.handle, float(rays)), "af_set_ray_flush_budget")

    def stage_times(self):
        """{stage: (total ms, launches)} recorded since set_timing(True)."""
        ms = (ctypes.c_float * 9)()
        n = (ctypes.c_int * 9)()
        _check(self.lib.af_get_stage_times(self.handle, ms, n), "af_get_stage_times")
        return {name: (ms[k], n[k]) for k, name in enumerate(self.STAGES)}

    # ---- learned lens surrogate ----
    def surrogate_train(self, n_samples=10_000_000, epochs=4, tiles_per_step=32, lr=2e-3, seed=1):
        """Train the lens-surrogate MLP on the tensor cores (see include/af.h)."""
        rep = (ctypes.c_double * 8)()
        _check(self.lib.af_surrogate_train(self.handle, int(n_samples), int(epochs), int(tiles_per_step),
                                           float(lr), int(seed), rep), "af_surrogate_train")
        keys = ("train_loss", "rms_angle_err", "max_delay_err", "max_lens_time_err", "fallback_fraction",
                "samples", "tolerance", "steps")
        return dict(zip(keys, list(rep)))

    def surrogate_enable(self, enable=True):
        _check(self.lib.af_surrogate_enable(self.handle, 1 if enable else 0), "af_surrogate_enable")

    def surrogate_eval(self, c):
        import torch
        phi = torch.empty((self.ne, self.npix), dtype=torch.float32, device=self._dev())
        tl = torch.empty_like(phi)
        _check(self.lib.af_surrogate_eval(self.handle, float(c), _ptr(phi), _ptr(tl)), "af_surrogate_eval")
        return phi, tl

    NPARAM = 33922

    def surrogate_params(self):
        import torch
        p = torch.empty(self.NPARAM, dtype=torch.float32, device=self._dev())
        _check(self.lib.af_surrogate_params(self.handle, _ptr(p), 0), "af_surrogate_params")
        return p

    def set_surrogate_params(self, p):
        _check(self.lib.af_surrogate_params(self.handle, _ptr(p.contiguous()), 1), "af_surrogate_params")

    def surrogate_grad(self, X, Y):
        """(gradient [NPARAM], loss) of the training loss on the batch X [n][4], Y [n][2]."""
        import torch
        g = torch.empty(self.NPARAM, dtype=torch.float32, device=self._dev())
        loss = ctypes.c_float()
        _check(self.lib.af_surrogate_grad(self.handle, _ptr(X.contiguous()), _ptr(Y.contiguous()), int(X.shape[0]),
                                          _ptr(g), ctypes.byref(loss)), "af_surrogate_grad")
        return g, loss.value

    def counters(self):
        """{apodized pairs, float64 exit solves, active CMPE terms, CMPE pairs per patch}."""
        c = (ctypes.c_longlong * 4)()
        _check(self.lib.af_get_counters(self.handle, c), "af_get_counters")
        return dict(n_apod=c[0], fp64_solves=c[1], n_active=c[2], npair=c[3])


try:
    import torch as _torch

    class AutofocusLoss(_torch.autograd.Function):
        """L(s) of Eq. 12 with the hand-written adjoint as its backward.

        forward: af_forward; backward: af_adjoint (delays are recomputed from the
        one-way tables, not stored per transmit/receive pair)."""

        @staticmethod
        def forward(ctx, s, plan, iq, iq_scale=None):
            s = s.contiguous()
            loss = _torch.empty(4, dtype=_torch.float32, device=s.device)
            plan.af_forward(iq, s, loss, iq_scale)
            ctx.plan = plan
            return loss[0].clone()

        @staticmethod
        def backward(ctx, gout):
            plan = ctx.plan
            grad = _torch.empty((plan.nz, plan.nx), dtype=_torch.float32, device=gout.device)
            plan.af_adjoint(grad)
            return grad * gout, None, None, None
except ImportError:  # pragma: no cover - torch is part of the image
    pass
