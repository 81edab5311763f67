"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/af.h, and its host-side validation returns the documented
status codes.  No compute call is made here."""
import ctypes
import dataclasses
import os
import re

import numpy as np
import pytest

import paper_2608_06853_b300 as af
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(af_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    lib = af.load()
    names = declared_symbols()
    assert {"af_plan", "af_forward", "af_adjoint", "af_step"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(af._SIGNATURES) == names


def test_status_strings():
    lib = af.load()
    assert lib.af_status_string(af.AF_OK) == b"AF_OK"
    assert lib.af_status_string(af.AF_ERR_STATE) == b"AF_ERR_STATE"


@pytest.mark.parametrize("maker", [synth.config_tiny, synth.config_full])
def test_valid_configs_pass_host_validation(maker):
    p = maker()
    assert af.check_config(p) == af.AF_OK
    for dt in (af.AF_IQ_BF16, af.AF_IQ_F16):
        assert af.check_config(p, dt) == af.AF_OK
    c, keep = af.make_config(p)
    nbytes = ctypes.c_size_t()
    assert af.load().af_workspace_bytes(ctypes.byref(c), ctypes.byref(nbytes)) == af.AF_OK
    assert nbytes.value > 0


def test_invalid_configs_are_rejected_with_codes():
    p = synth.config_tiny()
    R = dataclasses.replace
    lib = af.load()
    assert af.check_config(R(p, sub_width=3)) == af.AF_ERR_SHAPE
    assert af.check_config(R(p, sub_width=32)) == af.AF_ERR_UNSUPPORTED   # width 32 not built
    assert af.check_config(p, iq_dtype=7) == af.AF_ERR_DTYPE
    assert af.check_config(R(p, fnum=0.0)) == af.AF_ERR_ARG
    assert af.check_config(R(p, nseg=0)) == af.AF_ERR_ARG
    assert af.check_config(R(p, nx=1)) == af.AF_ERR_SHAPE
    assert af.check_config(R(p, nx=400, nz=400)) == af.AF_ERR_UNSUPPORTED
    assert af.check_config(R(p, ns=1)) == af.AF_ERR_SHAPE
    assert af.check_config(R(p, fs=-1.0)) == af.AF_ERR_ARG
    assert af.check_config(R(p, lr=float("nan"))) == af.AF_ERR_ARG
    bad = p.pix_x.copy()
    bad[3] = 1.0                                  # far outside the grid
    assert af.check_config(R(p, pix_x=bad)) == af.AF_ERR_ARG
    assert b"outside" in lib.af_last_error()
    inside_lens = p.pix_z.copy()
    inside_lens[0] = p.arc_cz + 0.5 * p.lens_radius
    inside_lens_x = p.pix_x.copy()
    inside_lens_x[0] = p.arc_cx
    assert af.check_config(R(p, pix_x=inside_lens_x, pix_z=inside_lens)) == af.AF_ERR_ARG
    assert af.check_config(R(p, c_lens=0.0)) == af.AF_ERR_ARG
    assert af.check_config(R(p, beta1=1.0)) == af.AF_ERR_ARG
    assert lib.af_check_config(None) == af.AF_ERR_ARG


def test_degenerate_but_valid_shapes():
    p = synth.config_tiny()
    R = dataclasses.replace
    # no patches: loss is the regulariser only
    assert af.check_config(R(p, n_patch=0, pix_x=np.zeros(0), pix_z=np.zeros(0))) == af.AF_OK
    # fewer than three subapertures: no common-midpoint pairs
    assert af.check_config(R(p, sub_width=16)) == af.AF_OK
    # straight-ray model (no lens)
    assert af.check_config(R(p, lens_mode=af.AF_LENS_NONE)) == af.AF_OK


def test_flat_lens_configs():
    """Linear array with a flat lens: valid as built; an element not above the lens
    line, a pixel not below it, or a lens line leaving the grid box is rejected."""
    p = synth.config_linear_tiny()
    R = dataclasses.replace
    lib = af.load()
    assert p.lens_mode == af.AF_LENS_PLANAR
    assert af.check_config(p) == af.AF_OK
    assert af.check_config(R(p, lens_mode=af.AF_LENS_NONE)) == af.AF_OK
    ez = p.elem_z.copy()
    ez[5] = p.lens_z + 1e-4
    assert af.check_config(R(p, elem_z=ez)) == af.AF_ERR_ARG
    assert b"above the lens" in lib.af_last_error()
    pz = p.pix_z.copy()
    pz[7] = p.lens_z - 1e-4
    assert af.check_config(R(p, pix_z=pz)) == af.AF_ERR_ARG
    assert af.check_config(R(p, lens_z=p.z0 - 1e-3)) == af.AF_ERR_ARG
    assert af.check_config(R(p, c_lens=0.0)) == af.AF_ERR_ARG


def test_plan_without_gpu_fails_cleanly():
    """Without a CUDA device af_plan reports AF_ERR_CUDA instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    c, keep = af.make_config(synth.config_tiny())
    h = ctypes.c_void_p()
    st = af.load().af_plan(ctypes.byref(c), None, ctypes.byref(h))
    assert st == af.AF_ERR_CUDA
    assert not h.value


def test_batch_calls_validate_arguments_on_the_host():
    """The batch entry points reject bad arguments before any CUDA call."""
    lib = af.load()
    h = ctypes.c_void_p(123)
    assert lib.af_batch_plan(0, None, None, ctypes.byref(h)) == af.AF_ERR_ARG
    assert not h.value                                   # *out cleared on failure
    assert lib.af_batch_plan(1, None, None, None) == af.AF_ERR_ARG
    good, keep = af.make_config(synth.config_tiny())
    bad, keep2 = af.make_config(dataclasses.replace(synth.config_tiny(), c_lens=0.0))
    arr = (ctypes.POINTER(af.AfConfig) * 2)(ctypes.pointer(good), ctypes.pointer(bad))
    assert lib.af_batch_plan(2, arr, None, ctypes.byref(h)) == af.AF_ERR_ARG   # member 1 invalid
    arr2 = (ctypes.POINTER(af.AfConfig) * 2)(ctypes.pointer(good), None)
    assert lib.af_batch_plan(2, arr2, None, ctypes.byref(h)) == af.AF_ERR_ARG  # NULL member
    assert b"configuration 1" in lib.af_last_error()
    p = ctypes.c_void_p()
    assert lib.af_batch_plan_of(None, 0, ctypes.byref(p)) == af.AF_ERR_ARG
    assert lib.af_batch_launch(None) == af.AF_ERR_ARG
    assert lib.af_batch_iterate(None, None, None, None, None, None, None, 1, None) == af.AF_ERR_ARG
    assert lib.af_batch_capture(None, None, None, None, None, None, None, None, 1, 1) == af.AF_ERR_ARG
    assert lib.af_batch_destroy(None) == af.AF_OK


def test_noalloc_wrapper_checks_arguments_before_any_call():
    """The allocation-free CMPE entry point reads nsub^2 * n_patch * patch_npix complex
    values; the binding refuses tensors that do not hold exactly that many, have the
    wrong dtype or layout, or are not on the current CUDA device, before calling it."""
    torch = pytest.importorskip("torch")
    nsub, n_patch, npix = 4, 3, 9
    loss = torch.zeros(1)
    short = torch.zeros((nsub * nsub, n_patch * npix - 1), dtype=torch.complex64)
    with pytest.raises(ValueError, match="complex values"):
        af.af_cmpe_loss_noalloc(short, nsub, n_patch, npix, 0.9, loss)
    with pytest.raises(ValueError, match="complex64"):
        af.af_cmpe_loss_noalloc(torch.zeros((nsub * nsub, n_patch * npix), dtype=torch.complex128),
                                nsub, n_patch, npix, 0.9, loss)
    good = torch.zeros((nsub * nsub, n_patch * npix), dtype=torch.complex64)
    with pytest.raises(ValueError, match="contiguous"):
        af.af_cmpe_loss_noalloc(torch.zeros((n_patch * npix, nsub * nsub), dtype=torch.complex64).t(),
                                nsub, n_patch, npix, 0.9, loss)
    with pytest.raises(ValueError, match="loss"):
        af.af_cmpe_loss_noalloc(good, nsub, n_patch, npix, 0.9, torch.zeros(1, dtype=torch.float64))
    with pytest.raises(ValueError, match="n_active"):
        af.af_cmpe_loss_noalloc(good, nsub, n_patch, npix, 0.9, loss, torch.zeros(1, dtype=torch.int64))
    with pytest.raises(ValueError, match="CUDA"):
        af.af_cmpe_loss_noalloc(good, nsub, n_patch, npix, 0.9, loss)


def test_new_entry_points_refuse_null_arguments_without_a_gpu():
    """af_sweep, af_cmpe_totals, af_set_cmpe_totals, af_fp32_lane_rate and
    af_set_ray_flush_budget check their arguments on the host before any CUDA call."""
    lib = af.load()
    sp = (ctypes.c_double * 2)(1500.0, 1540.0)
    assert lib.af_sweep(None, None, None, sp, 2, 1540.0, 1, None, None) == af.AF_ERR_ARG
    assert lib.af_cmpe_totals(None, None) == af.AF_ERR_ARG
    assert lib.af_set_cmpe_totals(None, None, None) == af.AF_ERR_ARG
    rate = ctypes.c_double()
    assert lib.af_fp32_lane_rate(None, None, ctypes.byref(rate)) == af.AF_ERR_ARG
    assert lib.af_set_wait_limit(-1) == af.AF_OK
    assert lib.af_set_ray_flush_budget(None, 10.0) == af.AF_ERR_ARG


def test_job_entry_points_refuse_null_arguments_without_a_gpu():
    """af_job_reserve / af_job_submit / af_job_wait check their arguments on the host."""
    lib = af.load()
    assert lib.af_job_reserve(None) == af.AF_ERR_ARG
    assert lib.af_job_submit(None, None, None, None, 1, None, None) == af.AF_ERR_ARG
    assert lib.af_job_wait(None) == af.AF_ERR_ARG
