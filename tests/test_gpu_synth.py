"""The GPU echo simulator (synth_gpu.cu) against the host simulator (synth.c).

Both model the same acquisition physics; the host version is the reference.
One-way times are float64 on both sides and agree to rounding.  The echoes
accumulate in float on the GPU and in double on the host.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_whole_small_acquisition_matches_host_simulator():
    p = synth.config_tiny()
    x, z, a = synth.sector_scatterers(p, 2000, 20261202)
    T_cpu = synth.oneway_times(p, x, z)
    T_gpu = synth.oneway_times_gpu(p, x, z).cpu().numpy()
    assert np.abs(T_gpu - T_cpu).max() <= 1e-13
    psi_cpu = synth.echoes(p, T_cpu, a)
    psi_gpu = synth.echoes_gpu(p, torch.from_numpy(T_cpu).cuda(), a).cpu().numpy()
    assert rel_l2(psi_gpu, psi_cpu) <= 1e-5
    # reciprocity is exact: each pair is computed once and written to both places
    assert np.array_equal(psi_gpu, psi_gpu.transpose(1, 0, 2))


def test_flat_lens_and_no_lens_times_match_host_simulator():
    p = synth.config_linear_tiny()
    x, z, _ = synth.sector_scatterers(p, 500, 7)
    assert np.abs(synth.oneway_times_gpu(p, x, z).cpu().numpy() - synth.oneway_times(p, x, z)).max() <= 1e-13
    q = dataclasses.replace(synth.config_tiny(), lens_mode=1)
    x, z, _ = synth.sector_scatterers(q, 500, 8)
    assert np.abs(synth.oneway_times_gpu(q, x, z).cpu().numpy() - synth.oneway_times(q, x, z)).max() <= 1e-13


def test_full_size_speckle_matches_host_on_sampled_pairs():
    """128 elements, 10 scatterers per resolution cell (~7e5), wavy fat/liver interface:
    the (t, r) traces of three elements, recomputed on the host from the host's own
    one-way times of those elements."""
    p = synth.config_full()
    n = synth.speckle_count(p)
    assert 6e5 < n < 8e5
    psi = synth.simulate_gpu(p, n, seed=20261203)
    x, z, a = synth.sector_scatterers(p, n, 20261203)
    els = [3, 64, 121]
    sub = dataclasses.replace(p, elem_x=p.elem_x[els], elem_z=p.elem_z[els])
    T_sub = synth.oneway_times(sub, x, z)
    ref = synth.echoes(sub, T_sub, a)
    got = psi[els][:, els].cpu().numpy()
    assert rel_l2(got, ref) <= 1e-5
    assert np.abs(got).max() > 0
