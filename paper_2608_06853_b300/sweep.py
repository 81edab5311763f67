"""Global sound-speed initialisation (Sec. II-C, Sec. III-A; Fig. 3).

The CMPE loss is evaluated with uniform slowness maps over a range of global
speeds (1340-1740 m/s in the paper) and the speed of lowest CMPE starts the
autofocus iterations.  With the dynamic grid, the CMPE pixels and their
kernel spacing move with the active speed c0 so that every patch observes the
same echoes at every c0: depths below the lens and in-patch offsets scale by
c0 / c_ref, directions about the arc centre are kept.  Each evaluation is one
af_forward on the GPU; this module only moves pixels and collects losses.
"""
from __future__ import annotations

import numpy as np
import torch


def dynamic_pixels(problem, c0: float):
    """Pixel positions of the patches for beamforming speed c0 (patch-major order kept)."""
    k = c0 / problem.c_ref
    cx, cz, RL = problem.arc_cx, problem.arc_cz, problem.lens_radius
    px = np.asarray(problem.pix_x, np.float64).reshape(problem.n_patch, problem.patch_npix)
    pz = np.asarray(problem.pix_z, np.float64).reshape(problem.n_patch, problem.patch_npix)
    ccx, ccz = px.mean(1, keepdims=True), pz.mean(1, keepdims=True)
    rho = np.hypot(ccx - cx, ccz - cz)
    ux, uz = (ccx - cx) / rho, (ccz - cz) / rho
    rho2 = RL + (rho - RL) * k
    ncx, ncz = cx + rho2 * ux, cz + rho2 * uz
    nx = ncx + k * (px - ccx)
    nz = ncz + k * (pz - ccz)
    # float32-representable, like every geometry input
    return (nx.ravel().astype(np.float32).astype(np.float64), nz.ravel().astype(np.float32).astype(np.float64))


def global_speed_sweep(plan, problem, iq, speeds=None, dynamic=True, iq_scale=None):
    """CMPE loss for uniform maps at each speed; returns (speeds, cmpe, active terms, best).
    The plan's pixels are restored afterwards."""
    dev = torch.device("cuda", torch.cuda.current_device())
    speeds = np.arange(1340.0, 1741.0, 10.0) if speeds is None else np.asarray(speeds, np.float64)
    cmpe, active = [], []
    try:
        # tensors made and read on the plan's stream, which its kernels run on
        with torch.cuda.stream(plan.stream):
            loss = torch.zeros(4, device=dev)
            for c0 in speeds:
                if dynamic:
                    plan.af_set_pixels(*dynamic_pixels(problem, c0))
                s = torch.full((problem.nz, problem.nx), 1.0 / c0, dtype=torch.float32, device=dev)
                plan.af_forward(iq, s, loss, iq_scale)
                _, _, m = plan.cmpe()
                cmpe.append(float(loss[1]))
                active.append(m)
    finally:
        if dynamic:
            plan.af_set_pixels(problem.pix_x, problem.pix_z)
    cmpe = np.asarray(cmpe)
    return speeds, cmpe, np.asarray(active), float(speeds[int(np.argmin(cmpe))])
