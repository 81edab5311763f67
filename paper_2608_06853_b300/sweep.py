"""Global sound-speed initialisation (Sec. II-C, Sec. III-A; Fig. 3).

The CMPE loss is evaluated with uniform slowness maps over a range of global
speeds (1340-1740 m/s in the paper) and the speed of lowest CMPE starts the
autofocus iterations.  With the dynamic grid the CMPE pixels and their kernel
spacing move with the active speed so that every patch observes the same echoes
at every speed.  The library does all of it on the device (af_sweep); this
module only picks the speeds and the minimum.
"""
from __future__ import annotations

import numpy as np
import torch


def global_speed_sweep(plan, problem, iq, speeds=None, dynamic=True, iq_scale=None):
    """CMPE loss for uniform maps at each speed; returns (speeds, cmpe, active terms, best).
    The plan's pixels are those of the problem's reference speed `problem.c_ref`."""
    speeds = np.arange(1340.0, 1741.0, 10.0) if speeds is None else np.asarray(speeds, np.float64)
    with torch.cuda.stream(plan.stream):
        cm, act = plan.af_sweep(iq, speeds, problem.c_ref, dynamic=dynamic, iq_scale=iq_scale)
        cmpe = cm.cpu().numpy().astype(np.float64)
        active = act.cpu().numpy()
    return speeds, cmpe, active, float(speeds[int(np.argmin(cmpe))])
