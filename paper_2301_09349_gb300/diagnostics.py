"""Host-side post-processing of force histories (not on the device path).

strouhal(): the shedding Strouhal number St = f D / U_inf from a lift
coefficient history C_l(t) (the paper reports St for the cylinder and the
sphere, Secs. 3-4): the dominant frequency is taken from the upward zero
crossings of C_l - mean(C_l) over the analysed window, each crossing located
by linear interpolation between samples, f = (crossings - 1) / (last - first).
"""
from __future__ import annotations

import numpy as np


def strouhal(t, cl, D: float = 1.0, U: float = 1.0, t_min: float = 0.0) -> float:
    t = np.asarray(t, dtype=np.float64)
    cl = np.asarray(cl, dtype=np.float64)
    sel = t >= t_min
    t, cl = t[sel], cl[sel]
    if len(t) < 4:
        return float("nan")
    y = cl - cl.mean()
    up = np.nonzero((y[:-1] < 0.0) & (y[1:] >= 0.0))[0]
    if len(up) < 2:
        return float("nan")
    tc = t[up] - y[up] * (t[up + 1] - t[up]) / (y[up + 1] - y[up])
    f = (len(tc) - 1) / (tc[-1] - tc[0])
    return float(f * D / U)
