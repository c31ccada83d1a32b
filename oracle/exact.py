"""Exact solutions used to pin the oracle (test infrastructure only)."""
from __future__ import annotations

import numpy as np


def burgers_sine_exact(x, y, t, a=0.5, b=0.25):
    """u_t + (u^2/2)_x + (u^2/2)_y = 0 with u0 = a + b sin(pi (x+y)).

    Both characteristic speeds equal u, so s = x + y is carried at speed 2u and
    u(x,y,t) solves u = a + b sin(pi (s - 2 u t)) (Newton per point); smooth
    until the breaking time 1/(2 pi b) (2/pi for b = 1/4)."""
    s = np.asarray(x, dtype=np.float64) + np.asarray(y, dtype=np.float64)
    u = a + b * np.sin(np.pi * s)
    for _ in range(60):
        ph = np.pi * (s - 2.0 * u * t)
        F = u - a - b * np.sin(ph)
        dF = 1.0 + b * np.cos(ph) * 2.0 * np.pi * t
        du = F / dF
        u = u - du
        if np.max(np.abs(du)) < 1e-15:
            break
    return u[:, None]
