"""Post-processing of the plane statistics (host side; the statistics come
from lbm_stats, [9][xbin][y]: <u>, <v>, <w>, <u'u'>, <v'v'>, <w'w'>, <u'v'>,
<u'w'>, <v'w'>, row y's cell centre at height y + 1/2 above the ground).
"""
from __future__ import annotations

import numpy as np


def at_height(profile, height: float) -> float:
    """A per-row profile at `height` (in cells above the ground): linear
    between the cell centres y + 1/2, the end rows' values beyond them."""
    p = np.asarray(profile, dtype=np.float64)
    return float(np.interp(height, np.arange(p.size) + 0.5, p))


def friction_velocity(stats, height: float, xbin=None) -> float:
    """The forest friction velocity of Sec. 5, u_* = (<u'v'>^2 + <v'w'>^2)^(1/4),
    from the Reynolds stresses at `height` (the paper takes y/h = 2, i.e.
    height = 2h in cells).  With several x-bins the stresses are averaged over
    the bins (equal widths) unless one bin is chosen."""
    s = np.asarray(stats, dtype=np.float64)
    uv, vw = s[6], s[8]
    if xbin is None:
        uv, vw = uv.mean(axis=0), vw.mean(axis=0)
    else:
        uv, vw = uv[xbin], vw[xbin]
    return float((at_height(uv, height) ** 2 + at_height(vw, height) ** 2) ** 0.25)
