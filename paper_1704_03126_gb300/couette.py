"""Couette-flow post-processing (Sec. II): the mean streamwise velocity profile and Q*.

* The mean streamwise velocity at height x2 is the average of u1 over x1 along the row (Sec. II.B
  compares these profiles between the rough and the smooth channel).  Solid cells count as zero, so
  that the profile integrates to the flow rate: Q = int u1_bar(x2) dx2 (the Q of the Couette section
  with the channel length divided out).
* Q* = Q_r / Q_s, the flow rate over the rough wall over that between smooth plates at the same Kn.

Both act on the fields the library returns (dvm_fields); nothing here solves anything.
"""
from __future__ import annotations

import numpy as np


def row_centres(ny: int, ly: float = 1.0, row_heights=None, y0: float = 0.0):
    """Heights x2 of the row centres: equal rows of ly / ny, or the given heights, from y0."""
    if row_heights is None:
        return y0 + (np.arange(ny) + 0.5) * (ly / ny)
    h = np.asarray(row_heights, dtype=np.float64)
    if h.shape != (ny,):
        raise ValueError("row_heights needs one entry per row")
    return y0 + np.cumsum(h) - 0.5 * h


def mean_profile(u1, mask, ly: float = 1.0, row_heights=None, y0: float = 0.0):
    """(x2 of each row centre, mean of u1 over the row with solid cells as zero)."""
    u1 = np.asarray(u1, dtype=np.float64)
    mask = np.asarray(mask)
    if u1.shape != mask.shape:
        raise ValueError("u1 and mask differ in shape")
    ny, nx = mask.shape
    u = np.where(mask == 0, u1, 0.0)
    return row_centres(ny, ly, row_heights, y0), u.sum(axis=1) / nx


def profile_at(y, ubar, points):
    """The profile interpolated linearly at the given heights."""
    return np.interp(np.asarray(points, dtype=np.float64), y, ubar)


def q_star(q_rough: float, q_smooth: float) -> float:
    """Q* = Q_r / Q_s (Sec. II)."""
    return q_rough / q_smooth
