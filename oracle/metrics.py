"""Replay-quality metric (FP64).  Test infrastructure only.

The paper names a "fast vector normalisation" (section "Algorithm Libraries", Normaliser) and live
per-iteration error charts (section on the process monitor) but defines no metric.  Reading taken
here: the intensity NMSE with the optimal scale,

    s*   = sum(I T) / sum(I^2)
    NMSE = sum((s* I - T)^2) / sum(T^2)

with I the replay intensity |R|^2 of the current hologram and T the target intensity A^2.  This is
the same quantity as 1 - (sum I T)^2 / (sum I^2 sum T^2) (tests pin the identity).
"""
from __future__ import annotations

import numpy as np


def optimal_scale(i: np.ndarray, t: np.ndarray) -> float:
    i = np.asarray(i, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    return float(np.sum(i * t) / np.sum(i * i))


def nmse(i: np.ndarray, t: np.ndarray) -> float:
    """Optimal-scale intensity NMSE of intensity ``i`` against target intensity ``t``."""
    i = np.asarray(i, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    s = optimal_scale(i, t)
    return float(np.sum((s * i - t) ** 2) / np.sum(t * t))
