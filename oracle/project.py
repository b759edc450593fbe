"""Projections onto the SLM-plane and replay-plane constraint sets (FP64).  Test infrastructure only.

The paper names a "base level quantisation algorithm" (section "Algorithm Libraries",
QuantiserCuda) and the amplitude-replacement step of Gerchberg-Saxton (HoloGenAlgGSCuda) without
formulas.  Readings taken here (each is the nearest-point projection onto its set):

SLM constraint (phase-only SLM, unit modulus):
* continuous: h = g / |g|, and h = 1 where g == 0;
* N-level (N >= 2): levels phi_q = 2 pi q / N; with a = arg(g) in [0, 2 pi),
  q = floor(a N / (2 pi) + 1/2) mod N, h = exp(i phi_q).  An exact midpoint between two levels goes
  to the higher index (mod N).  N = 2 is binary {0, pi}: h = +1 / -1.  g == 0 gives q = 0.

Multi-amplitude / complex-modulation SLM (section "Application": the SLM type option offers a
multi-amplitude SLM, MultiAmpSLM, with its own settings; reading): the pixel takes one of M given
complex values m_q (e.g. the measured responses of its drive levels); the projection is the
nearest of them in the complex plane, h = m_q with q = argmin |g - m_q| (the lowest index on a
tie).  For M unit-modulus values
at equal angles this is the N-level rule above.  Unlike the phase-only sets this one is not a
cone, so the scale of g matters: g is taken in the unitary scale of the loop (the replay target
carries the energy of a unit-modulus SLM field).

Replay constraint (amplitude replacement): R' = A * R / |R|, with R / |R| = 1 where R == 0.
"""
from __future__ import annotations

import numpy as np


def phase_of(g: np.ndarray) -> np.ndarray:
    """arg(g) folded into [0, 2 pi)."""
    a = np.angle(g)
    a = np.where(a < 0.0, a + 2.0 * np.pi, a)
    return np.where(a >= 2.0 * np.pi, 0.0, a)


def quantise_index(g: np.ndarray, n_levels: int) -> np.ndarray:
    """Nearest level index q (int64) of arg(g) among n_levels equally spaced phases."""
    a = phase_of(g)
    q = np.floor(a * n_levels / (2.0 * np.pi) + 0.5).astype(np.int64)
    return np.mod(q, n_levels)


def level_field(q: np.ndarray, n_levels: int) -> np.ndarray:
    """exp(2 pi i q / N) with the exact values +-1, +-i where they are representable."""
    ang = 2.0 * np.pi * np.asarray(q, dtype=np.float64) / n_levels
    h = np.exp(1j * ang)
    # make the level set exact on the axes (4 q / N integer)
    qq = (4 * np.asarray(q, dtype=np.int64)) % (4 * n_levels)
    on_axis = (qq % n_levels) == 0
    if np.any(on_axis):
        quarter = (qq // n_levels) % 4
        axis_vals = np.array([1.0 + 0.0j, 0.0 + 1.0j, -1.0 + 0.0j, 0.0 - 1.0j])
        h = np.where(on_axis, axis_vals[quarter], h)
    return h


def table_project(g: np.ndarray, table) -> tuple:
    """Nearest entry of a finite set of complex SLM values (Euclidean distance; on a tie the lowest
    index).  Returns (h, q) with q the entry index (int64)."""
    g = np.asarray(g, dtype=np.complex128)
    t = np.asarray(table, dtype=np.complex128).ravel()
    q = np.zeros(g.shape, dtype=np.int64)
    best = np.abs(g - t[0]) ** 2
    for i in range(1, t.size):
        d = np.abs(g - t[i]) ** 2
        closer = d < best
        q = np.where(closer, i, q)
        best = np.where(closer, d, best)
    return t[q], q


def slm_project(g: np.ndarray, n_levels):
    """SLM projection.  Returns (h, q): q is None for continuous phase (n_levels == 0).  n_levels may
    also be an array of complex SLM values (a multi-amplitude / complex-modulation SLM), projected
    onto by table_project."""
    g = np.asarray(g, dtype=np.complex128)
    if isinstance(n_levels, np.ndarray):
        return table_project(g, n_levels)
    if n_levels == 0:
        mag = np.abs(g)
        h = np.where(mag > 0.0, g / np.where(mag > 0.0, mag, 1.0), 1.0 + 0.0j)
        return h, None
    q = quantise_index(g, n_levels)
    return level_field(q, n_levels), q


def amplitude_replace(r: np.ndarray, amp: np.ndarray) -> np.ndarray:
    """R' = A R / |R| (R / |R| := 1 where R == 0)."""
    r = np.asarray(r, dtype=np.complex128)
    mag = np.abs(r)
    unit = np.where(mag > 0.0, r / np.where(mag > 0.0, mag, 1.0), 1.0 + 0.0j)
    return np.asarray(amp, dtype=np.float64) * unit


def hologram_phase(h: np.ndarray) -> np.ndarray:
    """Output phase of a unit-modulus hologram in [0, 2 pi)."""
    return phase_of(h)
