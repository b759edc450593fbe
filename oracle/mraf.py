"""Mixed-region amplitude freedom (MRAF) and hybrid input-output (HIO), iterative Fourier transform
variants with a signal window (FP64).  Test infrastructure only.

The paper's GS class covers "the Gerchberg-Saxton algorithm and other iterative Fourier transform
approaches" (section "Algorithm Libraries", HoloGenAlgGSCuda) and keeps region-of-interest helpers
(StridedChunkRange, same section); it prints no formula.  Reading taken here: MRAF (Pasienski &
DeMarco 2008).  The replay plane is split into a signal region S (the window where the target is
imposed) and a noise region N (its complement); with mixing parameter m in (0, 1]:

    R_k     = F(h_k * c)
    R'_k    = m A_s R_k / |R_k|   on S,      (1 - m) R_k   on N
    h_{k+1} = P_SLM(conj(c) * F^-1(R'_k))

with A_s = A sqrt(HW / sum_S A^2) on S (the target carries the energy of a unit-modulus field, as in
plain GS) and the NMSE of R6 taken over S only (ROI NMSE).  With S the whole plane the SLM
projection removes the factor m, so MRAF is plain GS for any m.  ``nmse[k]``, k = 0..n_iter, is the
ROI NMSE of h_k; h_0 = P_SLM(exp(i phi_0)).
"""
from __future__ import annotations

import numpy as np

from .fft import fft2
from .project import hologram_phase, slm_project


def roi_nmse(i: np.ndarray, t: np.ndarray, mask: np.ndarray) -> float:
    """NMSE = 1 - (sum IT)^2 / (sum I^2 sum T^2) over the pixels where mask is set."""
    m = np.asarray(mask, dtype=bool)
    ii = np.asarray(i, dtype=np.float64)[m]
    tt = np.asarray(t, dtype=np.float64)[m]
    s_it, s_ii, s_tt = np.sum(ii * tt), np.sum(ii * ii), np.sum(tt * tt)
    if s_ii <= 0.0 or s_tt <= 0.0:
        return 1.0
    return float(1.0 - s_it * s_it / (s_ii * s_tt))


def signal_amplitude(a: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """A_s = A sqrt(HW / sum_S A^2) on S, 0 on N (0 everywhere when the target has no energy on S)."""
    a = np.asarray(a, dtype=np.float64)
    m = np.asarray(mask, dtype=bool)
    e = np.sum(a[m] ** 2)
    return np.where(m, a * np.sqrt(a.size / e), 0.0) if e > 0.0 else np.zeros_like(a)


def mraf_replace(r: np.ndarray, a_s: np.ndarray, mask: np.ndarray, mix: float) -> np.ndarray:
    """R' = mix A_s R / |R| on S (R / |R| := 1 where R = 0), (1 - mix) R on N."""
    r = np.asarray(r, dtype=np.complex128)
    mag = np.abs(r)
    unit = np.where(mag > 0.0, r / np.where(mag > 0.0, mag, 1.0), 1.0 + 0.0j)
    return np.where(np.asarray(mask, dtype=bool), mix * a_s * unit, (1.0 - mix) * r)


def mraf_step(h, target_amp, mask, mix: float, n_levels: int = 0, c=None):
    """One MRAF iteration from SLM field h.  Returns dict(h, q, g, r_new) with g the pre-projection
    SLM-plane field and r_new the replaced replay field R'."""
    a_s = signal_amplitude(target_amp, mask)
    h = np.asarray(h, dtype=np.complex128)
    r = fft2(h if c is None else h * c)
    r_new = mraf_replace(r, a_s, mask, mix)
    g = fft2(r_new, inverse=True)
    if c is not None:
        g = np.conj(c) * g
    h1, q = slm_project(g, n_levels)
    return {"h": h1, "q": q, "g": g, "r_new": r_new}


def mraf(target_amp, mask, mix: float, init_phase, n_iter: int, n_levels: int = 0, c=None):
    """MRAF loop.  Returns dict(h, phase, q, nmse[n_iter+1]) with the ROI NMSE of every iterate."""
    a = np.asarray(target_amp, dtype=np.float64)
    t = a * a
    h, q = slm_project(np.exp(1j * np.asarray(init_phase, dtype=np.float64)), n_levels)
    curve = []
    for _ in range(n_iter):
        r = fft2(h if c is None else h * c)
        curve.append(roi_nmse(np.abs(r) ** 2, t, mask))
        step = mraf_step(h, a, mask, mix, n_levels, c)
        h, q = step["h"], step["q"]
    r = fft2(h if c is None else h * c)
    curve.append(roi_nmse(np.abs(r) ** 2, t, mask))
    return {"h": h, "phase": hologram_phase(h), "q": q, "nmse": np.array(curve)}


def hio_step(h, x, target_amp, mask, beta: float, n_levels: int = 0, c=None):
    """One HIO iteration from SLM field h_k and replay-plane input X_k (None for k = 0: X_0 = Y_0).
    Returns dict(h, q, g, x) with g the pre-projection SLM-plane field and x = X_{k+1}."""
    m = np.asarray(mask, dtype=bool)
    a_s = signal_amplitude(target_amp, m)
    h = np.asarray(h, dtype=np.complex128)
    y = fft2(h if c is None else h * c)
    if x is None:
        x = y
    mag = np.abs(y)
    unit = np.where(mag > 0.0, y / np.where(mag > 0.0, mag, 1.0), 1.0 + 0.0j)
    x_new = np.where(m, a_s * unit, x - beta * y)
    g = fft2(x_new, inverse=True)
    if c is not None:
        g = np.conj(c) * g
    h1, q = slm_project(g, n_levels)
    return {"h": h1, "q": q, "g": g, "x": x_new}


def hio(target_amp, mask, beta: float, init_phase, n_iter: int, n_levels: int = 0, c=None):
    """Fienup's hybrid input-output with the replay plane as the constrained domain (FP64).

    Reading of "other iterative Fourier transform approaches" (section "Algorithm Libraries"): HIO
    (Fienup 1982) with the roles of the planes as in hologram design.  The input is a replay-plane
    field X_k; the system maps it through the SLM constraint, h_k = P_SLM(conj(c) F^-1(X_k)), and
    back, Y_k = F(h_k c).  Where the replay constraint applies -- the signal region S -- the new input
    imposes the target, X_{k+1} = A_s Y_k / |Y_k|; elsewhere it feeds the output back negatively,
    X_{k+1} = X_k - beta Y_k.  The loop starts from h_0 = P_SLM(exp(i phi_0)) with X_0 := Y_0 on N.
    A_s as for MRAF (signal_amplitude); ``nmse[k]`` is the ROI NMSE of h_k.  With S the whole plane
    it is plain GS.  Returns dict(h, phase, q, nmse[n_iter+1]).
    """
    a = np.asarray(target_amp, dtype=np.float64)
    m = np.asarray(mask, dtype=bool)
    t = a * a
    h, q = slm_project(np.exp(1j * np.asarray(init_phase, dtype=np.float64)), n_levels)
    x = None
    curve = []
    for _ in range(n_iter):
        y = fft2(h if c is None else h * c)
        curve.append(roi_nmse(np.abs(y) ** 2, t, m))
        step = hio_step(h, x, a, m, beta, n_levels, c)
        h, q, x = step["h"], step["q"], step["x"]
    y = fft2(h if c is None else h * c)
    curve.append(roi_nmse(np.abs(y) ** 2, t, m))
    return {"h": h, "phase": hologram_phase(h), "q": q, "nmse": np.array(curve)}
