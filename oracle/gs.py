"""Gerchberg-Saxton phase retrieval (FP64).  Test infrastructure only.

The paper's HoloGenAlgGSCuda (section "Algorithm Libraries") implements "the Gerchberg-Saxton
algorithm and other iterative Fourier transform approaches"; the iteration body lives in
RunIterations() (section "Algorithm Interface").  No formula is printed.  Reading taken here
(Gerchberg & Saxton 1972, in the error-reduction form of Fienup 1982), for SLM field h_k:

    R_k     = F(h_k * c)                     (c = 1 Fourier, c = Fresnel chirp otherwise)
    NMSE_k  = NMSE(|R_k|^2, A^2)             (oracle.metrics)
    R'_k    = A_s * R_k / |R_k|              (amplitude replacement, A_s = A sqrt(HW / sum A^2))
    h_{k+1} = P_SLM(conj(c) * F^-1(R'_k))   (continuous / N-level / binary projection)

with h_0 = P_SLM(exp(i phi_0)) (reading: the starting phase is projected so that every h_k is a
realisable hologram).  ``nmse[k]`` for k = 0..n_iter is the NMSE of h_k; h_{n_iter} is the output.

Illumination (AlgorithmCuda stores "target, illumination and starting images", section "Algorithm
Libraries"): the SLM is lit with amplitude profile illum and only sets the phase, so the SLM-plane
constraint set is {illum e^{i phi}} and its nearest-point projection is illum * P_SLM(g); A_s then
carries the field energy sum illum^2 (reading: the target at the illuminated SLM's energy).

Multi-plane GS (averaged projections; not in the paper -- the comparator of the gradient-descent
optimiser): with P planes, chirps c_p and targets A_p,

    h_{k+1} = P_SLM( (1/P) sum_p conj(c_p) F^-1( A_{p,s} R_p / |R_p| ) ),   R_p = F(h_k c_p)

which is alternating projection in the product space of the P replay fields; ``nmse[k]`` is the mean
over planes.
"""
from __future__ import annotations

import numpy as np

from .fft import fft2
from .metrics import nmse
from .project import amplitude_replace, hologram_phase, slm_project


def scaled_amplitude(a: np.ndarray, energy: float | None = None) -> np.ndarray:
    """A_s = A sqrt(E / sum A^2): the replay amplitude carrying the SLM field's energy E (HW for a
    unit-modulus field, sum illum^2 under an illumination profile)."""
    a = np.asarray(a, dtype=np.float64)
    e = float(a.size) if energy is None else float(energy)
    return a * np.sqrt(e / np.sum(a * a))


def _illuminate(h: np.ndarray, illum) -> np.ndarray:
    """The SLM field under an illumination amplitude profile (None: uniform, unit amplitude)."""
    return h if illum is None else np.asarray(illum, dtype=np.float64) * h


def _energy(h: np.ndarray, illum) -> float:
    return float(h.size) if illum is None else float(np.sum(np.asarray(illum, dtype=np.float64) ** 2))


def gs(target_amp, init_phase, n_iter: int, n_levels: int = 0, c=None, illum=None):
    """Single-plane GS.  Returns dict(h, phase, q, nmse[n_iter+1]).

    illum: the SLM illumination amplitude profile [H][W] (AlgorithmCuda keeps an illumination image,
    section "Algorithm Libraries"); the SLM sets the phase only, so every SLM field is
    h = illum * P_SLM(.) and A_s carries its energy sum illum^2.  None: uniform unit illumination.
    """
    a = np.asarray(target_amp, dtype=np.float64)
    t = a * a
    h, q = slm_project(np.exp(1j * np.asarray(init_phase, dtype=np.float64)), n_levels)
    h = _illuminate(h, illum)
    a_s = scaled_amplitude(a, _energy(h, illum))
    curve = []
    for _ in range(n_iter):
        r = fft2(h if c is None else h * c)
        curve.append(nmse(np.abs(r) ** 2, t))
        g = fft2(amplitude_replace(r, a_s), inverse=True)
        if c is not None:
            g = np.conj(c) * g
        h, q = slm_project(g, n_levels)
        h = _illuminate(h, illum)
    r = fft2(h if c is None else h * c)
    curve.append(nmse(np.abs(r) ** 2, t))
    return {"h": h, "phase": hologram_phase(h), "q": q, "nmse": np.array(curve)}


def gs_step(h, target_amp, n_levels: int = 0, c=None, illum=None):
    """One GS iteration from a given SLM field h (teacher forcing).

    Returns dict(h, q, g) with g the pre-projection SLM-plane field conj(c) F^-1(R').
    """
    a = np.asarray(target_amp, dtype=np.float64)
    h = np.asarray(h, dtype=np.complex128)
    a_s = scaled_amplitude(a, _energy(h, illum))
    r = fft2(h if c is None else h * c)
    g = fft2(amplitude_replace(r, a_s), inverse=True)
    if c is not None:
        g = np.conj(c) * g
    h1, q = slm_project(g, n_levels)
    return {"h": _illuminate(h1, illum), "q": q, "g": g}


def replay_error(h, target_amp, c=None, illum=None) -> float:
    """Fienup's error  sum (|F(h c)| - A_s)^2  (non-increasing along GS, any projection)."""
    h = np.asarray(h, dtype=np.complex128)
    a_s = scaled_amplitude(target_amp, _energy(h, illum))
    r = fft2(h if c is None else h * c)
    return float(np.sum((np.abs(r) - a_s) ** 2))


def multiplane_gs(target_amps, init_phase, n_iter: int, chirps, n_levels: int = 0):
    """Averaged-projection multi-plane GS.  Returns dict(h, phase, q, nmse[n_iter+1] (plane mean))."""
    amps = [np.asarray(a, dtype=np.float64) for a in target_amps]
    ts = [a * a for a in amps]
    a_s = [scaled_amplitude(a) for a in amps]
    p = len(amps)
    h, q = slm_project(np.exp(1j * np.asarray(init_phase, dtype=np.float64)), n_levels)
    curve = []
    for _ in range(n_iter):
        acc = np.zeros_like(h)
        errs = []
        for k in range(p):
            r = fft2(h * chirps[k])
            errs.append(nmse(np.abs(r) ** 2, ts[k]))
            acc += np.conj(chirps[k]) * fft2(amplitude_replace(r, a_s[k]), inverse=True)
        curve.append(float(np.mean(errs)))
        h, q = slm_project(acc / p, n_levels)
    errs = [nmse(np.abs(fft2(h * chirps[k])) ** 2, ts[k]) for k in range(p)]
    curve.append(float(np.mean(errs)))
    return {"h": h, "phase": hologram_phase(h), "q": q, "nmse": np.array(curve)}


def multiplane_error(h, target_amps, chirps) -> float:
    """Product-space distance  sum_p sum (|F(h c_p)| - A_{p,s})^2."""
    e = 0.0
    for a, c in zip(target_amps, chirps):
        r = fft2(np.asarray(h, dtype=np.complex128) * c)
        e += float(np.sum((np.abs(r) - scaled_amplitude(a)) ** 2))
    return e
