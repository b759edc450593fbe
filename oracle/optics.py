"""Fourier and single-FFT Fresnel propagation (FP64).  Test infrastructure only.

The paper names "Fourier" and "Fresnel" holograms as keywords only (abstract keywords; section
"HoloGen").  Reading taken here (Goodman, Introduction to Fourier Optics, single-FFT Fresnel
transform):

* SLM pixel (i, j) sits at y_i = (i - floor(H/2)) p, x_j = (j - floor(W/2)) p for pitch p.
* Input-plane chirp  c_z[i, j] = exp(i pi (x_j^2 + y_i^2) / (lambda z)) = c_x[j] c_y[i].
* Fresnel forward:   R = F(h * c_z);   Fresnel inverse:  g = conj(c_z) * F^-1(R).
* The output-plane chirp and the constant exp(ikz)/(i lambda z) are omitted: they have unit modulus
  (up to a constant) and cancel in amplitude replacement and in every intensity.
* Fourier propagation is the same with c_z = 1 (the z -> infinity limit).
F is the unitary 2D DFT of ``oracle.fft``.
"""
from __future__ import annotations

import numpy as np

from .fft import fft2


def chirp_axes(h: int, w: int, wavelength: float, pitch: float, z: float):
    """Separable chirp factors (c_y[H], c_x[W]), complex128, straight from the definition."""
    y = (np.arange(h) - h // 2) * pitch
    x = (np.arange(w) - w // 2) * pitch
    cy = np.exp(1j * np.pi * y * y / (wavelength * z))
    cx = np.exp(1j * np.pi * x * x / (wavelength * z))
    return cy, cx


def chirp(h: int, w: int, wavelength: float, pitch: float, z: float) -> np.ndarray:
    """Full 2D input-plane chirp c_z[H][W] (outer product of the axis factors)."""
    cy, cx = chirp_axes(h, w, wavelength, pitch, z)
    return np.outer(cy, cx)


def chirp_direct(h: int, w: int, wavelength: float, pitch: float, z: float) -> np.ndarray:
    """The same chirp evaluated directly in 2D (no separation), for the separability pin."""
    y = (np.arange(h) - h // 2)[:, None] * pitch
    x = (np.arange(w) - w // 2)[None, :] * pitch
    return np.exp(1j * np.pi * (x * x + y * y) / (wavelength * z))


def propagate(field: np.ndarray, c: np.ndarray | None = None, inverse: bool = False) -> np.ndarray:
    """Forward  R = F(field * c)  or inverse  g = conj(c) * F^-1(field);  c = None means Fourier."""
    f = np.asarray(field, dtype=np.complex128)
    if not inverse:
        return fft2(f if c is None else f * c)
    g = fft2(f, inverse=True)
    return g if c is None else np.conj(c) * g
