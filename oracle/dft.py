"""Naive discrete Fourier transforms (FP64).  Test infrastructure only.

Convention (a reading: the paper only says cuFFT performs "the FFT element of the algorithms",
section "HoloGen"): the unitary 2D DFT

    X[k, l] = (H W)^(-1/2) sum_{m, n} x[m, n] exp(-2 pi i (k m / H + l n / W))

and its inverse with +i and the same scale.  Fields are in FFT order (DC at [0, 0]).
"""
from __future__ import annotations

import numpy as np


def dft_matrix(n: int, inverse: bool = False) -> np.ndarray:
    """Unnormalised DFT matrix D[k, m] = exp(-+ 2 pi i k m / n), float64 complex."""
    sign = 1.0 if inverse else -1.0
    k = np.arange(n)
    # reduce k*m mod n first so the angle stays small and exact in float64
    km = np.outer(k, k) % n
    return np.exp(sign * 2j * np.pi * km / n)


def dft1(x: np.ndarray, inverse: bool = False, axis: int = -1) -> np.ndarray:
    """Unnormalised 1D DFT along ``axis`` by matrix product (O(N^2))."""
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[axis]
    d = dft_matrix(n, inverse)
    xm = np.moveaxis(x, axis, -1)
    y = xm @ d.T
    return np.moveaxis(y, -1, axis)


def dft2(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Unitary 2D DFT of the last two axes via separable naive DFTs."""
    x = np.asarray(x, dtype=np.complex128)
    h, w = x.shape[-2], x.shape[-1]
    y = dft1(dft1(x, inverse, axis=-1), inverse, axis=-2)
    return y / np.sqrt(h * w)


def dft2_bruteforce(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Unitary 2D DFT as the explicit quadruple sum (tiny sizes only)."""
    x = np.asarray(x, dtype=np.complex128)
    h, w = x.shape
    sign = 1.0 if inverse else -1.0
    out = np.zeros((h, w), dtype=np.complex128)
    for k in range(h):
        for l in range(w):
            acc = 0.0 + 0.0j
            for m in range(h):
                for n in range(w):
                    acc += x[m, n] * np.exp(sign * 2j * np.pi * ((k * m) / h + (l * n) / w))
            out[k, l] = acc
    return out / np.sqrt(h * w)
