"""Own mixed-radix Stockham FFT (FP64).  Test infrastructure only.

Stands in for the paper's FFT handler (section "Algorithm Libraries", FFTHandlerCuda, which wraps
cuFFT).  Written from the textbook Stockham autosort formulation (decimation in time, natural-order
output without a bit-reversal pass): with Ns the length of the sub-transforms already done and R the
radix of the current stage, butterfly j = a*Ns + k (0 <= k < Ns) reads x[j + r N/R] (r < R),
multiplies input r by w_{Ns R}^{r k}, applies an R-point DFT and writes output q to
a*Ns*R + q*Ns + k.  Each stage is one vectorised numpy expression; the R-point DFT is a product with
the explicit R x R DFT matrix.  Any length is accepted: the radix sequence is 4s, then 2, 3, 5, and
any remaining prime factor as its own radix.

``fft2`` uses the unitary convention of ``oracle.dft``.
"""
from __future__ import annotations

import numpy as np


def radices(n: int) -> list[int]:
    """Radix sequence used for length n (product == n)."""
    out: list[int] = []
    m = n
    while m % 4 == 0:
        out.append(4)
        m //= 4
    for p in (2, 3, 5):
        while m % p == 0:
            out.append(p)
            m //= p
    p = 7
    while m > 1:
        while m % p == 0:
            out.append(p)
            m //= p
        p += 2
    return out


def _stockham_last_axis(x: np.ndarray, inverse: bool) -> np.ndarray:
    """Unnormalised DFT along the last axis of a 2D array (batch, n)."""
    b, n = x.shape
    sign = 1.0 if inverse else -1.0
    y = x
    ns = 1
    for r in radices(n):
        m = n // (ns * r)
        v = y.reshape(b, r, m, ns)  # v[b, r, a, k] = y[b, r*(n/r) + a*ns + k]
        rr = np.arange(r)
        kk = np.arange(ns)
        tw = np.exp(sign * 2j * np.pi * (np.outer(rr, kk) % (ns * r)) / (ns * r))  # (r, ns)
        v = v * tw[None, :, None, :]
        d = np.exp(sign * 2j * np.pi * (np.outer(rr, rr) % r) / r)  # d[q, r]
        out = np.tensordot(d, v, axes=([1], [1]))  # (q, b, a, k)
        y = out.transpose(1, 2, 0, 3).reshape(b, n)  # y[b, a*ns*r + q*ns + k]
        ns *= r
    return y


def fft1(x: np.ndarray, inverse: bool = False, axis: int = -1) -> np.ndarray:
    """Unnormalised 1D DFT along ``axis`` (any length)."""
    x = np.asarray(x, dtype=np.complex128)
    xm = np.moveaxis(x, axis, -1)
    shp = xm.shape
    y = _stockham_last_axis(np.ascontiguousarray(xm.reshape(-1, shp[-1])), inverse)
    return np.moveaxis(y.reshape(shp), -1, axis)


def fft2(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Unitary 2D DFT of the last two axes (rows first, then columns)."""
    x = np.asarray(x, dtype=np.complex128)
    h, w = x.shape[-2], x.shape[-1]
    y = fft1(x, inverse, axis=-1)
    y = fft1(y, inverse, axis=-2)
    return y / np.sqrt(h * w)


def ifft2(x: np.ndarray) -> np.ndarray:
    return fft2(x, inverse=True)
