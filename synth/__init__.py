"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the FP64 oracle.

This module holds input recipes only -- none of the method's arithmetic (no transform, no
projection, no error metric).  Every generator is driven by ``numpy.random.default_rng(seed)``
(PCG64) and returns float32 arrays, the dtype the library consumes; the oracle upcasts the same
float32 values to float64, so both sides see bit-identical inputs.

Recipes (the paper prints no workloads; these stand in for the target images, starting images and
batch tables that HoloGen's algorithm classes are fed -- section "Algorithm Libraries",
AlgorithmCuda / Randomiser):

* ``blur_target``  -- uniform[0,1) noise, circular separable Gaussian blur (sigma px, taps
  d in [-ceil(4 sigma), ceil(4 sigma)], weights normalised to sum 1), normalised to unit L2 energy.
  Used as a target *amplitude*.
* ``spots_target`` -- sum of ``n_spots`` Gaussian spots, centres uniform in [W/8, 7W/8) x
  [H/8, 7H/8), sigma ~ U[3, 20] px, peak ~ U[0.5, 1), evaluated directly (no wrap) on a zero
  background, unit L2 energy.  Used as an amplitude (Fresnel GS) or an intensity (multi-plane GD).
* ``uniform_phase`` -- uniform [0, 2 pi) starting phase.
* ``symmetrise``   -- A[k] = sqrt((A0[k]^2 + A0[-k]^2) / 2) in FFT order, so that the target is
  reachable by a real (binary) hologram whose replay intensity is point-symmetric.
* ``mixed_sizes``  -- seeded draw of (H, W) hologram sizes for the mixed-size batch.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "blur_target",
    "spots_target",
    "uniform_phase",
    "symmetrise",
    "mixed_sizes",
    "MIXED_SIZE_SET",
]

# (H, W) pairs of the mixed-size serving batch.  "1536x864" is read as width 1536, height 864.
MIXED_SIZE_SET = ((512, 512), (1024, 1024), (864, 1536), (2048, 2048), (4096, 4096))


def _circular_blur_axis(x: np.ndarray, w: np.ndarray, axis: int) -> np.ndarray:
    """Periodic (wrap-around) filtering of x with the symmetric taps w along ``axis``."""
    from scipy import ndimage

    return ndimage.correlate1d(x, w, axis=axis, mode="wrap")


def blur_target(h: int, w: int, sigma: float = 2.0, seed: int = 0) -> np.ndarray:
    """Smoothed-noise target amplitude, float32 [h][w], unit L2 energy."""
    rng = np.random.default_rng(seed)
    u = rng.random((h, w))
    r = int(math.ceil(4.0 * sigma))
    d = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-(d * d) / (2.0 * sigma * sigma))
    k /= k.sum()
    b = _circular_blur_axis(u, k, axis=1)
    b = _circular_blur_axis(b, k, axis=0)
    b /= np.sqrt(np.sum(b * b))
    return b.astype(np.float32)


def spots_target(h: int, w: int, n_spots: int = 50, seed: int = 0) -> np.ndarray:
    """Sum of Gaussian spots on a zero background, float32 [h][w], unit L2 energy."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(w / 8.0, 7.0 * w / 8.0, n_spots)
    cy = rng.uniform(h / 8.0, 7.0 * h / 8.0, n_spots)
    sig = rng.uniform(3.0, 20.0, n_spots)
    amp = rng.uniform(0.5, 1.0, n_spots)
    x = np.arange(w, dtype=np.float64)
    y = np.arange(h, dtype=np.float64)
    img = np.zeros((h, w), dtype=np.float64)
    for k in range(n_spots):
        gx = np.exp(-((x - cx[k]) ** 2) / (2.0 * sig[k] ** 2))
        gy = np.exp(-((y - cy[k]) ** 2) / (2.0 * sig[k] ** 2))
        img += amp[k] * np.outer(gy, gx)
    img /= np.sqrt(np.sum(img * img))
    return img.astype(np.float32)


def uniform_phase(h: int, w: int, seed: int = 1) -> np.ndarray:
    """Uniform [0, 2 pi) phase, float32 [h][w] (values of 2 pi rounding to float32 are folded to 0)."""
    rng = np.random.default_rng(seed)
    p = (rng.random((h, w)) * (2.0 * np.pi)).astype(np.float32)
    p[p >= np.float32(2.0 * np.pi)] = 0.0
    return p


def symmetrise(a0: np.ndarray) -> np.ndarray:
    """Point-symmetric version of an FFT-ordered amplitude: sqrt((A0[k]^2 + A0[-k]^2)/2)."""
    a = a0.astype(np.float64)
    flipped = np.roll(a[::-1, ::-1], shift=(1, 1), axis=(0, 1))  # A0[-k mod n]
    s = np.sqrt(0.5 * (a * a + flipped * flipped))
    return s.astype(np.float32)


def mixed_sizes(n: int = 64, seed: int = 5000, size_set=MIXED_SIZE_SET) -> list[tuple[int, int]]:
    """Seeded draw of n (H, W) sizes from ``size_set``."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(size_set), size=n)
    return [tuple(size_set[i]) for i in idx]
