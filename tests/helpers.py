"""Shared helpers for the GPU parity tests: device set-up and the comparison rules.

Comparison rules (GPU float32 vs oracle float64):
* fields: relative L2 error <= 1e-4 per transform;
* continuous phase: the SLM fields exp(i phi) agree to relative L2 <= 1e-4 (the field bound), and on
  every pixel the phase error times |g| (g: the oracle's pre-projection field) stays within the
  float32 rounding of the transforms, 8 u log2(HW) rms(g) with u = 2^-24.  The phase of a small field
  is ill-conditioned: a float32 FFT round trip leaves an absolute error of order u log2(HW) rms(g)
  on every pixel (measured on GB300: up to 3.4e-6 rms(g) at 2^22 pixels, u log2(HW) = 1.3e-6), i.e.
  ~3e-4 rad at |g| = 1e-2 rms but ~3e-6 rad at a typical pixel;
* quantised phase: level indices equal on >= 99.9 % of pixels, and every mismatch on a non-tiny
  pixel has an oracle pre-quantisation phase within 1e-4 rad of a level boundary;
* NMSE: within 1 % relative.
"""
from __future__ import annotations

import numpy as np
import pytest

FIELD_TOL = 1e-4
PHASE_TOL = 1e-4
NMSE_RTOL = 1e-2
LEVEL_AGREE = 0.999
TINY = 1e-2
MAX_EXEMPT = 1e-3


def cuda_device():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from __graft_entry__ import build

    build()
    return torch.device("cuda:0")


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def wrap(d):
    return np.angle(np.exp(1j * np.asarray(d, dtype=np.float64)))


def not_tiny(g) -> np.ndarray:
    m = np.abs(g)
    return m >= TINY * np.sqrt(np.mean(m * m))


ROUNDING_MULT = 8.0  # float32 transform rounding bound: ROUNDING_MULT * 2^-24 * log2(HW) * rms(g)


def check_continuous_phase(phase_gpu, g_oracle, h_oracle):
    phase_gpu = np.asarray(phase_gpu, dtype=np.float64)
    assert rel_l2(np.exp(1j * phase_gpu), h_oracle) <= FIELD_TOL
    m = np.abs(g_oracle)
    rms = np.sqrt(np.mean(m * m))
    err = np.abs(wrap(phase_gpu - np.angle(h_oracle)))
    bound = ROUNDING_MULT * 2.0 ** -24 * np.log2(m.size) * rms
    worst = float(np.max(err * m))
    assert worst <= bound, f"phase error x |g| = {worst / rms:.3e} rms(g) > {bound / rms:.3e} rms(g)"
    return float(np.max(err[not_tiny(g_oracle)])) if np.any(not_tiny(g_oracle)) else 0.0


def check_levels(q_gpu, q_oracle, g_oracle, n_levels):
    q_gpu = np.asarray(q_gpu).astype(np.int64)
    q_oracle = np.asarray(q_oracle).astype(np.int64)
    mism = q_gpu != q_oracle
    agree = 1.0 - float(np.mean(mism))
    assert agree >= LEVEL_AGREE, f"level agreement {agree:.6f}"
    if np.any(mism):
        a = np.mod(np.angle(g_oracle), 2 * np.pi)
        # distance to the nearest boundary 2 pi (k + 1/2) / N
        t = a * n_levels / (2 * np.pi) - 0.5
        dist = np.abs(t - np.round(t)) * 2 * np.pi / n_levels
        bad = mism & not_tiny(g_oracle) & (dist > PHASE_TOL)
        assert not np.any(bad), f"{int(bad.sum())} mismatches away from a level boundary (max {dist[bad].max():.3e} rad)"
    return agree


def check_nmse(got, want, rtol=NMSE_RTOL):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    rel = np.abs(got - want) / np.abs(want)
    assert np.all(rel <= rtol), f"NMSE rel error {rel.max():.3e}: got {got}, want {want}"
    return float(rel.max())
