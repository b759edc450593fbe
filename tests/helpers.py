"""Shared helpers for the GPU parity tests: device set-up and the comparison rules.

Comparison rules (GPU float32 vs oracle float64):
* fields: relative L2 error <= 1e-4 per transform;
* continuous phase: wrapped angle error <= 1e-4 rad on pixels whose oracle pre-projection field is
  not tiny, |g| >= 1e-2 rms(g).  The phase of a small field is ill-conditioned: a float32 FFT
  round trip leaves an absolute error of a few 1e-7 rms(g) on every pixel, i.e. ~3e-5 rad at
  |g| = 1e-2 rms but ~3e-4 rad at 1e-3 rms.  At most 0.1 % of pixels may be exempt;
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


def check_continuous_phase(phase_gpu, g_oracle, h_oracle):
    ok = not_tiny(g_oracle)
    assert np.mean(~ok) <= MAX_EXEMPT, f"{np.mean(~ok):.2e} of pixels exempt"
    err = np.abs(wrap(np.asarray(phase_gpu, dtype=np.float64) - np.angle(h_oracle)))
    worst = float(err[ok].max()) if np.any(ok) else 0.0
    assert worst <= PHASE_TOL, f"max wrapped phase error {worst:.3e} rad"
    return worst


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
