"""Pins for the oracle's MRAF (mixed-region amplitude freedom) and its region-of-interest NMSE.

* With the signal region the whole plane, MRAF is plain GS for any mixing parameter (the SLM
  projection removes the factor m): checked against the pinned GS oracle, every projection, Fourier
  and Fresnel.
* With an empty signal region the replay field is only scaled by (1 - m), so a projected hologram is
  a fixed point.
* Energy bookkeeping of one replacement: sum_S |R'|^2 = m^2 HW and sum_N |R'|^2 = (1 - m)^2 sum_N |R|^2.
* One step on 6 x 8 with the explicit DFT matrices equals the FFT-based step.
* ROI NMSE: the whole-plane mask gives the plain NMSE; values outside the mask do not matter; an
  exact (scaled) match on the mask gives 0.
"""
import numpy as np
import pytest

from oracle import dft, gs, mraf, optics, project
from oracle.fft import fft2
from oracle.metrics import nmse
import synth

LAM, PITCH = 532e-9, 8e-6


def _window(h, w, y0, y1, x0, x1):
    m = np.zeros((h, w), dtype=bool)
    m[y0:y1, x0:x1] = True
    return m


@pytest.mark.parametrize("n_levels", [0, 2, 4])
@pytest.mark.parametrize("fresnel", [False, True])
@pytest.mark.parametrize("mix", [1.0, 0.6])
def test_full_signal_region_is_gs(n_levels, fresnel, mix):
    h_, w_ = 24, 30
    a = synth.blur_target(h_, w_, 2.0, seed=31).astype(np.float64)
    phi = synth.uniform_phase(h_, w_, seed=32).astype(np.float64)
    c = optics.chirp(h_, w_, LAM, PITCH, 0.05) if fresnel else None
    ref = gs.gs(a, phi, 5, n_levels, c)
    out = mraf.mraf(a, np.ones((h_, w_), dtype=bool), mix, phi, 5, n_levels, c)
    assert np.allclose(out["h"], ref["h"], atol=1e-10)
    if n_levels:
        assert np.array_equal(out["q"], ref["q"])
    assert np.allclose(out["nmse"], ref["nmse"], atol=1e-12)


@pytest.mark.parametrize("n_levels", [0, 4])
def test_empty_signal_region_keeps_the_hologram(n_levels):
    h_, w_ = 16, 20
    a = synth.blur_target(h_, w_, 2.0, seed=33).astype(np.float64)
    h0, _ = project.slm_project(np.exp(1j * synth.uniform_phase(h_, w_, seed=34).astype(np.float64)), n_levels)
    step = mraf.mraf_step(h0, a, np.zeros((h_, w_), dtype=bool), 0.3, n_levels)
    assert np.allclose(step["h"], h0, atol=1e-12)


def test_replacement_energy_bookkeeping():
    h_, w_ = 32, 32
    a = synth.blur_target(h_, w_, 2.0, seed=35).astype(np.float64)
    mask = _window(h_, w_, 4, 20, 6, 26)
    h0 = np.exp(1j * synth.uniform_phase(h_, w_, seed=36).astype(np.float64))
    mix = 0.7
    r = fft2(h0)
    r_new = mraf.mraf_step(h0, a, mask, mix)["r_new"]
    assert np.isclose(np.sum(np.abs(r_new[mask]) ** 2), mix * mix * h_ * w_, rtol=1e-12)
    assert np.isclose(np.sum(np.abs(r_new[~mask]) ** 2), (1 - mix) ** 2 * np.sum(np.abs(r[~mask]) ** 2), rtol=1e-12)


def test_one_step_by_explicit_dft():
    h_, w_ = 6, 8
    rng = np.random.default_rng(37)
    a = rng.random((h_, w_))
    mask = _window(h_, w_, 1, 5, 2, 7)
    h0 = np.exp(2j * np.pi * rng.random((h_, w_)))
    mix = 0.45
    step = mraf.mraf_step(h0, a, mask, mix)
    # the same step with the DFT matrices and the replacement written out element by element
    r = dft.dft2_bruteforce(h0)
    e = sum(a[y, x] ** 2 for y in range(h_) for x in range(w_) if mask[y, x])
    r_new = np.empty_like(r)
    for y in range(h_):
        for x in range(w_):
            if mask[y, x]:
                r_new[y, x] = mix * a[y, x] * np.sqrt(h_ * w_ / e) * r[y, x] / abs(r[y, x])
            else:
                r_new[y, x] = (1 - mix) * r[y, x]
    g = dft.dft2_bruteforce(r_new, inverse=True)
    assert np.allclose(step["g"], g, atol=1e-12)
    assert np.allclose(step["h"], g / np.abs(g), atol=1e-12)


def test_roi_nmse_properties():
    rng = np.random.default_rng(38)
    i, t = rng.random((12, 14)), rng.random((12, 14))
    full = np.ones((12, 14), dtype=bool)
    assert np.isclose(mraf.roi_nmse(i, t, full), nmse(i, t), rtol=1e-12)
    mask = _window(12, 14, 2, 9, 3, 12)
    i2, t2 = i.copy(), t.copy()
    i2[~mask] = 5.0
    t2[~mask] = -3.0
    assert mraf.roi_nmse(i, t, mask) == mraf.roi_nmse(i2, t2, mask)
    exact = np.where(mask, 2.5 * t, i)
    assert abs(mraf.roi_nmse(exact, t, mask)) < 1e-14


# ------------------------------------------------------------------ hybrid input-output


@pytest.mark.parametrize("n_levels", [0, 2, 4])
@pytest.mark.parametrize("fresnel", [False, True])
def test_hio_full_signal_region_is_gs(n_levels, fresnel):
    h_, w_ = 24, 30
    a = synth.blur_target(h_, w_, 2.0, seed=71).astype(np.float64)
    phi = synth.uniform_phase(h_, w_, seed=72).astype(np.float64)
    c = optics.chirp(h_, w_, LAM, PITCH, 0.05) if fresnel else None
    ref = gs.gs(a, phi, 5, n_levels, c)
    out = mraf.hio(a, np.ones((h_, w_), dtype=bool), 0.7, phi, 5, n_levels, c)
    assert np.allclose(out["h"], ref["h"], atol=1e-10)
    assert np.allclose(out["nmse"], ref["nmse"], atol=1e-12)


def test_hio_two_steps_by_explicit_dft():
    h_, w_ = 6, 8
    rng = np.random.default_rng(73)
    a = rng.random((h_, w_))
    mask = _window(h_, w_, 1, 4, 2, 6)
    phi0 = 2 * np.pi * rng.random((h_, w_))
    beta = 0.8
    out = mraf.hio(a, mask, beta, phi0, 2)
    # the same two iterations with the DFT matrices and the update written element by element
    e = sum(a[y, x] ** 2 for y in range(h_) for x in range(w_) if mask[y, x])
    a_s = a * np.sqrt(h_ * w_ / e)
    h = np.exp(1j * phi0)
    x_in = None
    for _ in range(2):
        y_out = dft.dft2_bruteforce(h)
        if x_in is None:
            x_in = y_out.copy()
        nxt = np.empty_like(y_out)
        for yy in range(h_):
            for xx in range(w_):
                if mask[yy, xx]:
                    nxt[yy, xx] = a_s[yy, xx] * y_out[yy, xx] / abs(y_out[yy, xx])
                else:
                    nxt[yy, xx] = x_in[yy, xx] - beta * y_out[yy, xx]
        x_in = nxt
        g = dft.dft2_bruteforce(x_in, inverse=True)
        h = g / np.abs(g)
    assert np.allclose(out["h"], h, atol=1e-12)


def test_hio_keeps_the_signal_region_constraint_and_feeds_back():
    """After one update the input equals A_s Y/|Y| on S and (1 - beta) Y_0 on N (X_0 = Y_0)."""
    h_, w_ = 16, 16
    a = synth.blur_target(h_, w_, 2.0, seed=74).astype(np.float64)
    mask = _window(h_, w_, 2, 9, 3, 11)
    phi0 = synth.uniform_phase(h_, w_, seed=75).astype(np.float64)
    beta = 0.6
    h1 = mraf.hio(a, mask, beta, phi0, 1)["h"]
    y0 = fft2(np.exp(1j * phi0))
    x1 = np.where(mask, mraf.signal_amplitude(a, mask) * y0 / np.abs(y0), (1 - beta) * y0)
    g = fft2(x1, inverse=True)
    assert np.allclose(h1, g / np.abs(g), atol=1e-12)
