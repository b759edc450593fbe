"""Pins of the direct-binary-search oracle (oracle.dbs) against the definitions it restates.

* the single-pixel replay update equals a full transform of the flipped hologram (Fourier and
  Fresnel), so the update is the replay of the hologram it claims to be;
* a sweep visits the pixels in row-major order and keeps exactly the flips that lower the NMSE
  (checked against a brute-force recomputation of every trial);
* the NMSE never increases from sweep to sweep, and a hologram on which a sweep keeps no flip is a
  local minimum: no single flip (recomputed by full transforms) lowers its NMSE;
* a hologram whose replay is the target (NMSE 0) is a fixed point; zero sweeps return the start.
"""
import numpy as np
import pytest

import synth
from oracle import dbs, optics
from oracle.fft import fft2
from oracle.metrics import nmse

LAM, PITCH = 532e-9, 8e-6


def _binary(h_, w_, seed):
    rng = np.random.default_rng(seed)
    return np.where(rng.random((h_, w_)) < 0.5, 1.0, -1.0)


@pytest.mark.parametrize("fresnel", [False, True])
def test_single_pixel_update_is_the_transform_of_the_flipped_hologram(fresnel):
    h_, w_ = 12, 10
    c = optics.chirp(h_, w_, LAM, PITCH, 0.02) if fresnel else None
    h = _binary(h_, w_, 1)
    r = fft2(h if c is None else h * c)
    for m, n in [(0, 0), (3, 7), (11, 9), (5, 0)]:
        h2 = h.copy()
        h2[m, n] = -h2[m, n]
        want = fft2(h2 if c is None else h2 * c)
        assert np.allclose(dbs.flip_update(r, h, m, n, c), want, atol=1e-12)


@pytest.mark.parametrize("fresnel", [False, True])
def test_sweep_keeps_exactly_the_improving_flips_in_row_major_order(fresnel):
    h_, w_ = 8, 6
    c = optics.chirp(h_, w_, LAM, PITCH, 0.02) if fresnel else None
    a = synth.blur_target(h_, w_, 1.0, seed=2).astype(np.float64)
    t = a * a
    h0 = _binary(h_, w_, 3)
    r0 = fft2(h0 if c is None else h0 * c)
    visits = []

    def record(p, e_old, e_new):
        visits.append(p)
        return e_new < e_old

    h1, r1, flipped = dbs.sweep(h0, r0, t, c, decide=record)
    assert visits == list(range(h_ * w_))
    # brute force: replay every trial with full transforms
    h = h0.copy()
    for p in range(h_ * w_):
        m, n = divmod(p, w_)
        e_old = nmse(np.abs(fft2(h if c is None else h * c)) ** 2, t)
        hf = h.copy()
        hf[m, n] = -hf[m, n]
        e_new = nmse(np.abs(fft2(hf if c is None else hf * c)) ** 2, t)
        assert flipped[m, n] == (e_new < e_old)
        if e_new < e_old:
            h = hf
    assert np.array_equal(h, h1)
    assert np.allclose(r1, fft2(h1 if c is None else h1 * c), atol=1e-10)


def test_nmse_non_increasing_and_converged_hologram_is_a_local_minimum():
    h_, w_ = 6, 8
    a = synth.blur_target(h_, w_, 1.0, seed=4).astype(np.float64)
    t = a * a
    phi0 = synth.uniform_phase(h_, w_, seed=5).astype(np.float64)
    out = dbs.dbs(a, phi0, 12)
    assert np.all(np.diff(out["nmse"]) <= 1e-15)
    # run sweeps until one keeps nothing, then check every single flip by full transforms
    h, r = dbs.start(phi0)
    for _ in range(50):
        h, r, flipped = dbs.sweep(h, r, t)
        if not flipped.any():
            break
    assert not flipped.any()
    e = nmse(np.abs(fft2(h)) ** 2, t)
    for m in range(h_):
        for n in range(w_):
            hf = h.copy()
            hf[m, n] = -hf[m, n]
            assert nmse(np.abs(fft2(hf)) ** 2, t) >= e


def test_reachable_target_is_a_fixed_point_and_zero_sweeps_return_the_start():
    h_, w_ = 8, 8
    hstar = _binary(h_, w_, 6)
    a = np.abs(fft2(hstar))
    phi0 = np.where(hstar > 0, 0.0, np.pi)
    out = dbs.dbs(a, phi0, 2)
    assert np.array_equal(out["h"], hstar)
    assert np.all(out["nmse"] < 1e-24)
    out0 = dbs.dbs(synth.blur_target(h_, w_, 1.0, seed=7), phi0, 0)
    assert np.array_equal(out0["h"], hstar) and out0["nmse"].shape == (1,)
    assert np.array_equal(out0["q"], (hstar < 0).astype(np.int64))


# ------------------------------------------------------------------ simulated annealing


def test_annealing_at_vanishing_temperature_is_dbs():
    h_, w_ = 8, 8
    a = synth.blur_target(h_, w_, 1.0, seed=8).astype(np.float64)
    phi0 = synth.uniform_phase(h_, w_, seed=9).astype(np.float64)
    ref = dbs.dbs(a, phi0, 3)
    out = dbs.sa(a, phi0, 3, 1e-300, 0.5, seed=10)
    assert np.array_equal(out["h"], ref["h"])
    assert np.allclose(out["nmse"], ref["nmse"], rtol=0, atol=0)


def test_annealing_at_huge_temperature_keeps_every_flip():
    h_, w_ = 6, 10
    a = synth.blur_target(h_, w_, 1.0, seed=11).astype(np.float64)
    phi0 = synth.uniform_phase(h_, w_, seed=12).astype(np.float64)
    h0, _ = dbs.start(phi0)
    out = dbs.sa(a, phi0, 1, 1e300, 1.0, seed=13)
    assert np.array_equal(out["h"], -h0)
    out2 = dbs.sa(a, phi0, 2, 1e300, 1.0, seed=13)
    assert np.array_equal(out2["h"], h0)


def test_annealing_rule_uses_the_pixel_and_sweep_draws():
    """The kept worsening flips of one sweep are exactly those whose draw u[p] lies below
    exp(-(E' - E) / T), recomputed here from full transforms."""
    h_, w_ = 6, 6
    a = synth.blur_target(h_, w_, 1.0, seed=14).astype(np.float64)
    t = a * a
    phi0 = synth.uniform_phase(h_, w_, seed=15).astype(np.float64)
    temp = 2e-3
    out = dbs.sa(a, phi0, 1, temp, 0.9, seed=16, item=3)
    from oracle.philox import anneal_uniform

    u = anneal_uniform(h_ * w_, 0, 3, 16)
    h, _ = dbs.start(phi0)
    for p in range(h_ * w_):
        m, n = divmod(p, w_)
        e_old = nmse(np.abs(fft2(h)) ** 2, t)
        hf = h.copy()
        hf[m, n] = -hf[m, n]
        e_new = nmse(np.abs(fft2(hf)) ** 2, t)
        if e_new < e_old or u[p] < np.exp(-(e_new - e_old) / temp):
            h = hf
    assert np.array_equal(h, out["h"])
    assert 0 < np.sum(out["h"] != dbs.start(phi0)[0]) < h_ * w_
