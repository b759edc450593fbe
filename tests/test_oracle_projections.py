"""Pins for the oracle's SLM projection, amplitude replacement and NMSE.

Brute-force nearest level by angular distance over every level, explicit tie cases, idempotence,
exact level sets, and a hand-computed NMSE.
"""
import os

import numpy as np
import pytest

from oracle import metrics, project

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_c(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


@pytest.mark.parametrize("n_levels", [2, 3, 4, 5, 8, 16])
def test_quantise_is_nearest_level(n_levels):
    g = _rand_c((4000,), n_levels)
    q = project.quantise_index(g, n_levels)
    levels = 2 * np.pi * np.arange(n_levels) / n_levels
    a = np.mod(np.angle(g), 2 * np.pi)
    dist = np.abs(np.angle(np.exp(1j * (a[:, None] - levels[None, :]))))  # wrapped |a - phi_k|
    best = np.argmin(dist, axis=1)
    # away from ties the nearest level is unique
    sorted_d = np.sort(dist, axis=1)
    clear = (sorted_d[:, 1] - sorted_d[:, 0]) > 1e-9
    assert np.array_equal(q[clear], best[clear])
    # and the projection minimises |h - g / |g|| over the level set
    h, _ = project.slm_project(g, n_levels)
    u = g / np.abs(g)
    cand = np.exp(1j * levels)[None, :]
    assert np.all(np.abs(h - u) <= np.min(np.abs(cand - u[:, None]), axis=1) + 1e-12)


def test_quantise_ties_and_zero():
    # binary: Re g = 0 -> Im > 0 goes to pi (q = 1), Im < 0 goes to 0
    g = np.array([1j, -1j, 0.0, -1.0, 1.0, complex(-1.0, -0.0)])
    q = project.quantise_index(g, 2)
    assert list(q) == [1, 0, 0, 1, 0, 1]
    # 4 levels: exact midpoints pi/4 and 3 pi/4 go to the higher index
    g4 = np.array([1 + 1j, -1 + 1j, -1 - 1j, 1 - 1j])
    assert list(project.quantise_index(g4, 4)) == [1, 2, 3, 0]
    # zero field: continuous -> 1, quantised -> level 0
    h, _ = project.slm_project(np.zeros(3, dtype=complex), 0)
    assert np.all(h == 1.0)
    h, q = project.slm_project(np.zeros(3, dtype=complex), 8)
    assert np.all(q == 0) and np.all(h == 1.0)


@pytest.mark.parametrize("n_levels", [0, 2, 4, 8])
def test_projection_idempotent_and_exact_levels(n_levels):
    g = _rand_c((50, 30), 3) * 3.7
    h, q = project.slm_project(g, n_levels)
    h2, q2 = project.slm_project(h, n_levels)
    np.testing.assert_allclose(np.abs(h), 1.0, atol=1e-15)
    if n_levels == 0:
        np.testing.assert_allclose(h2, h, atol=1e-15)
    else:
        assert np.array_equal(q2, q)
        level_set = project.level_field(np.arange(n_levels), n_levels)
        assert np.all(np.min(np.abs(h.ravel()[:, None] - level_set[None, :]), axis=1) == 0.0)
    if n_levels == 2:
        assert set(np.unique(h.real)) <= {-1.0, 1.0} and np.all(h.imag == 0.0)
    if n_levels == 4:
        assert set(np.unique(np.round(h * 1.0, 0))) <= {1, 1j, -1, -1j}


def test_amplitude_replacement():
    r = _rand_c((20, 20), 5)
    r[3, 4] = 0.0
    a = np.random.default_rng(9).random((20, 20))
    out = project.amplitude_replace(r, a)
    np.testing.assert_allclose(np.abs(out), a, atol=1e-14)
    mask = np.abs(r) > 0
    np.testing.assert_allclose(np.angle(out[mask]), np.angle(r[mask]), atol=1e-12)
    assert out[3, 4] == a[3, 4]


def _golden_nmse():
    vals = {}
    with open(os.path.join(GOLDEN, "nmse_hand.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            vals[k] = np.array([float(x) for x in v])
    return vals


def test_nmse_hand_computed():
    g = _golden_nmse()
    i = g["I"].reshape(2, 2)
    t = g["T"].reshape(2, 2)
    assert abs(metrics.optimal_scale(i, t) - g["scale"][0]) < 1e-15
    assert abs(metrics.nmse(i, t) - g["nmse"][0]) < 1e-15


def test_nmse_identities():
    r = np.random.default_rng(4)
    t = r.random((32, 32))
    assert metrics.nmse(3.5 * t, t) < 1e-28
    i = r.random((32, 32))
    rho2 = np.sum(i * t) ** 2 / (np.sum(i * i) * np.sum(t * t))
    assert abs(metrics.nmse(i, t) - (1.0 - rho2)) < 1e-14
    # scale invariance in I
    assert abs(metrics.nmse(7.0 * i, t) - metrics.nmse(i, t)) < 1e-14
