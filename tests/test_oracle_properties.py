"""Randomised property checks of the oracle pieces added for the search and region variants (CPU
only).  Each property is a definition or identity, checked on seeded random shapes and values (the
draws come from numpy's PCG64, so every machine runs the same cases): the single-pixel replay update
is the transform of the flipped hologram, the table projection is a nearest point with the
lowest-index tie rule, MRAF with m = 1 and HIO with the whole plane as signal region are GS, and an
annealing rule never rejects an improving flip."""
import numpy as np
import pytest

from oracle import dbs, gs, mraf, project
from oracle.fft import fft2

SIZES = [2, 3, 4, 5, 6, 8, 9, 10, 12]


@pytest.mark.parametrize("case", range(40))
def test_flip_update_is_the_flipped_transform(case):
    rng = np.random.default_rng(7000 + case)
    h, w = int(rng.choice(SIZES)), int(rng.choice(SIZES))
    fresnel = bool(rng.integers(2))
    hol = np.where(rng.random((h, w)) < 0.5, 1.0, -1.0)
    c = np.exp(2j * np.pi * rng.random((h, w))) if fresnel else None
    r = fft2(hol if c is None else hol * c)
    m, n = int(rng.integers(h)), int(rng.integers(w))
    flipped = hol.copy()
    flipped[m, n] = -flipped[m, n]
    want = fft2(flipped if c is None else flipped * c)
    assert np.allclose(dbs.flip_update(r, hol, m, n, c), want, atol=1e-12)


@pytest.mark.parametrize("case", range(60))
def test_table_projection_is_a_nearest_point(case):
    rng = np.random.default_rng(8000 + case)
    n_pix, n_tab = int(rng.integers(1, 41)), int(rng.integers(2, 10))
    table = rng.standard_normal(n_tab) + 1j * rng.standard_normal(n_tab)
    table[rng.integers(n_tab)] = table[0]  # a repeated value: the lower index must win
    g = rng.standard_normal(n_pix) + 1j * rng.standard_normal(n_pix)
    h, q = project.table_project(g, table)
    d = np.abs(g[:, None] - table[None, :])
    assert np.all(np.abs(g - h) <= d.min(axis=1) + 1e-15)
    assert np.array_equal(q, np.argmin(d, axis=1))  # argmin returns the first of equal minima


@pytest.mark.parametrize("case", range(15))
def test_region_variants_with_the_whole_plane_are_gs(case):
    rng = np.random.default_rng(9000 + case)
    h, w = int(rng.choice([4, 6, 8])), int(rng.choice([4, 6, 8]))
    levels = int(rng.choice([0, 2, 4]))
    beta = float(rng.uniform(0.1, 1.9))
    a = rng.random((h, w)) + 0.1
    phi = 2 * np.pi * rng.random((h, w))
    ref = gs.gs(a, phi, 3, levels)
    whole = np.ones((h, w), dtype=bool)
    for out in (mraf.mraf(a, whole, 1.0, phi, 3, levels), mraf.hio(a, whole, beta, phi, 3, levels)):
        assert np.allclose(out["nmse"], ref["nmse"], atol=1e-12)
        if levels:
            assert np.array_equal(out["q"], ref["q"])
        else:
            assert np.allclose(out["h"], ref["h"], atol=1e-10)


@pytest.mark.parametrize("case", range(50))
def test_annealing_rule_keeps_every_improving_flip(case):
    rng = np.random.default_rng(10000 + case)
    e_old, de = float(rng.uniform(0.0, 1.0)), float(rng.uniform(-0.5, 0.5))
    u, temp = float(rng.uniform(0.0, 0.999999)), float(np.exp(rng.uniform(np.log(1e-6), np.log(10.0))))
    if case == 0:
        de = 0.0  # a flip that leaves the NMSE unchanged: kept iff u < exp(0) = 1
    rule = dbs.metropolis(np.array([u]), temp)
    keep = rule(0, e_old, e_old + de)
    if de < 0:
        assert keep
    else:
        assert keep == (u < np.exp(-de / temp))
