"""Randomised property checks of the oracle pieces added for the search and region variants
(hypothesis; CPU only).  Each property is a definition or identity, checked on random shapes and
values: the single-pixel replay update is the transform of the flipped hologram, the table
projection is a nearest point with the lowest-index tie rule, MRAF with m = 1 and HIO with the whole
plane as signal region are GS, and an annealing rule never rejects an improving flip."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from oracle import dbs, gs, mraf, project  # noqa: E402
from oracle.fft import fft2  # noqa: E402

SIZES = st.sampled_from([2, 3, 4, 5, 6, 8, 9, 10, 12])


@settings(max_examples=40, deadline=None)
@given(h=SIZES, w=SIZES, seed=st.integers(0, 2**31 - 1), fresnel=st.booleans())
def test_flip_update_is_the_flipped_transform(h, w, seed, fresnel):
    rng = np.random.default_rng(seed)
    hol = np.where(rng.random((h, w)) < 0.5, 1.0, -1.0)
    c = np.exp(2j * np.pi * rng.random((h, w))) if fresnel else None
    r = fft2(hol if c is None else hol * c)
    m, n = int(rng.integers(h)), int(rng.integers(w))
    flipped = hol.copy()
    flipped[m, n] = -flipped[m, n]
    want = fft2(flipped if c is None else flipped * c)
    assert np.allclose(dbs.flip_update(r, hol, m, n, c), want, atol=1e-12)


@settings(max_examples=60, deadline=None)
@given(n_pix=st.integers(1, 40), n_tab=st.integers(2, 9), seed=st.integers(0, 2**31 - 1))
def test_table_projection_is_a_nearest_point(n_pix, n_tab, seed):
    rng = np.random.default_rng(seed)
    table = rng.standard_normal(n_tab) + 1j * rng.standard_normal(n_tab)
    table[rng.integers(n_tab)] = table[0]  # a repeated value: the lower index must win
    g = rng.standard_normal(n_pix) + 1j * rng.standard_normal(n_pix)
    h, q = project.table_project(g, table)
    d = np.abs(g[:, None] - table[None, :])
    assert np.all(np.abs(g - h) <= d.min(axis=1) + 1e-15)
    assert np.array_equal(q, np.argmin(d, axis=1))  # argmin returns the first of equal minima


@settings(max_examples=15, deadline=None)
@given(h=st.sampled_from([4, 6, 8]), w=st.sampled_from([4, 6, 8]), seed=st.integers(0, 2**31 - 1),
       levels=st.sampled_from([0, 2, 4]), beta=st.floats(0.1, 1.9))
def test_region_variants_with_the_whole_plane_are_gs(h, w, seed, levels, beta):
    rng = np.random.default_rng(seed)
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


@settings(max_examples=50, deadline=None)
@given(e_old=st.floats(0.0, 1.0), de=st.floats(-0.5, 0.5), u=st.floats(0.0, 0.999999),
       temp=st.floats(1e-6, 10.0))
def test_annealing_rule_keeps_every_improving_flip(e_old, de, u, temp):
    rule = dbs.metropolis(np.array([u]), temp)
    keep = rule(0, e_old, e_old + de)
    if de < 0:
        assert keep
    else:
        assert keep == (u < np.exp(-de / temp))
