"""Pins of the multi-amplitude / complex-modulation SLM projection (oracle.project.table_project)
and of GS, MRAF and HIO run with it.

* the projection is the nearest table entry (explicit loops over pixels and entries), the lowest
  index on a tie;
* a table of N unit values at equal angles reproduces the N-level phase quantiser;
* GS under a multi-amplitude table keeps Fienup's error reduction (nearest-point projections on
  both sides, unitary transforms), Fourier and Fresnel;
* MRAF and HIO with the whole plane as signal region reduce to GS under the same table.
"""
import numpy as np
import pytest

import synth
from oracle import gs, mraf, optics, project

LAM, PITCH = 532e-9, 8e-6
# 2 amplitudes x 4 phases, and a 3-entry table with a zero level
TABLE8 = np.array([a * np.exp(1j * np.pi / 2 * k) for a in (0.5, 1.0) for k in range(4)])
TABLE3 = np.array([0.0, 1.0, np.exp(2j * np.pi / 3) * 0.8])


@pytest.mark.parametrize("table", [TABLE8, TABLE3])
def test_table_projection_is_the_nearest_entry(table):
    rng = np.random.default_rng(1)
    g = (rng.standard_normal((7, 9)) + 1j * rng.standard_normal((7, 9))) * 0.8
    h, q = project.table_project(g, table)
    for y in range(7):
        for x in range(9):
            d = [abs(g[y, x] - m) for m in table]
            best = min(d)
            assert q[y, x] == d.index(best)
            assert h[y, x] == table[q[y, x]]


def test_table_projection_ties_take_the_lowest_index():
    table = np.array([1.0, -1.0, 1j])
    h, q = project.table_project(np.array([0.0, 1j * 1e-300, -0.5 + 0.5j]), table)
    assert q.tolist()[0] == 0            # equidistant from all three
    assert q.tolist()[2] in (1, 2) and q.tolist()[2] == 1  # equidistant from -1 and i


@pytest.mark.parametrize("n", [2, 3, 4, 8])
def test_unit_circle_table_is_the_phase_quantiser(n):
    rng = np.random.default_rng(n)
    g = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    table = project.level_field(np.arange(n), n)
    _, q_t = project.table_project(g, table)
    _, q_n = project.slm_project(g, n)
    assert np.array_equal(q_t, q_n)


@pytest.mark.parametrize("fresnel", [False, True])
def test_gs_with_a_table_reduces_the_replay_error(fresnel):
    h_, w_ = 24, 20
    a = synth.blur_target(h_, w_, 2.0, seed=3).astype(np.float64)
    phi = synth.uniform_phase(h_, w_, seed=4).astype(np.float64)
    c = optics.chirp(h_, w_, LAM, PITCH, 0.02) if fresnel else None
    out = gs.gs(a, phi, 0, TABLE8, c)
    h = out["h"]
    errs = []
    for _ in range(12):
        errs.append(gs.replay_error(h, a, c))
        h = gs.gs_step(h, a, TABLE8, c)["h"]
    assert np.all(np.diff(errs) <= 1e-9 * errs[0])
    assert set(np.unique(np.round(h, 12))) <= set(np.round(TABLE8, 12))


def test_region_variants_with_the_whole_plane_are_gs_under_a_table():
    h_, w_ = 16, 24
    a = synth.blur_target(h_, w_, 2.0, seed=5).astype(np.float64)
    phi = synth.uniform_phase(h_, w_, seed=6).astype(np.float64)
    ref = gs.gs(a, phi, 5, TABLE8)
    whole = np.ones((h_, w_), dtype=bool)
    for out in (mraf.mraf(a, whole, 1.0, phi, 5, TABLE8), mraf.hio(a, whole, 0.7, phi, 5, TABLE8)):
        assert np.allclose(out["h"], ref["h"], atol=1e-10)
        assert np.allclose(out["nmse"], ref["nmse"], atol=1e-12)
