"""Pins for the oracle's algorithms: GS, multi-plane GS, OSPR (with Philox) and gradient descent.

* GS: Fienup's error-reduction property (the replay-amplitude error never increases, for every
  projection and for Fourier and Fresnel), the fixed point of an exactly reachable target, and one
  8x8 iteration by the explicit quadruple DFT sum.
* Multi-plane GS: P = 1 reduces to GS; the product-space error never increases.
* OSPR: Philox known-answer vectors, Hermitian replay of a real hologram, bit packing, the NMSE trend
  over subframes.
* GD: central finite differences of the loss, an independent float64 autograd of the same loss
  (library, test only), Adam against torch.optim.Adam.
"""
import os

import numpy as np
import pytest

from oracle import dft, gd, gs, optics, ospr, philox, project
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LAM, PITCH = 532e-9, 8e-6


# ------------------------------------------------------------------ GS


@pytest.mark.parametrize("n_levels", [0, 2, 4, 8])
@pytest.mark.parametrize("fresnel", [False, True])
def test_gs_error_reduction(n_levels, fresnel):
    h_, w_ = 32, 40
    a = synth.blur_target(h_, w_, 1.5, seed=21).astype(np.float64)
    c = optics.chirp(h_, w_, LAM, PITCH, 0.02) if fresnel else None
    phi0 = synth.uniform_phase(h_, w_, seed=22).astype(np.float64)
    h, _ = project.slm_project(np.exp(1j * phi0), n_levels)
    errs = [gs.replay_error(h, a, c)]
    for _ in range(25):
        h = gs.gs_step(h, a, n_levels, c)["h"]
        errs.append(gs.replay_error(h, a, c))
    e = np.array(errs)
    assert np.all(e[1:] <= e[:-1] * (1 + 1e-12)), e
    assert e[-1] < e[0]


def test_gs_run_matches_step_chain_and_curve():
    a = synth.blur_target(16, 24, 2.0, seed=3).astype(np.float64)
    phi0 = synth.uniform_phase(16, 24, seed=4).astype(np.float64)
    out = gs.gs(a, phi0, 6, n_levels=4)
    h, _ = project.slm_project(np.exp(1j * phi0), 4)
    from oracle.fft import fft2
    from oracle.metrics import nmse
    for k in range(6):
        assert abs(out["nmse"][k] - nmse(np.abs(fft2(h)) ** 2, a * a)) < 1e-14
        h = gs.gs_step(h, a, 4)["h"]
    np.testing.assert_allclose(out["h"], h, atol=0)


@pytest.mark.parametrize("n_levels", [0, 4])
def test_gs_fixed_point(n_levels):
    r = np.random.default_rng(31)
    if n_levels:
        hstar = project.level_field(r.integers(0, n_levels, (24, 16)), n_levels)
    else:
        hstar = np.exp(2j * np.pi * r.random((24, 16)))
    from oracle.fft import fft2
    a = np.abs(fft2(hstar))
    out = gs.gs(a, project.phase_of(hstar), 5, n_levels=n_levels)
    np.testing.assert_allclose(out["h"], hstar, atol=1e-12)
    assert np.max(out["nmse"]) < 1e-24


def test_gs_one_iteration_bruteforce_8x8():
    a = synth.blur_target(8, 8, 1.0, seed=5).astype(np.float64)
    phi0 = synth.uniform_phase(8, 8, seed=6).astype(np.float64)
    h0 = np.exp(1j * phi0)
    r = dft.dft2_bruteforce(h0)
    a_s = a * np.sqrt(64 / np.sum(a * a))
    rp = a_s * r / np.abs(r)
    g = dft.dft2_bruteforce(rp, inverse=True)
    want = g / np.abs(g)
    np.testing.assert_allclose(gs.gs_step(h0, a, 0)["h"], want, atol=1e-13)


# ------------------------------------------------------------------ multi-plane GS


def test_multiplane_p1_equals_gs():
    a = synth.spots_target(32, 32, 6, seed=41).astype(np.float64)
    phi0 = synth.uniform_phase(32, 32, seed=42).astype(np.float64)
    c = optics.chirp(32, 32, LAM, PITCH, 0.05)
    m = gs.multiplane_gs([a], phi0, 5, [c], n_levels=0)
    s = gs.gs(a, phi0, 5, n_levels=0, c=c)
    np.testing.assert_allclose(m["h"], s["h"], atol=1e-12)
    np.testing.assert_allclose(m["nmse"], s["nmse"], atol=1e-13)


def test_multiplane_error_reduction():
    n = 32
    amps = [synth.spots_target(n, n, 6, seed=s).astype(np.float64) for s in (51, 52, 53)]
    cs = [optics.chirp(n, n, LAM, PITCH, z) for z in (0.02, 0.03, 0.04)]
    phi0 = synth.uniform_phase(n, n, seed=54).astype(np.float64)
    h = np.exp(1j * phi0)
    errs = [gs.multiplane_error(h, amps, cs)]
    for _ in range(15):
        h = gs.multiplane_gs(amps, project.phase_of(h), 1, cs)["h"]
        errs.append(gs.multiplane_error(h, amps, cs))
    e = np.array(errs)
    assert np.all(e[1:] <= e[:-1] * (1 + 1e-12)), e


# ------------------------------------------------------------------ Philox / OSPR


def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        v = [int(x, 16) for x in row]
        out = philox.philox4x32_10(tuple(v[0:4]), tuple(v[4:6]))
        assert [int(o) for o in out] == v[6:10]


def test_ospr_uniform_properties():
    u = philox.ospr_uniform(1 << 16, 3, 2, 1234)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2**24 == np.floor(u * 2**24))
    assert abs(u.mean() - 0.5) < 0.01
    # distinct subframes and targets give different draws
    assert not np.array_equal(u, philox.ospr_uniform(1 << 16, 4, 2, 1234))
    assert not np.array_equal(u, philox.ospr_uniform(1 << 16, 3, 3, 1234))


def test_bit_pack_roundtrip():
    q = np.random.default_rng(3).integers(0, 2, (7, 70))
    w = ospr.pack_bits(q)
    assert w.shape == (7, 3) and w.dtype == np.uint32
    assert np.array_equal(ospr.unpack_bits(w, 70), q)
    # LSB-first: pixel 0 is bit 0 of word 0
    q1 = np.zeros((1, 40), dtype=np.int64)
    q1[0, 0] = 1
    q1[0, 33] = 1
    assert list(ospr.pack_bits(q1)[0]) == [1, 2]


def test_ospr_replay_is_hermitian():
    a = synth.symmetrise(synth.blur_target(24, 30, 2.0, seed=61)).astype(np.float64)
    sf = ospr.ospr_subframe(a, 0, 0, 77)
    i = sf["intensity"]
    i_neg = np.roll(i[::-1, ::-1], (1, 1), axis=(0, 1))
    np.testing.assert_allclose(i, i_neg, rtol=1e-12, atol=1e-12 * i.max())
    assert set(np.unique(sf["h"].real)) <= {-1.0, 1.0}


def test_ospr_nmse_falls_with_subframes():
    curves = []
    for t in range(3):
        a = synth.symmetrise(synth.blur_target(32, 32, 2.0, seed=70 + t)).astype(np.float64)
        curves.append(ospr.ospr(a, 16, t, 3000)["nmse"])
    c = np.mean(curves, axis=0)
    assert c[15] < c[3] < c[0]


def _binarise_by_hand(g):
    """Nearest of {+1, -1}: -1 where Re g < 0, and on Re g == 0 where Im g > 0 (the tie rule)."""
    q = ((g.real < 0.0) | ((g.real == 0.0) & (g.imag > 0.0))).astype(np.int64)
    return 1.0 - 2.0 * q, q


def _ospr_subframe_by_hand(a, subframe, target, seed, c=None):
    """One classic OSPR subframe written out with the explicit quadruple DFT sum: theta = 2 pi u
    (u from the Philox generator pinned by its known-answer vectors), A_s = A sqrt(HW / sum A^2),
    g = conj(c) F^-1(A_s e^{i theta}), h = binary(g), I = |F(h c)|^2."""
    hh, ww = a.shape
    u = philox.ospr_uniform(hh * ww, subframe, target, seed).reshape(hh, ww)
    a_s = a * np.sqrt(hh * ww / np.sum(a * a))
    g = dft.dft2_bruteforce(a_s * np.exp(2j * np.pi * u), inverse=True)
    if c is not None:
        g = np.conj(c) * g
    h, q = _binarise_by_hand(g)
    r = dft.dft2_bruteforce(h if c is None else h * c)
    return h, q, g, np.abs(r) ** 2


@pytest.mark.parametrize("fresnel", [False, True])
def test_ospr_subframe_by_explicit_dft(fresnel):
    # unsymmetrised, non-square target: a forward transform in place of F^-1, theta = pi u, or A^2 in
    # place of A change the bits here (a symmetrised target would hide the transform direction)
    hh, ww = 6, 10
    a = np.random.default_rng(401).uniform(0.1, 1.0, (hh, ww))
    c = optics.chirp(hh, ww, LAM, PITCH, 0.01) if fresnel else None
    for s, t, seed in ((0, 0, 77), (3, 2, 2**40 + 5)):
        h, q, g, inten = _ospr_subframe_by_hand(a, s, t, seed, c)
        sf = ospr.ospr_subframe(a, s, t, seed, 0, c)
        assert np.array_equal(sf["q"], q)
        np.testing.assert_array_equal(sf["h"], h)
        np.testing.assert_allclose(sf["g"], g, rtol=0, atol=1e-12 * np.abs(g).max())
        np.testing.assert_allclose(sf["intensity"], inten, rtol=0, atol=1e-12 * inten.max())
    # the pin has power: each of these misreadings flips some bits on this input
    u = philox.ospr_uniform(hh * ww, 0, 0, 77).reshape(hh, ww)
    a_s = a * np.sqrt(hh * ww / np.sum(a * a))
    _, q_ok, _, _ = _ospr_subframe_by_hand(a, 0, 0, 77, c)
    wrong = [dft.dft2_bruteforce(a_s * np.exp(2j * np.pi * u)),               # forward transform
             dft.dft2_bruteforce(a_s * np.exp(1j * np.pi * u), inverse=True),  # theta = pi u
             dft.dft2_bruteforce(a_s ** 2 * np.exp(2j * np.pi * u), inverse=True)]  # A^2 for A
    for gw in wrong:
        gw = gw if c is None else np.conj(c) * gw
        assert not np.array_equal(_binarise_by_hand(gw)[1], q_ok)


@pytest.mark.parametrize("fresnel", [False, True])
def test_ospr_refinement_is_binary_gs_chain(fresnel):
    # n_iter > 0: the subframe's start followed by n_iter binary GS iterations against A
    hh, ww = 8, 12
    a = np.random.default_rng(402).uniform(0.1, 1.0, (hh, ww))
    c = optics.chirp(hh, ww, LAM, PITCH, 0.01) if fresnel else None
    h0, _, _, _ = _ospr_subframe_by_hand(a, 1, 4, 99, c)
    for n_iter in (1, 3):
        h = h0
        for _ in range(n_iter):
            st = gs.gs_step(h, a, 2, c)
            h, q = st["h"], st["q"]
        sf = ospr.ospr_subframe(a, 1, 4, 99, n_iter, c)
        np.testing.assert_array_equal(sf["h"], h)
        assert np.array_equal(sf["q"], q)
        r = dft.dft2_bruteforce(h if c is None else h * c)
        np.testing.assert_allclose(sf["intensity"], np.abs(r) ** 2, rtol=0,
                                   atol=1e-12 * sf["intensity"].max())


def test_ospr_accumulated_nmse_by_hand():
    # nmse[s] is the optimal-scale NMSE of the mean replay intensity of subframes 0..s against A^2,
    # here from brute-force intensities and the closed form 1 - (sum I T)^2 / (sum I^2 sum T^2)
    hh, ww = 6, 8
    a = np.random.default_rng(403).uniform(0.1, 1.0, (hh, ww))
    out = ospr.ospr(a, 4, 7, 31)
    t = a * a
    acc = np.zeros_like(t)
    for s in range(4):
        _, q, _, inten = _ospr_subframe_by_hand(a, s, 7, 31)
        assert np.array_equal(out["q"][s], q)
        assert np.array_equal(ospr.unpack_bits(out["bits"][s], ww), q)
        acc += inten
        i = acc / (s + 1)
        want = 1.0 - np.sum(i * t) ** 2 / (np.sum(i * i) * np.sum(t * t))
        assert abs(out["nmse"][s] - want) <= 1e-12
    np.testing.assert_allclose(out["i_acc"], acc, rtol=0, atol=1e-12 * acc.max())


def test_ospr_bits_match_levels():
    a = synth.symmetrise(synth.blur_target(16, 40, 2.0, seed=81)).astype(np.float64)
    out = ospr.ospr(a, 3, 1, 5, n_iter=2)
    for s in range(3):
        assert np.array_equal(ospr.unpack_bits(out["bits"][s], 40), out["q"][s])


# ------------------------------------------------------------------ GD


def _gd_problem(n=64, seed=90):
    ts = [synth.spots_target(n, n, 8, seed=seed + p).astype(np.float64) ** 2 for p in range(3)]
    ts = [t / np.sqrt(np.sum(t * t)) for t in ts]
    cs = [optics.chirp(n, n, LAM, PITCH, z) for z in (0.08, 0.10, 0.12)]
    phi = synth.uniform_phase(n, n, seed=seed + 9).astype(np.float64)
    return phi, ts, cs


def test_gd_gradient_finite_differences():
    phi, ts, cs = _gd_problem()
    _, _, g = gd.loss_and_grad(phi, ts, cs)
    r = np.random.default_rng(5)
    idx = r.choice(phi.size, 48, replace=False)
    eps = 1e-6
    fd = []
    for k in idx:
        e = np.zeros(phi.size)
        e[k] = eps
        e = e.reshape(phi.shape)
        fd.append((gd.loss_only(phi + e, ts, cs) - gd.loss_only(phi - e, ts, cs)) / (2 * eps))
    fd = np.array(fd)
    assert np.linalg.norm(fd - g.ravel()[idx]) / np.linalg.norm(fd) < 1e-6
    # directional derivative over all pixels at once
    v = r.standard_normal(phi.shape)
    t = 1e-6
    dfd = (gd.loss_only(phi + t * v, ts, cs) - gd.loss_only(phi - t * v, ts, cs)) / (2 * t)
    assert abs(dfd - np.sum(g * v)) / abs(dfd) < 1e-6


def test_gd_gradient_vs_float64_autograd():
    torch = pytest.importorskip("torch")
    phi, ts, cs = _gd_problem(n=48, seed=95)
    _, lp, g = gd.loss_and_grad(phi, ts, cs)
    tp = torch.tensor(phi, dtype=torch.float64, requires_grad=True)
    h = torch.exp(1j * tp.to(torch.complex128))
    losses = []
    for t, c in zip(ts, cs):
        u = torch.fft.fft2(h * torch.tensor(c), norm="ortho")
        i = u.real**2 + u.imag**2
        tt = torch.tensor(t)
        s = (i * tt).sum() / (i * i).sum()
        s = s.detach()  # the optimal scale is held fixed (envelope theorem)
        losses.append(((s * i - tt) ** 2).sum() / (tt * tt).sum())
    loss = torch.stack(losses).mean()
    loss.backward()
    assert abs(loss.item() - np.mean(lp)) < 1e-12
    np.testing.assert_allclose(tp.grad.numpy(), g, rtol=0, atol=1e-10 * np.abs(g).max())


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(8)
    phi = r.random((6, 5))
    m = np.zeros_like(phi)
    v = np.zeros_like(phi)
    tp = torch.tensor(phi, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=0.05, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 6):
        g = r.standard_normal(phi.shape)
        phi, m, v = gd.adam_update(phi, g, m, v, step, 0.05)
        opt.zero_grad()
        tp.grad = torch.tensor(g)
        opt.step()
        np.testing.assert_allclose(tp.detach().numpy(), phi, rtol=0, atol=1e-14)


def test_gd_decreases_loss():
    phi, ts, cs = _gd_problem(n=32, seed=99)
    out = gd.gd_run(phi, ts, cs, 30, 0.05)
    assert out["loss"][-1] < 0.5 * out["loss"][0]


# ------------------------------------------------------------------ GS under an illumination profile


def _gaussian_beam(h, w, waist):
    y = np.arange(h) - (h - 1) / 2
    x = np.arange(w) - (w - 1) / 2
    return np.exp(-(y[:, None] ** 2 + x[None, :] ** 2) / (2 * waist ** 2))


@pytest.mark.parametrize("n_levels", [0, 2, 4])
def test_gs_unit_illumination_is_gs(n_levels):
    a = synth.blur_target(20, 24, 2.0, seed=51).astype(np.float64)
    phi0 = synth.uniform_phase(20, 24, seed=52).astype(np.float64)
    ref = gs.gs(a, phi0, 5, n_levels)
    out = gs.gs(a, phi0, 5, n_levels, illum=np.ones((20, 24)))
    np.testing.assert_array_equal(out["h"], ref["h"])
    np.testing.assert_array_equal(out["nmse"], ref["nmse"])


@pytest.mark.parametrize("n_levels", [0, 4])
def test_gs_constant_illumination_keeps_the_phases(n_levels):
    a = synth.blur_target(20, 24, 2.0, seed=53).astype(np.float64)
    phi0 = synth.uniform_phase(20, 24, seed=54).astype(np.float64)
    ref = gs.gs(a, phi0, 5, n_levels)
    out = gs.gs(a, phi0, 5, n_levels, illum=np.full((20, 24), 0.37))
    assert np.allclose(out["h"], 0.37 * ref["h"], atol=1e-12)
    assert np.allclose(out["nmse"], ref["nmse"], atol=1e-12)


@pytest.mark.parametrize("n_levels", [0, 2, 8])
@pytest.mark.parametrize("fresnel", [False, True])
def test_gs_error_reduction_under_gaussian_illumination(n_levels, fresnel):
    h_, w_ = 32, 40
    a = synth.blur_target(h_, w_, 1.5, seed=55).astype(np.float64)
    illum = _gaussian_beam(h_, w_, 9.0)
    c = optics.chirp(h_, w_, LAM, PITCH, 0.02) if fresnel else None
    h, _ = project.slm_project(np.exp(1j * synth.uniform_phase(h_, w_, seed=56).astype(np.float64)), n_levels)
    h = illum * h
    errs = [gs.replay_error(h, a, c, illum)]
    for _ in range(25):
        step = gs.gs_step(h, a, n_levels, c, illum)
        h = step["h"]
        assert np.allclose(np.abs(h), illum, atol=1e-12)
        errs.append(gs.replay_error(h, a, c, illum))
    e = np.array(errs)
    assert np.all(e[1:] <= e[:-1] * (1 + 1e-12)), e
    assert e[-1] < e[0]
