"""Pins for the oracle's transforms: naive DFT, own Stockham FFT and Fresnel propagation.

Each check is tied to something other than the oracle itself: hand-computed DFTs, closed forms
(delta, plane wave, the transform of a chirped Gaussian), the explicit quadruple DFT sum, Parseval,
and -- test only -- numpy's own FFT in float64.
"""
import os

import numpy as np
import pytest

from oracle import dft, fft, optics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_c(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b))


def _golden_dft():
    out = {}
    with open(os.path.join(GOLDEN, "dft_hand.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            case, idx, re, im = line.split()
            out.setdefault(case, {})[int(idx)] = complex(float(re), float(im))
    return out


def test_dft_hand_computed():
    g = _golden_dft()
    x = np.array([1, 2, 3, 4], dtype=np.complex128)
    want = np.array([g["dft1_4"][k] for k in range(4)])
    np.testing.assert_allclose(dft.dft1(x), want, atol=1e-13)
    np.testing.assert_allclose(fft.fft1(x), want, atol=1e-13)
    x2 = np.array([[1, 2], [3, 4]], dtype=np.complex128)
    want2 = np.array([g["dft2_2x2"][k] for k in range(4)]).reshape(2, 2) / 2.0  # unitary: /sqrt(4)
    np.testing.assert_allclose(dft.dft2(x2), want2, atol=1e-13)
    np.testing.assert_allclose(fft.fft2(x2), want2, atol=1e-13)


@pytest.mark.parametrize("hw", [(8, 8), (6, 10), (5, 7)])
def test_delta_and_plane_wave(hw):
    h, w = hw
    d = np.zeros((h, w), dtype=np.complex128)
    d[0, 0] = 1.0
    for f2 in (dft.dft2, fft.fft2):
        np.testing.assert_allclose(f2(d), np.full((h, w), 1.0 / np.sqrt(h * w)), atol=1e-14)
    k0, l0 = h - 2, 1
    m = np.arange(h)[:, None]
    n = np.arange(w)[None, :]
    pw = np.exp(2j * np.pi * (k0 * m / h + l0 * n / w))
    want = np.zeros((h, w), dtype=np.complex128)
    want[k0, l0] = np.sqrt(h * w)
    for f2 in (dft.dft2, fft.fft2):
        np.testing.assert_allclose(f2(pw), want, atol=1e-12)


def test_naive_dft_vs_bruteforce_8x8():
    x = _rand_c((8, 8), 7)
    np.testing.assert_allclose(dft.dft2(x), dft.dft2_bruteforce(x), atol=1e-12)
    np.testing.assert_allclose(dft.dft2(x, inverse=True), dft.dft2_bruteforce(x, inverse=True), atol=1e-12)
    np.testing.assert_allclose(fft.fft2(x), dft.dft2_bruteforce(x), atol=1e-12)


SIZES = [1, 2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 20, 25, 27, 30, 32, 45, 60, 64]


@pytest.mark.parametrize("n", SIZES)
def test_fft1_vs_naive(n):
    x = _rand_c((3, n), n)
    for inv in (False, True):
        assert _rel(fft.fft1(x, inv), dft.dft1(x, inv)) <= 1e-12


def test_fft2_vs_naive_grid():
    for h in SIZES[::3]:
        for w in SIZES[1::4]:
            x = _rand_c((h, w), h * 100 + w)
            assert _rel(fft.fft2(x), dft.dft2(x)) <= 1e-12
            assert _rel(fft.fft2(x, inverse=True), dft.dft2(x, inverse=True)) <= 1e-12


def test_fft_identities():
    x = _rand_c((24, 40), 3)
    y = _rand_c((24, 40), 4)
    X = fft.fft2(x)
    # Parseval (unitary)
    assert abs(np.sum(np.abs(X) ** 2) / np.sum(np.abs(x) ** 2) - 1.0) < 1e-13
    # inverse of forward
    assert _rel(fft.fft2(X, inverse=True), x) < 1e-13
    # linearity
    a, b = 0.3 - 1.2j, 2.0 + 0.5j
    assert _rel(fft.fft2(a * x + b * y), a * X + b * fft.fft2(y)) < 1e-13
    # shift theorem: x[m - s, n - t] <-> X[k, l] exp(-2 pi i (k s / H + l t / W))
    s, t = 5, 11
    xs = np.roll(x, (s, t), axis=(0, 1))
    k = np.arange(24)[:, None]
    l = np.arange(40)[None, :]
    assert _rel(fft.fft2(xs), X * np.exp(-2j * np.pi * (k * s / 24 + l * t / 40))) < 1e-12


@pytest.mark.parametrize("hw", [(1080, 1920), (2048, 2048)])
def test_fft2_vs_numpy_large(hw):
    x = _rand_c(hw, 11)
    ref = np.fft.fft2(x, norm="ortho")
    assert _rel(fft.fft2(x), ref) < 1e-13


def test_fft1_vs_numpy_4096_rows():
    x = _rand_c((16, 4096), 12)
    assert _rel(fft.fft1(x), np.fft.fft(x, axis=-1)) < 1e-13


# ---------------------------------------------------------------- Fresnel


LAM, PITCH = 532e-9, 8e-6


def test_chirp_separable_matches_direct():
    for hw, z in (((64, 48), 0.1), ((33, 20), 0.08)):
        np.testing.assert_allclose(optics.chirp(*hw, LAM, PITCH, z), optics.chirp_direct(*hw, LAM, PITCH, z), atol=1e-12)


def test_fresnel_lens_identity():
    h, w = 32, 48
    c = optics.chirp(h, w, LAM, PITCH, 0.1)
    out = optics.propagate(np.conj(c), c)
    want = np.zeros((h, w), dtype=np.complex128)
    want[0, 0] = np.sqrt(h * w)
    np.testing.assert_allclose(out, want, atol=1e-11)


def test_fresnel_far_limit_is_fourier():
    x = _rand_c((16, 24), 5)
    c = optics.chirp(16, 24, LAM, PITCH, 1e9)
    assert _rel(optics.propagate(x, c), fft.fft2(x)) < 1e-8


def test_fresnel_unitary_and_inverse():
    x = _rand_c((40, 30), 6)
    c = optics.chirp(40, 30, LAM, PITCH, 0.12)
    r = optics.propagate(x, c)
    assert abs(np.sum(np.abs(r) ** 2) / np.sum(np.abs(x) ** 2) - 1.0) < 1e-13
    assert _rel(optics.propagate(r, c, inverse=True), x) < 1e-13


def _chirped_gaussian_1d(n, w_px, beta):
    """Closed form of sum_m exp(-alpha m^2) exp(-2 pi i k n / N) with m = n - N//2 (Poisson summation,
    exact to rounding when both the Gaussian and its transform sit well inside their windows)."""
    alpha = 1.0 / w_px**2 - 1j * beta
    k = np.arange(n)
    ks = np.where(k < n / 2, k, k - n)
    om = 2 * np.pi * ks / n
    return np.exp(-2j * np.pi * k * (n // 2) / n) * np.sqrt(np.pi / alpha) * np.exp(-(om**2) / (4 * alpha))


def test_fresnel_chirped_gaussian_closed_form():
    # beta = pi p^2 / (lambda z) radians per px^2; pick z so beta = 5e-3
    beta = 5e-3
    z = np.pi * PITCH**2 / (LAM * beta)
    h, w = 128, 256
    wy, wx = 10.0, 12.0
    y = np.arange(h) - h // 2
    x = np.arange(w) - w // 2
    g = np.outer(np.exp(-(y**2) / wy**2), np.exp(-(x**2) / wx**2))
    out = optics.propagate(g, optics.chirp(h, w, LAM, PITCH, z))
    want = np.outer(_chirped_gaussian_1d(h, wy, beta), _chirped_gaussian_1d(w, wx, beta)) / np.sqrt(h * w)
    assert _rel(out, want) < 1e-12
    # the opposite chirp sign is far from it
    wrong = np.outer(_chirped_gaussian_1d(h, wy, -beta), _chirped_gaussian_1d(w, wx, -beta)) / np.sqrt(h * w)
    assert _rel(out, wrong) > 0.1
