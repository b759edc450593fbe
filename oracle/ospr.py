"""One-Step Phase-Retrieval (FP64).  Test infrastructure only.

The paper's HoloGenAlgOSPRCuda (section "Algorithm Libraries") implements One-Step Phase-Retrieval;
no formula is printed.  Reading taken here (Cable, Buckley et al. 2004, classic OSPR), for target t
with amplitude A (FFT order), S subframes s = 0..S-1:

    theta_s[p] = 2 pi u_s[p]          u from oracle.philox.ospr_uniform(p, s, t, seed)
    E_s        = A_s exp(i theta_s)   (A_s as in GS: energy of a unit-modulus field)
    h_s        = P_binary(conj(c) F^-1(E_s))              (h = +1 / -1, ties as oracle.project)
    [n_iter > 0: h_s continues with n_iter binary GS iterations against A]
    I_acc     += |F(h_s c)|^2
    nmse[s]    = NMSE(I_acc / (s + 1), A^2)

Bits: bit = 1 where h = -1 (phase pi), packed LSB-first into uint32 words along each row,
ceil(W / 32) words per row.

A real +-1 hologram has a point-symmetric (Hermitian) Fourier replay, I[k] = I[-k mod N]; targets fed
to OSPR are therefore symmetrised by the input generator.
"""
from __future__ import annotations

import numpy as np

from .fft import fft2
from .gs import scaled_amplitude
from .metrics import nmse
from .philox import ospr_uniform
from .project import amplitude_replace, slm_project


def subframe_phase(h: int, w: int, subframe: int, target: int, seed: int) -> np.ndarray:
    u = ospr_uniform(h * w, subframe, target, seed).reshape(h, w)
    return 2.0 * np.pi * u


def pack_bits(q: np.ndarray) -> np.ndarray:
    """Pack a [H][W] 0/1 array LSB-first into uint32 words along rows: [H][ceil(W/32)]."""
    hh, ww = q.shape
    nw = (ww + 31) // 32
    out = np.zeros((hh, nw), dtype=np.uint64)
    for j in range(ww):
        out[:, j // 32] |= (q[:, j].astype(np.uint64) & np.uint64(1)) << np.uint64(j % 32)
    return out.astype(np.uint32)


def unpack_bits(words: np.ndarray, w: int) -> np.ndarray:
    hh = words.shape[0]
    out = np.zeros((hh, w), dtype=np.int64)
    for j in range(w):
        out[:, j] = (words[:, j // 32].astype(np.uint64) >> np.uint64(j % 32)) & np.uint64(1)
    return out


def ospr_subframe(target_amp, subframe: int, target: int, seed: int, n_iter: int = 0, c=None):
    """One subframe: returns dict(h, q, g, intensity) where g is the pre-binarisation field of the
    last projection and ``intensity`` = |F(h c)|^2 (unitary)."""
    a = np.asarray(target_amp, dtype=np.float64)
    a_s = scaled_amplitude(a)
    hh, ww = a.shape
    theta = subframe_phase(hh, ww, subframe, target, seed)
    g = fft2(a_s * np.exp(1j * theta), inverse=True)
    if c is not None:
        g = np.conj(c) * g
    h, q = slm_project(g, 2)
    for _ in range(n_iter):
        r = fft2(h if c is None else h * c)
        g = fft2(amplitude_replace(r, a_s), inverse=True)
        if c is not None:
            g = np.conj(c) * g
        h, q = slm_project(g, 2)
    r = fft2(h if c is None else h * c)
    return {"h": h, "q": q, "g": g, "intensity": np.abs(r) ** 2}


def ospr(target_amp, n_subframes: int, target: int, seed: int, n_iter: int = 0, c=None):
    """OSPR for one target.  Returns dict(bits [S][H][ceil(W/32)], q [S][H][W], nmse [S], i_acc)."""
    a = np.asarray(target_amp, dtype=np.float64)
    t = a * a
    i_acc = np.zeros(a.shape, dtype=np.float64)
    curve, qs, bits = [], [], []
    for s in range(n_subframes):
        sf = ospr_subframe(a, s, target, seed, n_iter, c)
        i_acc += sf["intensity"]
        curve.append(nmse(i_acc / (s + 1), t))
        qs.append(sf["q"])
        bits.append(pack_bits(sf["q"]))
    return {"bits": np.array(bits), "q": np.array(qs), "nmse": np.array(curve), "i_acc": i_acc}
