"""Direct binary search (DBS) with a single-pixel replay update, and simulated annealing over the same
trial flips (FP64).  Test infrastructure only.

The paper lists a direct-search algorithm for binary holograms and a replay updater that changes a
single pixel (section "Algorithm Libraries": the DS algorithm class and FFTUpdaterCuda) without
formulas.  Reading taken here (Seldowitz, Allebach & Sweeney 1987): a binary hologram h in {+1, -1}
(phase {0, pi}) with replay R = F(h c) (unitary F, c = 1 Fourier or the Fresnel chirp) is improved
one pixel at a time.  A sweep visits the SLM pixels p = (m, n) in row-major order; for each it tries
the flip h_p -> -h_p, whose replay change is the single-pixel update

    R'[k, l] = R[k, l] + d_p exp(-2 pi i (k m / H + l n / W)) / sqrt(HW),   d_p = -2 h_p c_p,

and keeps it when the NMSE of |R'|^2 against T = A^2 (optimal scale, oracle.metrics) is strictly
lower than that of |R|^2; otherwise the hologram and R stay as they were.  The start is the binary
projection h_0 = P_2(exp(i phi_0)).  ``nmse[s]`` for s = 0..n_sweeps is the NMSE after s sweeps.
"""
from __future__ import annotations

import numpy as np

from .fft import fft2
from .metrics import nmse
from .project import slm_project


def pixel_basis(h_: int, w_: int, m: int, n: int) -> np.ndarray:
    """The unitary DFT of a unit impulse at SLM pixel (m, n): exp(-2 pi i (k m / H + l n / W)) / sqrt(HW)."""
    ey = np.exp(-2j * np.pi * ((np.arange(h_) * m) % h_) / h_)
    ex = np.exp(-2j * np.pi * ((np.arange(w_) * n) % w_) / w_)
    return np.outer(ey, ex) / np.sqrt(h_ * w_)


def flip_update(r: np.ndarray, h: np.ndarray, m: int, n: int, c=None) -> np.ndarray:
    """The replay field after flipping SLM pixel (m, n) of h (the single-pixel replay update)."""
    cp = 1.0 if c is None else c[m, n]
    d = -2.0 * h[m, n] * cp
    return r + d * pixel_basis(r.shape[0], r.shape[1], m, n)


def start(init_phase, c=None):
    """h_0 = P_2(exp(i phi_0)) (real +-1 field) and its replay R_0 = F(h_0 c)."""
    h0, _ = slm_project(np.exp(1j * np.asarray(init_phase, dtype=np.float64)), 2)
    h0 = np.real(h0)
    return h0, fft2(h0 if c is None else h0 * c)


def sweep(h: np.ndarray, r: np.ndarray, t: np.ndarray, c=None, decide=None):
    """One DBS sweep in row-major pixel order.  Returns (h, r, flipped) with flipped[m, n] whether the
    flip at (m, n) was kept.  decide(p, e_old, e_new) -> bool replaces the rule e_new < e_old (used by
    tests to follow another implementation's decisions)."""
    h = np.array(h, dtype=np.float64)
    r = np.array(r, dtype=np.complex128)
    h_, w_ = h.shape
    flipped = np.zeros(h.shape, dtype=bool)
    e = nmse(np.abs(r) ** 2, t)
    for m in range(h_):
        for n in range(w_):
            r_new = flip_update(r, h, m, n, c)
            e_new = nmse(np.abs(r_new) ** 2, t)
            keep = e_new < e if decide is None else decide(m * w_ + n, e, e_new)
            if keep:
                h[m, n] = -h[m, n]
                r, e = r_new, e_new
                flipped[m, n] = True
    return h, r, flipped


def dbs(target_amp, init_phase, n_sweeps: int, c=None):
    """DBS loop.  Returns dict(h, phase, q, nmse[n_sweeps+1])."""
    a = np.asarray(target_amp, dtype=np.float64)
    t = a * a
    h, r = start(init_phase, c)
    curve = [nmse(np.abs(r) ** 2, t)]
    for _ in range(n_sweeps):
        h, r, _ = sweep(h, r, t, c)
        curve.append(nmse(np.abs(r) ** 2, t))
    q = (h < 0).astype(np.int64)
    return {"h": h, "phase": np.pi * q.astype(np.float64), "q": q, "nmse": np.array(curve)}


def sa(target_amp, init_phase, n_sweeps: int, t0: float, alpha: float, seed: int, item: int = 0, c=None):
    """Simulated annealing over the same trial flips (FP64).

    The paper lists a simulated-annealing class beside direct search (section "Algorithm
    Libraries") without formulas.  Reading taken here (Kirkpatrick, Gelatt & Vecchi 1983, with the
    flips, order and energy of DBS): sweep s runs at temperature T_s = t0 alpha^s (T_0 = t0, then
    multiplied by alpha after each sweep); a trial flip is kept when it lowers the NMSE E, or
    otherwise when u < exp(-(E' - E) / T_s), with u the Philox draw of (pixel, sweep)
    (philox.anneal_uniform).  Returns dict(h, phase, q, nmse[n_sweeps+1])."""
    from .philox import anneal_uniform

    a = np.asarray(target_amp, dtype=np.float64)
    t = a * a
    h, r = start(init_phase, c)
    curve = [nmse(np.abs(r) ** 2, t)]
    temp = float(t0)
    for s in range(n_sweeps):
        u = anneal_uniform(h.size, s, item, seed)
        h, r, _ = sweep(h, r, t, c, decide=metropolis(u, temp))
        curve.append(nmse(np.abs(r) ** 2, t))
        temp *= alpha
    q = (h < 0).astype(np.int64)
    return {"h": h, "phase": np.pi * q.astype(np.float64), "q": q, "nmse": np.array(curve)}


def metropolis(u: np.ndarray, temp: float):
    """The acceptance rule of one annealing sweep: keep an improving flip, otherwise keep it when
    u[p] < exp(-(E' - E) / T)."""

    def rule(p, e_old, e_new):
        return e_new < e_old or u[p] < np.exp(-(e_new - e_old) / temp)

    return rule
