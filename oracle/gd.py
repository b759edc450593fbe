"""Gradient-descent (Wirtinger) hologram optimisation (FP64).  Test infrastructure only.

Not in the paper: its algorithm libraries are GS, SA, DS and OSPR (section "Algorithm Libraries").
This is the differentiable counterpart of multi-plane Fresnel GS.  For phase parameters phi
[H][W], P planes with chirps c_p and target intensities T_p:

    h   = exp(i phi)
    U_p = F(h c_p),   I_p = |U_p|^2                          (F unitary)
    s_p = sum(I_p T_p) / sum(I_p^2)                          (optimal scale)
    L_p = sum((s_p I_p - T_p)^2) / sum(T_p^2),   L = (1/P) sum_p L_p

Gradient (s_p is optimal, so dL/ds_p = 0 and s_p is held fixed -- envelope theorem):

    dL/dI_p = (2/P) s_p (s_p I_p - T_p) / sum(T_p^2)
    g       = sum_p conj(c_p) F^-1(dL/dI_p * U_p)
    dL/dphi = 2 Im(g conj(h))

Adam (Kingma & Ba 2015), step t >= 1:
    m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2
    phi <- phi - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
"""
from __future__ import annotations

import numpy as np

from .fft import fft2


def loss_and_grad(phi, target_ints, chirps):
    """Returns (L, [L_p], dL/dphi) for phase ``phi`` [H][W]."""
    phi = np.asarray(phi, dtype=np.float64)
    h = np.exp(1j * phi)
    p = len(target_ints)
    g = np.zeros_like(h)
    losses = []
    for t, c in zip(target_ints, chirps):
        t = np.asarray(t, dtype=np.float64)
        u = fft2(h * c)
        i = np.abs(u) ** 2
        s = np.sum(i * t) / np.sum(i * i)
        tt = np.sum(t * t)
        losses.append(float(np.sum((s * i - t) ** 2) / tt))
        dldi = (2.0 / p) * s * (s * i - t) / tt
        g += np.conj(c) * fft2(dldi * u, inverse=True)
    grad = 2.0 * np.imag(g * np.conj(h))
    return float(np.mean(losses)), losses, grad


def loss_only(phi, target_ints, chirps) -> float:
    h = np.exp(1j * np.asarray(phi, dtype=np.float64))
    out = []
    for t, c in zip(target_ints, chirps):
        t = np.asarray(t, dtype=np.float64)
        i = np.abs(fft2(h * c)) ** 2
        s = np.sum(i * t) / np.sum(i * i)
        out.append(np.sum((s * i - t) ** 2) / np.sum(t * t))
    return float(np.mean(out))


def adam_update(phi, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step; returns (phi, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    phi = phi - lr * mhat / (np.sqrt(vhat) + eps)
    return phi, m, v


def gd_run(phi0, target_ints, chirps, n_steps: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """n_steps of Adam; returns dict(phi, loss [n_steps] (before each update), plane_loss)."""
    phi = np.asarray(phi0, dtype=np.float64).copy()
    m = np.zeros_like(phi)
    v = np.zeros_like(phi)
    curve, planes = [], []
    for t in range(1, n_steps + 1):
        l, lp, g = loss_and_grad(phi, target_ints, chirps)
        curve.append(l)
        planes.append(lp)
        phi, m, v = adam_update(phi, g, m, v, t, lr, beta1, beta2, eps)
    return {"phi": phi, "m": m, "v": v, "loss": np.array(curve), "plane_loss": np.array(planes)}
