"""Philox4x32-10 counter-based random numbers (Salmon, Moraes, Dror & Shaw, SC'11).

Test infrastructure only.  The paper's Randomiser (section "Algorithm Libraries") "allows for
randomisation of different combinations of phase and amplitude" without naming a generator.  A
counter-based generator is chosen so that the random phase of (target, subframe, pixel) is a pure
function of its indices; it is written here from its published definition:

* state: counter (c0, c1, c2, c3) and key (k0, k1), all uint32;
* one round: (hi0, lo0) = 0xD2511F53 * c0, (hi1, lo1) = 0xCD9E8D57 * c2 (64-bit products split in
  halves); new counter = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0);
* between rounds the key is bumped by (0x9E3779B9, 0xBB67AE85); ten rounds.

Vectorised over numpy uint64 arrays holding uint32 values.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)
SH = np.uint64(32)


def philox4x32_10(counter, key):
    """counter: 4 arrays (or ints), key: 2 arrays (or ints).  Returns 4 uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK for c in counter)
    k0, k1 = (np.asarray(k, dtype=np.uint64) & MASK for k in key)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> SH, p0 & MASK
        hi1, lo1 = p1 >> SH, p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(c.astype(np.uint32) for c in (c0, c1, c2, c3))


def ospr_uniform(n_pixels: int, subframe: int, target: int, seed: int) -> np.ndarray:
    """Uniform [0, 1) draws u = (x >> 8) 2^-24 for pixels p = 0..n-1 (FFT order).

    x is word 0 of Philox4x32-10 with counter (p, subframe, 0, 0) and key
    (seed_lo, seed_hi ^ target).
    """
    p = np.arange(n_pixels, dtype=np.uint64)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    k0 = seed & 0xFFFFFFFF
    k1 = ((seed >> 32) ^ int(target)) & 0xFFFFFFFF
    x0, _, _, _ = philox4x32_10((p, subframe, 0, 0), (k0, k1))
    return (x0 >> np.uint32(8)).astype(np.float64) * (2.0 ** -24)


def init_uniform(n_pixels: int, item: int, seed: int) -> np.ndarray:
    """Starting-phase draws u for pixels p = 0..n-1: word 0 of Philox4x32-10 with counter
    (p, 0, 1, 0) and key (seed_lo, seed_hi ^ item), u = (x >> 8) 2^-24.  phi_0 = 2 pi u."""
    p = np.arange(n_pixels, dtype=np.uint64)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    k0 = seed & 0xFFFFFFFF
    k1 = ((seed >> 32) ^ int(item)) & 0xFFFFFFFF
    x0, _, _, _ = philox4x32_10((p, 0, 1, 0), (k0, k1))
    return (x0 >> np.uint32(8)).astype(np.float64) * (2.0 ** -24)


def anneal_uniform(n_pixels: int, sweep: int, item: int, seed: int) -> np.ndarray:
    """Acceptance draws of simulated annealing for the trial flips p = 0..n-1 of one sweep: word 0 of
    Philox4x32-10 with counter (p, sweep, 2, 0) and key (seed_lo, seed_hi ^ item), u = (x >> 8) 2^-24."""
    p = np.arange(n_pixels, dtype=np.uint64)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    k0 = seed & 0xFFFFFFFF
    k1 = ((seed >> 32) ^ int(item)) & 0xFFFFFFFF
    x0, _, _, _ = philox4x32_10((p, sweep, 2, 0), (k0, k1))
    return (x0 >> np.uint32(8)).astype(np.float64) * (2.0 ** -24)
