"""Writes tests/golden/gs2048_curve.txt: the FP64 oracle's NMSE curve of the 2048 x 2048 Fourier GS
headline run (continuous phase, 100 iterations; smoothed-noise target sigma 2 px seed 0, uniform
starting phase seed 1), and its self-sensitivity: the same run from the starting phase plus
N(0, 1e-7) rad noise (three draws, seeds 11, 12, 13), with the largest relative spread of each
iterate's NMSE against the unperturbed curve.

Calls only the oracle and the seeded input generators (synth).  Takes about 10-15 minutes of one
CPU core per run (two 2048^2 float64 transforms per iteration).

    python tests/golden/make_gs2048_curve.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import gs as ogs  # noqa: E402

N, N_ITER = 2048, 100
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gs2048_curve.txt")


def main():
    a = synth.blur_target(N, N, 2.0, seed=0).astype(np.float64)
    phi0 = synth.uniform_phase(N, N, seed=1).astype(np.float64)
    t0 = time.time()
    ref = ogs.gs(a, phi0, N_ITER, 0)["nmse"]
    print(f"reference run {time.time() - t0:.0f} s", flush=True)
    spreads = []
    for seed in (11, 12, 13):
        noise = np.random.default_rng(seed).normal(0.0, 1e-7, (N, N))
        cur = ogs.gs(a, phi0 + noise, N_ITER, 0)["nmse"]
        spreads.append(np.abs(cur - ref) / ref)
        print(f"perturbed run {seed}: max rel spread {spreads[-1].max():.3e}", flush=True)
    spread = np.max(np.array(spreads), axis=0)
    with open(OUT, "w") as f:
        f.write("# FP64 oracle NMSE curve of Fourier GS at 2048 x 2048, continuous phase, 100 iterations\n")
        f.write("# (oracle.gs.gs; target synth.blur_target(2048, 2048, 2.0, seed=0), start phase\n")
        f.write("# synth.uniform_phase(2048, 2048, seed=1)), written by tests/golden/make_gs2048_curve.py.\n")
        f.write("# Columns: iterate k, NMSE of h_k, largest relative change of that NMSE over three reruns\n")
        f.write("# from the start phase + N(0, 1e-7) rad (the oracle's self-sensitivity).\n")
        for k in range(N_ITER + 1):
            f.write(f"{k} {ref[k]:.17e} {spread[k]:.6e}\n")
    print(f"wrote {OUT}; max self-sensitivity {spread.max():.3e}")


if __name__ == "__main__":
    main()
