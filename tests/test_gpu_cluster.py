"""The whole-run cluster kernel (strip width -1, the default for a square 64, 128 or 256 pixel class
of one item): one thread-block cluster per item holds the field in shared memory for the whole loop.

* against the FP64 oracle: the first and second iterations teacher-forced and the NMSE curve, for
  continuous, 4-level and binary SLMs, Fourier and Fresnel (the generic GS tests also run through it
  at 64^2 and 256^2, and the strip-width test checks it bitwise against the two-pass kernels);
* n_iter = 0 writes the projected start; a class of more items than one launch takes (chunks)
  gives each item the result of a one-item plan; classes that cannot use it (non-square) sit
  beside it in one plan; MRAF and illuminated runs of such a class fall back to the two-pass
  kernels and keep their results.
"""
import numpy as np
import pytest

import synth
from oracle import gs as ogs
from oracle import optics, project
from oracle.fft import fft2
from oracle.metrics import nmse
from tests.helpers import check_continuous_phase, check_levels, check_nmse, cuda_device

LAM, PITCH = 532e-9, 8e-6


def _gs(hg, dev, sizes, targets, phases, n_iter, levels=0, z=None, width=None, cluster_items=()):
    import torch

    kw = dict(propagation=hg.HG_FRESNEL, wavelength_m=LAM, pitch_m=PITCH, z_m=[z]) if z else {}
    with hg.Plan([s[0] for s in sizes], [s[1] for s in sizes], quant_levels=levels, **kw) as plan:
        if width is not None:
            for i in range(len(sizes)):
                plan.set_strip_width(i, width)
        for i in cluster_items:
            plan.set_strip_width(i, hg.HG_STRIP_CLUSTER)
        widths = [plan.strip_width(i) for i in range(len(sizes))]
        ph = [torch.zeros(s, dtype=torch.float32, device=dev) for s in sizes]
        lv = [torch.zeros(s, dtype=torch.uint8, device=dev) for s in sizes] if levels else None
        nm = torch.zeros((len(sizes), n_iter + 1), dtype=torch.float32, device=dev)
        plan.gs([torch.from_numpy(t).to(dev) for t in targets], n_iter,
                init_phase=[torch.from_numpy(p).to(dev) for p in phases], phase_out=ph, level_out=lv, nmse_out=nm)
        plan.sync()
        return ([x.cpu().numpy() for x in ph], None if lv is None else [x.cpu().numpy() for x in lv],
                nm.cpu().numpy(), widths)


@pytest.mark.gpu
@pytest.mark.parametrize("n, levels, z", [(256, 0, None), (256, 2, None), (128, 4, 0.05), (64, 0, 0.02),
                                          (128, 0, None)])
def test_cluster_steps_against_oracle(n, levels, z):
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    a = synth.blur_target(n, n, 2.0, seed=500 + n + levels)
    rng = np.random.default_rng(501)
    phi0 = (2 * np.pi * rng.integers(0, levels, (n, n)) / levels).astype(np.float32) if levels else \
        synth.uniform_phase(n, n, seed=502)
    c = optics.chirp(n, n, LAM, PITCH, z) if z else None
    ph1, q1, nm1, widths = _gs(hg, dev, [(n, n)], [a], [phi0], 1, levels, z)
    assert widths == [hg.HG_STRIP_CLUSTER]
    ph2, q2, _, _ = _gs(hg, dev, [(n, n)], [a], [phi0], 2, levels, z)
    a64 = a.astype(np.float64)
    h0, _ = project.slm_project(np.exp(1j * phi0.astype(np.float64)), levels)
    s1 = ogs.gs_step(h0, a64, levels, c)
    if levels:
        check_levels(q1[0], s1["q"], s1["g"], levels)
        h1 = project.level_field(q1[0], levels)
    else:
        check_continuous_phase(ph1[0], s1["g"], s1["h"])
        h1 = np.exp(1j * ph1[0].astype(np.float64))
    s2 = ogs.gs_step(h1, a64, levels, c)
    if levels:
        check_levels(q2[0], s2["q"], s2["g"], levels)
    else:
        check_continuous_phase(ph2[0], s2["g"], s2["h"])

    def e(hh):
        r = fft2(hh if c is None else hh * c)
        return nmse(np.abs(r) ** 2, a64 * a64)

    check_nmse(nm1[0], [e(h0), e(h1)], rtol=1e-3)


@pytest.mark.gpu
def test_cluster_nmse_curve():
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    a = synth.spots_target(256, 256, 20, seed=510)
    phi0 = synth.uniform_phase(256, 256, seed=511)
    _, _, nm, _ = _gs(hg, dev, [(256, 256)], [a], [phi0], 20)
    ref = ogs.gs(a.astype(np.float64), phi0.astype(np.float64), 20, 0)
    check_nmse(nm[0], ref["nmse"])


@pytest.mark.gpu
@pytest.mark.parametrize("levels", [0, 8])
def test_cluster_zero_iterations_writes_the_projected_start(levels):
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    a = synth.blur_target(128, 128, 2.0, seed=520)
    phi0 = synth.uniform_phase(128, 128, seed=521)
    ph, q, nm, _ = _gs(hg, dev, [(128, 128)], [a], [phi0], 0, levels)
    ref_ph, ref_q, ref_nm, _ = _gs(hg, dev, [(128, 128)], [a], [phi0], 0, levels, width=0)
    assert np.array_equal(ph[0], ref_ph[0])
    if levels:
        assert np.array_equal(q[0], ref_q[0])
    np.testing.assert_allclose(nm, ref_nm, rtol=1e-5, atol=1e-7)
    h0, _ = project.slm_project(np.exp(1j * phi0.astype(np.float64)), levels)
    assert nm.shape == (1, 1)
    assert abs(nm[0, 0] - nmse(np.abs(fft2(h0)) ** 2, a.astype(np.float64) ** 2)) <= 1e-3 * nm[0, 0]


@pytest.mark.gpu
def test_cluster_chunks_and_mixed_classes():
    """40 items of 128^2 (two launches of at most 32 items) beside non-square classes in one plan:
    every item as a one-item plan computes it."""
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    sizes = [(128, 128)] * 40 + [(128, 256), (256, 256), (64, 64)]
    targets = [synth.blur_target(h, w, 2.0, seed=600 + i) for i, (h, w) in enumerate(sizes)]
    phases = [synth.uniform_phase(h, w, seed=700 + i) for i, (h, w) in enumerate(sizes)]
    ph, q, nm, widths = _gs(hg, dev, sizes, targets, phases, 6, 4, cluster_items=(0, 41))
    assert widths[0] == widths[41] == hg.HG_STRIP_CLUSTER and widths[40] != hg.HG_STRIP_CLUSTER
    for i in (0, 17, 31, 32, 39, 40, 41, 42):
        ph1, q1, nm1, _ = _gs(hg, dev, [sizes[i]], [targets[i]], [phases[i]], 6, 4)
        assert np.array_equal(q[i], q1[0]), i
        np.testing.assert_allclose(nm[i], nm1[0], rtol=1e-5, atol=1e-7)


@pytest.mark.gpu
def test_cluster_class_falls_back_for_mraf_and_illumination():
    import torch
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    n = 256
    a = torch.from_numpy(synth.blur_target(n, n, 2.0, seed=530)).to(dev)
    p0 = torch.from_numpy(synth.uniform_phase(n, n, seed=531)).to(dev)
    mask = torch.zeros((n, n), dtype=torch.uint8, device=dev)
    mask[n // 8: 3 * n // 8, n // 8: 3 * n // 8] = 1
    illum = torch.from_numpy(np.exp(-np.linspace(-1, 1, n)[:, None] ** 2 - np.linspace(-1, 1, n)[None, :] ** 2)
                             .astype(np.float32)).to(dev)
    res = {}
    for width in (None, 0):
        with hg.Plan([n], [n]) as plan:
            if width is not None:
                plan.set_strip_width(0, width)
            out = []
            ph = torch.zeros((n, n), dtype=torch.float32, device=dev)
            plan.mraf([a], 0.5, 4, signal_mask=[mask], init_phase=[p0], phase_out=[ph])
            plan.sync()
            out.append(ph.cpu().numpy())
            plan.set_illumination([illum])
            ph = torch.zeros((n, n), dtype=torch.float32, device=dev)
            plan.gs([a], 4, init_phase=[p0], phase_out=[ph])
            plan.sync()
            out.append(ph.cpu().numpy())
            res[width] = out
    for x, y in zip(res[None], res[0]):
        d = np.angle(np.exp(1j * (x.astype(np.float64) - y)))
        assert np.max(np.abs(d)) < 1e-3
