"""GS under an SLM illumination amplitude profile (hg_plan_set_illumination) against the FP64 oracle.

* teacher-forced one step (continuous and quantised; row-major and tiled fields; Fourier and
  Fresnel): the GPU's phases / levels after one and two iterations against oracle.gs.gs_step with
  the same profile;
* a unit profile reproduces plain GS bitwise; NMSE curves within 1 %;
* runs that do not take a profile reject a plan that has one.
"""
import numpy as np
import pytest

import synth
from oracle import gs as ogs
from oracle import optics, project
from tests.helpers import check_continuous_phase, check_levels, check_nmse, cuda_device

LAM, PITCH = 532e-9, 8e-6


def _beam(h, w):
    y = np.arange(h) - (h - 1) / 2
    x = np.arange(w) - (w - 1) / 2
    return np.exp(-(y[:, None] ** 2 / (2 * (0.3 * h) ** 2) + x[None, :] ** 2 / (2 * (0.3 * w) ** 2))).astype(np.float32)


def _run(hg, dev, a, illum, n_iter, levels=0, phi0=None, z=None):
    import torch

    h, w = a.shape
    kw = dict(propagation=hg.HG_FRESNEL, wavelength_m=LAM, pitch_m=PITCH, z_m=[z]) if z else {}
    with hg.Plan([h], [w], quant_levels=levels, **kw) as plan:
        ti = None if illum is None else torch.from_numpy(illum).to(dev)
        if ti is not None:
            plan.set_illumination([ti])
        ph = torch.zeros((h, w), dtype=torch.float32, device=dev)
        lv = torch.zeros((h, w), dtype=torch.uint8, device=dev) if levels else None
        nm = torch.zeros((1, n_iter + 1), dtype=torch.float32, device=dev)
        plan.gs([torch.from_numpy(a).to(dev)], n_iter, init_phase=[torch.from_numpy(phi0).to(dev)], phase_out=[ph],
                level_out=None if lv is None else [lv], nmse_out=nm)
        plan.sync()
        return ph.cpu().numpy(), (None if lv is None else lv.cpu().numpy()), nm.cpu().numpy()[0]


@pytest.mark.gpu
@pytest.mark.parametrize("h, w, levels, z", [(64, 64, 0, None), (120, 64, 4, 0.05), (512, 512, 0, None),
                                             (512, 512, 8, 0.1), (2048, 1024, 2, None)])
def test_illuminated_gs_one_step_teacher_forced(h, w, levels, z):
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    a = synth.blur_target(h, w, 2.0, seed=h + w + 7 * levels)
    illum = _beam(h, w)
    c = optics.chirp(h, w, LAM, PITCH, z) if z else None
    phi0 = synth.uniform_phase(h, w, seed=61)
    ph1, q1, nm1 = _run(hg, dev, a, illum, 1, levels, phi0, z)
    ph2, q2, _ = _run(hg, dev, a, illum, 2, levels, phi0, z)
    a64, il = a.astype(np.float64), illum.astype(np.float64)
    u0, _ = project.slm_project(np.exp(1j * phi0.astype(np.float64)), levels)
    h0 = il * u0
    s1 = ogs.gs_step(h0, a64, levels, c, il)
    if levels:
        check_levels(q1, s1["q"], s1["g"], levels)
        h1 = il * project.level_field(q1, levels)
    else:
        check_continuous_phase(ph1, s1["g"], s1["h"] / il)
        h1 = il * np.exp(1j * ph1.astype(np.float64))
    s2 = ogs.gs_step(h1, a64, levels, c, il)
    if levels:
        check_levels(q2, s2["q"], s2["g"], levels)
    else:
        check_continuous_phase(ph2, s2["g"], s2["h"] / il)
    from oracle.fft import fft2
    from oracle.metrics import nmse

    def e(hh):
        return nmse(np.abs(fft2(hh if c is None else hh * c)) ** 2, a64 * a64)

    check_nmse(nm1, [e(h0), e(h1)], rtol=1e-3)


@pytest.mark.gpu
@pytest.mark.parametrize("h, w", [(256, 256), (512, 512)])
def test_unit_illumination_is_plain_gs_bitwise(h, w):
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    a = synth.blur_target(h, w, 2.0, seed=62)
    phi0 = synth.uniform_phase(h, w, seed=63)
    ref = _run(hg, dev, a, None, 6, 4, phi0)
    out = _run(hg, dev, a, np.ones((h, w), dtype=np.float32), 6, 4, phi0)
    assert np.array_equal(out[1], ref[1]) and np.array_equal(out[2], ref[2])


@pytest.mark.gpu
def test_illuminated_gs_nmse_curve():
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    a = synth.blur_target(128, 128, 2.0, seed=64)
    illum = _beam(128, 128)
    phi0 = synth.uniform_phase(128, 128, seed=65)
    _, _, nm = _run(hg, dev, a, illum, 10, 0, phi0)
    ref = ogs.gs(a.astype(np.float64), phi0.astype(np.float64), 10, 0, illum=illum.astype(np.float64))
    check_nmse(nm, ref["nmse"])


@pytest.mark.gpu
def test_runs_without_profile_support_reject_it():
    import torch
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    a = torch.ones((64, 64), dtype=torch.float32, device=dev)
    il = torch.ones((64, 64), dtype=torch.float32, device=dev)
    with hg.Plan([64], [64], quant_levels=2) as plan:
        plan.set_illumination([il])
        with pytest.raises(hg.HologenError):
            plan.mraf([a], 0.5, 2)
        with pytest.raises(hg.HologenError):
            plan.ospr([a], 2)
        plan.set_illumination(None)
        plan.mraf([a], 0.5, 2)
        plan.sync()
    with hg.Plan([64], [64], propagation=hg.HG_FRESNEL, wavelength_m=LAM, pitch_m=PITCH, z_m=[0.05, 0.1]) as plan:
        with pytest.raises(hg.HologenError):
            plan.set_illumination([il])
