"""GPU parity of mixed-region amplitude freedom (hg_mraf_run) against the FP64 oracle (oracle.mraf).

* one step, teacher-forced, as for GS: the GPU's h_k is fed to the oracle's MRAF step and compared
  with the GPU's h_{k+1} (continuous: wrapped phase error within the FP32 bound; levels: >= 99.9 %
  equal, mismatches only at level boundaries), on row-major and tiled fields, Fourier and Fresnel;
* the ROI NMSE of the iterates within 1 % of the oracle's, end to end;
* the whole plane as signal region and m = 1 reproduce hg_gs_run's hologram;
* argument errors.
"""
import numpy as np
import pytest

import synth
from oracle import mraf as omraf
from oracle import optics, project
from oracle.fft import fft2
from tests.helpers import check_continuous_phase, check_levels, check_nmse, cuda_device

LAM, PITCH = 532e-9, 8e-6


def _window(h, w):
    """An off-axis signal window in FFT order (rows and columns [1/8, 3/8) of the plane)."""
    m = np.zeros((h, w), dtype=np.uint8)
    m[h // 8: 3 * h // 8, w // 8: 3 * w // 8] = 1
    return m


def _level_phase(q, n):
    return (2 * np.pi * q / n).astype(np.float32)


def _run(hg, dev, a, mask, mix, n_iter, levels=0, phi0=None, fresnel_z=None):
    import torch

    h, w = a.shape
    kw = {}
    if fresnel_z is not None:
        kw = dict(propagation=hg.HG_FRESNEL, wavelength_m=LAM, pitch_m=PITCH, z_m=[fresnel_z])
    with hg.Plan([h], [w], quant_levels=levels, **kw) as plan:
        ta = torch.from_numpy(a).to(dev)
        tm = None if mask is None else [torch.from_numpy(mask).to(dev)]
        tp = None if phi0 is None else [torch.from_numpy(phi0).to(dev)]
        ph = torch.zeros((h, w), dtype=torch.float32, device=dev)
        lv = torch.zeros((h, w), dtype=torch.uint8, device=dev) if levels else None
        nm = torch.zeros((1, n_iter + 1), dtype=torch.float32, device=dev)
        plan.mraf([ta], mix, n_iter, signal_mask=tm, init_phase=tp, phase_out=[ph],
                  level_out=None if lv is None else [lv], nmse_out=nm)
        plan.sync()
        return ph.cpu().numpy(), (None if lv is None else lv.cpu().numpy()), nm.cpu().numpy()[0]


CASES = [
    # (H, W, levels, mix, fresnel z)
    (64, 64, 0, 0.6, None),
    (64, 64, 4, 0.5, None),
    (120, 64, 8, 0.7, 0.05),
    (512, 512, 0, 0.5, None),
    (512, 512, 2, 0.8, None),
    (2048, 1024, 0, 0.6, None),
    (1080, 1920, 4, 0.5, 0.1),
    (360, 480, 0, 0.6, None),
    (90, 100, 4, 0.5, 0.05),
]


@pytest.mark.gpu
@pytest.mark.parametrize("h, w, levels, mix, z", CASES)
def test_mraf_one_step_teacher_forced(h, w, levels, mix, z):
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    a = synth.blur_target(h, w, 2.0, seed=h + 3 * w + levels)
    mask = _window(h, w)
    c = optics.chirp(h, w, LAM, PITCH, z) if z else None
    rng = np.random.default_rng(9)
    phi0 = _level_phase(rng.integers(0, levels, (h, w)), levels) if levels else synth.uniform_phase(h, w, seed=10)
    ph1, q1, nm1 = _run(hg, dev, a, mask, mix, 1, levels, phi0, z)
    ph2, q2, nm2 = _run(hg, dev, a, mask, mix, 2, levels, phi0, z)
    a64 = a.astype(np.float64)
    h0, _ = project.slm_project(np.exp(1j * phi0.astype(np.float64)), levels)
    s1 = omraf.mraf_step(h0, a64, mask.astype(bool), mix, levels, c)
    if levels:
        check_levels(q1, s1["q"], s1["g"], levels)
        h1 = project.level_field(q1, levels)
    else:
        check_continuous_phase(ph1, s1["g"], s1["h"])
        h1 = np.exp(1j * ph1.astype(np.float64))
    s2 = omraf.mraf_step(h1, a64, mask.astype(bool), mix, levels, c)
    if levels:
        check_levels(q2, s2["q"], s2["g"], levels)
    else:
        check_continuous_phase(ph2, s2["g"], s2["h"])

    def e(hh):
        r = fft2(hh if c is None else hh * c)
        return omraf.roi_nmse(np.abs(r) ** 2, a64 * a64, mask.astype(bool))

    check_nmse(nm1, [e(h0), e(h1)], rtol=1e-3)


@pytest.mark.gpu
def test_mraf_roi_nmse_curve():
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    a = synth.spots_target(256, 256, 20, seed=41)
    mask = _window(256, 256)
    phi0 = synth.uniform_phase(256, 256, seed=42)
    _, _, nm = _run(hg, dev, a, mask, 0.5, 12, 0, phi0)
    ref = omraf.mraf(a.astype(np.float64), mask.astype(bool), 0.5, phi0.astype(np.float64), 12, 0)
    check_nmse(nm, ref["nmse"])


@pytest.mark.gpu
@pytest.mark.parametrize("h, w", [(256, 256), (512, 512)])
def test_mraf_whole_plane_is_gs(h, w):
    import torch
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    a = synth.blur_target(h, w, 2.0, seed=43)
    phi0 = synth.uniform_phase(h, w, seed=44)
    ph_m, _, nm_m = _run(hg, dev, a, None, 1.0, 6, 0, phi0)
    with hg.Plan([h], [w]) as plan:
        ph = torch.zeros((h, w), dtype=torch.float32, device=dev)
        nm = torch.zeros((1, 7), dtype=torch.float32, device=dev)
        plan.gs([torch.from_numpy(a).to(dev)], 6, init_phase=[torch.from_numpy(phi0).to(dev)], phase_out=[ph],
                nmse_out=nm)
        plan.sync()
    d = np.angle(np.exp(1j * (ph_m - ph.cpu().numpy())))
    assert np.max(np.abs(d)) < 1e-3
    np.testing.assert_allclose(nm_m, nm.cpu().numpy()[0], rtol=1e-4)


@pytest.mark.gpu
def test_mraf_argument_errors():
    import torch
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    a = torch.ones((64, 64), dtype=torch.float32, device=dev)
    with hg.Plan([64], [64]) as plan:
        for bad in (0.0, -0.5, 1.5):
            with pytest.raises(hg.HologenError) as e:
                plan.mraf([a], bad, 2)
            assert e.value.status == hg.HG_ERR_INVALID_ARG
    with hg.Plan([64], [64], propagation=hg.HG_FRESNEL, wavelength_m=LAM, pitch_m=PITCH, z_m=[0.05, 0.1]) as plan:
        with pytest.raises(hg.HologenError):
            plan.mraf([a, a], 0.5, 2)
