"""Targets in display order (HG_TARGET_CENTRED): a plan given fftshift(A) and the flag must produce
exactly what a plain plan produces from A (the plan reads pixel (i, j) of the FFT-ordered replay
plane from ((i + H/2) mod H, (j + W/2) mod W), numpy's ifftshift), for every path that takes
targets: single- and multi-plane GS, MRAF and HIO (masks shifted alike), OSPR and gradient
descent.  Bitwise: the kernels see the same values in the same places."""
import numpy as np
import pytest

import synth
from tests.helpers import cuda_device

LAM, PITCH = 532e-9, 8e-6


def _shift(x):
    return np.ascontiguousarray(np.fft.fftshift(x))


def _t(dev, x):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def _gs(hg, dev, a, flags, levels, kw, mode=None, mask=None):
    import torch

    h, w = a.shape
    with hg.Plan([h], [w], quant_levels=levels, flags=flags, **kw) as plan:
        ph = torch.zeros((h, w), dtype=torch.float32, device=dev)
        nm = torch.zeros((1, 6), dtype=torch.float32, device=dev)
        p0 = [_t(dev, synth.uniform_phase(h, w, seed=7))]
        if mode == "mraf":
            plan.mraf([_t(dev, a)], 0.6, 5, signal_mask=[_t(dev, mask)], init_phase=p0, phase_out=[ph], nmse_out=nm)
        elif mode == "hio":
            plan.hio([_t(dev, a)], 0.7, 5, signal_mask=[_t(dev, mask)], init_phase=p0, phase_out=[ph], nmse_out=nm)
        else:
            plan.gs([_t(dev, a)], 5, init_phase=p0, phase_out=[ph], nmse_out=nm)
        plan.sync()
        return ph.cpu().numpy(), nm.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("h, w, levels, fresnel", [(512, 512, 0, False), (2048, 2048, 0, False), (256, 256, 4, True),
                                                    (1080, 1920, 4, True), (15, 16, 2, False), (120, 64, 0, True),
                                                    (27, 125, 4, False), (75, 90, 0, True)])
def test_centred_gs_equals_shifted_plain(h, w, levels, fresnel):
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    kw = dict(propagation=hg.HG_FRESNEL, wavelength_m=LAM, pitch_m=PITCH, z_m=[0.1]) if fresnel else {}
    a = synth.spots_target(h, w, 6, seed=h + w) if min(h, w) >= 64 else synth.blur_target(h, w, 1.0, seed=3)
    p_ref, n_ref = _gs(hg, dev, a, 0, levels, kw)
    p_c, n_c = _gs(hg, dev, _shift(a), hg.HG_TARGET_CENTRED, levels, kw)
    assert np.array_equal(p_ref, p_c)
    assert np.array_equal(n_ref, n_c)


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["mraf", "hio"])
def test_centred_signal_region_paths(mode):
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    h, w = 512, 1024
    a = synth.spots_target(h, w, 10, seed=5)
    mask = np.zeros((h, w), dtype=np.uint8)
    mask[h // 8: 3 * h // 8, w // 8: 3 * w // 8] = 1
    p_ref, n_ref = _gs(hg, dev, a, 0, 0, {}, mode, mask)
    p_c, n_c = _gs(hg, dev, _shift(a), hg.HG_TARGET_CENTRED, 0, {}, mode, _shift(mask))
    assert np.array_equal(p_ref, p_c)
    assert np.array_equal(n_ref, n_c)


@pytest.mark.gpu
def test_centred_multiplane_gs():
    import torch
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    n = 256
    ts = [synth.spots_target(n, n, 8, seed=20 + p) for p in range(2)]
    kw = dict(propagation=hg.HG_FRESNEL, wavelength_m=LAM, pitch_m=PITCH, z_m=[0.08, 0.12])
    out = []
    for flags, tt in ((0, ts), (hg.HG_TARGET_CENTRED, [_shift(t) for t in ts])):
        with hg.Plan([n], [n], flags=flags, **kw) as plan:
            ph = torch.zeros((n, n), dtype=torch.float32, device=dev)
            nm = torch.zeros((1, 5), dtype=torch.float32, device=dev)
            plan.gs([_t(dev, t) for t in tt], 4, seed=9, phase_out=[ph], nmse_out=nm)
            plan.sync()
            out.append((ph.cpu().numpy(), nm.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.gpu
def test_centred_ospr():
    import torch
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    h, w, ns = 256, 512, 4
    a = synth.symmetrise(synth.blur_target(h, w, 2.0, seed=31))
    out = []
    for flags, aa in ((0, a), (hg.HG_TARGET_CENTRED, _shift(a))):
        with hg.Plan([h], [w], quant_levels=2, flags=flags) as plan:
            bits = torch.zeros((ns, h, (w + 31) // 32), dtype=torch.int32, device=dev)
            nm = torch.zeros((1, ns), dtype=torch.float32, device=dev)
            plan.ospr([_t(dev, aa)], ns, 0, 77, bits_out=[bits], nmse_out=nm)
            plan.sync()
            out.append((bits.cpu().numpy(), nm.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.gpu
def test_centred_gradient_descent():
    import torch
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    n = 256
    kw = dict(propagation=hg.HG_FRESNEL, wavelength_m=LAM, pitch_m=PITCH, z_m=[0.08, 0.1, 0.12])
    ts = []
    for p in range(3):
        t = synth.spots_target(n, n, 8, seed=40 + p).astype(np.float64) ** 2
        ts.append((t / np.sqrt(np.sum(t * t))).astype(np.float32))
    out = []
    for flags, tt in ((0, ts), (hg.HG_TARGET_CENTRED, [_shift(t) for t in ts])):
        with hg.Plan([n], [n], flags=flags, **kw) as plan:
            phi = _t(dev, synth.uniform_phase(n, n, seed=43))
            m = torch.zeros_like(phi)
            v = torch.zeros_like(phi)
            loss = torch.zeros((1, 4), dtype=torch.float32, device=dev)
            grad = torch.zeros_like(phi)
            targets = [_t(dev, t) for t in tt]
            for step in (1, 2):
                plan.gd_step([phi], targets, [m], [v], step, loss_out=loss, grad_out=[grad])
            plan.sync()
            out.append((phi.cpu().numpy(), loss.cpu().numpy(), grad.cpu().numpy()))
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)

