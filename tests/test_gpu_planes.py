"""GPU parity of the multi-plane paths against the FP64 oracle.

* Multi-plane GS (averaged projections over P Fresnel planes): one teacher-forced step on the
  row-major field and on fields tiled in column strips, and the plane-mean NMSE curve within 1 %.
* Gradient descent (hand-written Wirtinger adjoint): the GPU gradient against FP64 central finite
  differences of the oracle's loss (rel <= 1e-3, 64x64, P = 3) and against the oracle's analytic
  gradient (rel-L2 <= 1e-4); the loss per plane; Adam steps; the autograd front end.
"""
import numpy as np
import pytest

import synth
from oracle import gd as ogd
from oracle import gs as ogs
from oracle import optics, project
from tests.helpers import check_continuous_phase, check_levels, check_nmse, cuda_device, rel_l2

LAM, PITCH = 532e-9, 8e-6
ZS = (0.08, 0.10, 0.12)


def _fresnel(hg, zs=ZS):
    return dict(propagation=hg.HG_FRESNEL, wavelength_m=LAM, pitch_m=PITCH, z_m=list(zs))


def _intensity_targets(n, seed):
    ts = []
    for p in range(3):
        t = synth.spots_target(n, n, 12, seed=seed + p).astype(np.float64) ** 2
        ts.append((t / np.sqrt(np.sum(t * t))).astype(np.float32))
    return ts


# ------------------------------------------------------------------ multi-plane GS


@pytest.mark.gpu
@pytest.mark.parametrize("levels,n,width", [(0, 64, None), (4, 64, None), (0, 256, 0), (0, 256, 2), (4, 256, 4),
                                            (0, 256, 8), (4, 512, 2)])
def test_multiplane_gs_one_step(levels, n, width):
    """One step on the default field layout (width None), the row-major field (0) and fields tiled in
    column strips of 2, 4 and 8."""
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    amps = [np.sqrt(t) for t in _intensity_targets(n, 10)]
    cs = [optics.chirp(n, n, LAM, PITCH, z) for z in ZS]
    rng = np.random.default_rng(3)
    phi0 = (2 * np.pi * rng.integers(0, levels, (n, n)) / levels).astype(np.float32) if levels else \
        synth.uniform_phase(n, n, seed=4)
    with hg.Plan([n], [n], quant_levels=levels, **_fresnel(hg)) as plan:
        if width is not None:
            plan.set_strip_width(0, width)
            assert plan.strip_width(0) == width
        ta = [torch.from_numpy(a).to(dev) for a in amps]
        tp = torch.from_numpy(phi0).to(dev)
        ph = torch.zeros((n, n), dtype=torch.float32, device=dev)
        lv = torch.zeros((n, n), dtype=torch.uint8, device=dev) if levels else None
        nm = torch.zeros((1, 2), dtype=torch.float32, device=dev)
        plan.gs(ta, 1, init_phase=[tp], phase_out=[ph], level_out=None if lv is None else [lv], nmse_out=nm)
        plan.sync()
    a64 = [a.astype(np.float64) for a in amps]
    h0, _ = project.slm_project(np.exp(1j * phi0.astype(np.float64)), levels)
    # oracle: one averaged-projection step from h0, with its pre-projection field
    from oracle.fft import fft2

    acc = np.zeros((n, n), dtype=np.complex128)
    for a, c in zip(a64, cs):
        r = fft2(h0 * c)
        acc += np.conj(c) * fft2(project.amplitude_replace(r, ogs.scaled_amplitude(a)), inverse=True)
    g = acc / 3
    h1, q1 = project.slm_project(g, levels)
    if levels:
        check_levels(lv.cpu().numpy(), q1, g, levels)
    else:
        check_continuous_phase(ph.cpu().numpy(), g, h1)
    ref = ogs.multiplane_gs(a64, phi0.astype(np.float64), 1, cs, levels)
    check_nmse(nm.cpu().numpy()[0, :1], ref["nmse"][:1], rtol=1e-3)


@pytest.mark.gpu
@pytest.mark.parametrize("width", [None, 0])
def test_multiplane_gs_curve_256(width):
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    n, iters = 256, 10
    amps = [np.sqrt(t) for t in _intensity_targets(n, 20)]
    cs = [optics.chirp(n, n, LAM, PITCH, z) for z in ZS]
    phi0 = synth.uniform_phase(n, n, seed=21)
    with hg.Plan([n], [n], **_fresnel(hg)) as plan:
        if width is not None:
            plan.set_strip_width(0, width)
        nm = torch.zeros((1, iters + 1), dtype=torch.float32, device=dev)
        plan.gs([torch.from_numpy(a).to(dev) for a in amps], iters, init_phase=[torch.from_numpy(phi0).to(dev)],
                nmse_out=nm)
        plan.sync()
    ref = ogs.multiplane_gs([a.astype(np.float64) for a in amps], phi0.astype(np.float64), iters, cs)
    check_nmse(nm.cpu().numpy()[0], ref["nmse"])


@pytest.mark.gpu
def test_multiplane_gs_mixed_size_batch_matches_single_items():
    """Items of two sizes in one multi-plane plan (each size class on its own field layout, targets
    re-laid out per item and plane): every item's phase and NMSE curve equal those of a one-item
    plan bit for bit, and the start's NMSE matches the oracle."""
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    sizes, zs, iters = [256, 512, 256], (0.08, 0.12), 3
    amps = [[np.sqrt(t) for t in _intensity_targets(n, 30 + 10 * i)[:2]] for i, n in enumerate(sizes)]
    phis = [synth.uniform_phase(n, n, seed=31 + 10 * i) for i, n in enumerate(sizes)]

    def run(plan, items):
        ta = [torch.from_numpy(a).to(dev) for i in items for a in amps[i]]
        tp = [torch.from_numpy(phis[i]).to(dev) for i in items]
        ph = [torch.zeros((sizes[i], sizes[i]), dtype=torch.float32, device=dev) for i in items]
        nm = torch.zeros((len(items), iters + 1), dtype=torch.float32, device=dev)
        plan.gs(ta, iters, init_phase=tp, phase_out=ph, nmse_out=nm)
        plan.sync()
        return [x.cpu().numpy() for x in ph], nm.cpu().numpy()

    with hg.Plan(sizes, sizes, **_fresnel(hg, zs)) as plan:
        widths = [plan.strip_width(i) for i in range(3)]
        ph_b, nm_b = run(plan, [0, 1, 2])
    for i, n in enumerate(sizes):
        with hg.Plan([n], [n], **_fresnel(hg, zs)) as plan:
            assert plan.strip_width(0) == widths[i]
            ph1, nm1 = run(plan, [i])
        assert np.array_equal(ph1[0], ph_b[i])
        assert np.array_equal(nm1[0], nm_b[i])
    cs = [optics.chirp(512, 512, LAM, PITCH, z) for z in zs]
    ref = ogs.multiplane_gs([a.astype(np.float64) for a in amps[1]], phis[1].astype(np.float64), 1, cs)
    check_nmse(nm_b[1][:1], ref["nmse"][:1], rtol=1e-3)


# ------------------------------------------------------------------ gradient descent


def _gd_setup(n, seed):
    ts = _intensity_targets(n, seed)
    cs = [optics.chirp(n, n, LAM, PITCH, z) for z in ZS]
    phi = synth.uniform_phase(n, n, seed=seed + 9)
    return ts, cs, phi


def _gpu_grad(hg, dev, ts, phi, zs=ZS):
    import torch

    n = phi.shape[0]
    with hg.Plan([n], [n], **_fresnel(hg, zs)) as plan:
        tt = [torch.from_numpy(t).to(dev) for t in ts]
        tp = torch.from_numpy(phi).to(dev)
        loss = torch.zeros((1, len(zs) + 1), dtype=torch.float32, device=dev)
        grad = torch.zeros_like(tp)
        hg.hg_gd_forward(plan.handle, [tp], tt, loss)
        hg.hg_gd_backward(plan.handle, [tp], tt, [grad])
        plan.sync()
        return grad.cpu().numpy().astype(np.float64), loss.cpu().numpy()[0]


@pytest.mark.gpu
def test_gd_gradient_vs_oracle_and_finite_differences():
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    ts, cs, phi = _gd_setup(64, 90)
    g_gpu, loss = _gpu_grad(hg, dev, ts, phi)
    t64 = [t.astype(np.float64) for t in ts]
    p64 = phi.astype(np.float64)
    l_ref, lp_ref, g_ref = ogd.loss_and_grad(p64, t64, cs)
    check_nmse(loss, list(lp_ref) + [l_ref], rtol=1e-4)
    assert rel_l2(g_gpu, g_ref) <= 1e-4
    # FP64 central finite differences of the oracle loss on sampled pixels
    rng = np.random.default_rng(1)
    idx = rng.choice(p64.size, 64, replace=False)
    eps = 1e-6
    fd = []
    for k in idx:
        e = np.zeros(p64.size)
        e[k] = eps
        e = e.reshape(p64.shape)
        fd.append((ogd.loss_only(p64 + e, t64, cs) - ogd.loss_only(p64 - e, t64, cs)) / (2 * eps))
    fd = np.array(fd)
    assert np.linalg.norm(g_gpu.ravel()[idx] - fd) / np.linalg.norm(fd) <= 1e-3


@pytest.mark.gpu
def test_gd_fourier_single_plane_gradient():
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    n = 128
    t = _intensity_targets(n, 40)[0]
    phi = synth.uniform_phase(n, n, seed=41)
    with hg.Plan([n], [n]) as plan:
        tp = torch.from_numpy(phi).to(dev)
        tt = [torch.from_numpy(t).to(dev)]
        grad = torch.zeros_like(tp)
        loss = torch.zeros((1, 2), dtype=torch.float32, device=dev)
        hg.hg_gd_forward(plan.handle, [tp], tt, loss)
        hg.hg_gd_backward(plan.handle, [tp], tt, [grad])
        plan.sync()
    l_ref, _, g_ref = ogd.loss_and_grad(phi.astype(np.float64), [t.astype(np.float64)], [np.ones((n, n))])
    assert abs(loss.cpu().numpy()[0, 1] - l_ref) <= 1e-4 * l_ref
    assert rel_l2(grad.cpu().numpy(), g_ref) <= 1e-4


@pytest.mark.gpu
def test_gd_adam_steps_track_oracle():
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    n, steps = 64, 25
    ts, cs, phi = _gd_setup(n, 60)
    ref = ogd.gd_run(phi.astype(np.float64), [t.astype(np.float64) for t in ts], cs, steps, 0.05)
    with hg.Plan([n], [n], **_fresnel(hg)) as plan:
        tp = torch.from_numpy(phi).to(dev)
        tt = [torch.from_numpy(t).to(dev) for t in ts]
        m = torch.zeros_like(tp)
        v = torch.zeros_like(tp)
        loss = torch.zeros((steps, 4), dtype=torch.float32, device=dev)
        for k in range(steps):
            plan.gd_step([tp], tt, [m], [v], k + 1, 0.05, loss_out=loss[k])
        plan.sync()
        got = loss.cpu().numpy()[:, 3]
    check_nmse(got, ref["loss"])
    assert got[-1] < 0.5 * got[0]


@pytest.mark.gpu
def test_gd_first_adam_step_matches_oracle_update():
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    ts, cs, phi = _gd_setup(64, 70)
    t64 = [t.astype(np.float64) for t in ts]
    with hg.Plan([64], [64], **_fresnel(hg)) as plan:
        tp = torch.from_numpy(phi).to(dev)
        m = torch.zeros_like(tp)
        v = torch.zeros_like(tp)
        grad = torch.zeros_like(tp)
        plan.gd_step([tp], [torch.from_numpy(t).to(dev) for t in ts], [m], [v], 1, 0.05, grad_out=[grad])
        plan.sync()
    g_gpu = grad.cpu().numpy().astype(np.float64)
    # the update applied is Adam's from the GPU gradient (checked against the oracle above)
    phi1, m1, v1 = ogd.adam_update(phi.astype(np.float64), g_gpu, 0.0 * g_gpu, 0.0 * g_gpu, 1, 0.05)
    assert np.max(np.abs(tp.cpu().numpy() - phi1)) <= 1e-5
    assert rel_l2(m.cpu().numpy(), m1) <= 1e-6
    _, _, g_ref = ogd.loss_and_grad(phi.astype(np.float64), t64, cs)
    assert rel_l2(g_gpu, g_ref) <= 1e-4


@pytest.mark.gpu
def test_autograd_front_end():
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    ts, cs, phi = _gd_setup(64, 80)
    with hg.Plan([64], [64], **_fresnel(hg)) as plan:
        tt = [torch.from_numpy(t).to(dev) for t in ts]
        tp = torch.from_numpy(phi).to(dev).requires_grad_(True)
        loss = hg.hologram_loss(plan, tp, tt)
        (3.0 * loss).backward()
        torch.cuda.synchronize()
    l_ref, _, g_ref = ogd.loss_and_grad(phi.astype(np.float64), [t.astype(np.float64) for t in ts], cs)
    assert abs(loss.item() - l_ref) <= 1e-4 * l_ref
    assert rel_l2(tp.grad.cpu().numpy(), 3.0 * g_ref) <= 1e-4
