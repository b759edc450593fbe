"""Every hologram size whose sides are products of 2, 3 and 5 (up to 4096): the boundary accepts them
all, and the lengths without a compiled instance run on the generic kernels.  The single-plane paths
at such sizes are covered by the propagation, GS, OSPR, MRAF, HIO, DBS and display-order tests (their
size lists include generic lengths); here:

* multi-plane GS (averaged projections, one launch per plane on the generic row lengths): one
  teacher-forced step and the NMSE curve against the FP64 oracle;
* gradient descent: per-plane loss and gradient against the oracle, Adam steps tracking it;
* a batch mixing generic and compiled lengths: bitwise what one-item plans give;
* the graph-replayed run equal to the stream-launched one.
"""
import numpy as np
import pytest

import synth
from oracle import gd as ogd
from oracle import gs as ogs
from oracle import optics, project
from oracle.fft import fft2
from oracle.metrics import nmse
from tests.helpers import check_continuous_phase, check_levels, check_nmse, cuda_device, rel_l2

LAM, PITCH = 532e-9, 8e-6
ZS = (0.03, 0.04, 0.05)


def _fresnel(hg, zs=ZS):
    return dict(propagation=hg.HG_FRESNEL, wavelength_m=LAM, pitch_m=PITCH, z_m=list(zs))


def _intensities(h, w, seed, planes=3):
    ts = []
    for p in range(planes):
        t = synth.spots_target(h, w, 8, seed=seed + p).astype(np.float64) ** 2
        ts.append((t / np.sqrt(np.sum(t * t))).astype(np.float32))
    return ts


@pytest.mark.gpu
@pytest.mark.parametrize("h, w, levels", [(100, 120, 0), (90, 1280, 4), (1000, 64, 0), (60, 1000, 4)])
def test_multiplane_gs_generic_lengths_one_step_and_curve(h, w, levels):
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    amps = [np.sqrt(t) for t in _intensities(h, w, 31)]
    cs = [optics.chirp(h, w, LAM, PITCH, z) for z in ZS]
    rng = np.random.default_rng(32)
    phi0 = (2 * np.pi * rng.integers(0, levels, (h, w)) / levels).astype(np.float32) if levels else \
        synth.uniform_phase(h, w, seed=33)
    n_iter = 6
    outs = []
    with hg.Plan([h], [w], quant_levels=levels, **_fresnel(hg)) as plan:
        ta = [torch.from_numpy(a).to(dev) for a in amps]
        tp = torch.from_numpy(phi0).to(dev)
        for it in (1, n_iter):
            ph = torch.zeros((h, w), dtype=torch.float32, device=dev)
            lv = torch.zeros((h, w), dtype=torch.uint8, device=dev) if levels else None
            nm = torch.zeros((1, it + 1), dtype=torch.float32, device=dev)
            plan.gs(ta, it, init_phase=[tp], phase_out=[ph], level_out=None if lv is None else [lv], nmse_out=nm)
            plan.sync()
            outs.append((ph.cpu().numpy(), None if lv is None else lv.cpu().numpy(), nm.cpu().numpy()[0]))
    a64 = [a.astype(np.float64) for a in amps]
    h0, _ = project.slm_project(np.exp(1j * phi0.astype(np.float64)), levels)
    acc = np.zeros((h, w), dtype=np.complex128)
    for a, c in zip(a64, cs):
        acc += np.conj(c) * fft2(project.amplitude_replace(fft2(h0 * c), ogs.scaled_amplitude(a)), inverse=True)
    g = acc / 3
    h1, q1 = project.slm_project(g, levels)
    if levels:
        check_levels(outs[0][1], q1, g, levels)
    else:
        check_continuous_phase(outs[0][0], g, h1)
    ref = ogs.multiplane_gs(a64, phi0.astype(np.float64), n_iter, cs, levels)
    check_nmse(outs[0][2][:1], ref["nmse"][:1], rtol=1e-3)
    if not levels:  # quantised trajectories part at level flips; continuous ones are stable here
        check_nmse(outs[1][2], ref["nmse"])


@pytest.mark.gpu
@pytest.mark.parametrize("h, w, zs", [(100, 120, ZS), (45, 1280, ZS[:2]), (128, 27, None), (45, 1000, ZS[:2])])
def test_gd_generic_lengths_gradient_and_adam(h, w, zs):
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    P = len(zs) if zs else 1
    ts = _intensities(h, w, 41, P)
    cs = [optics.chirp(h, w, LAM, PITCH, z) for z in zs] if zs else [np.ones((h, w))]
    phi = synth.uniform_phase(h, w, seed=42)
    kw = _fresnel(hg, zs) if zs else {}
    steps = 8
    with hg.Plan([h], [w], **kw) as plan:
        tt = [torch.from_numpy(t).to(dev) for t in ts]
        tp = torch.from_numpy(phi).to(dev)
        loss = torch.zeros((1, P + 1), dtype=torch.float32, device=dev)
        grad = torch.zeros_like(tp)
        hg.hg_gd_forward(plan.handle, [tp], tt, loss)
        hg.hg_gd_backward(plan.handle, [tp], tt, [grad])
        m = torch.zeros_like(tp)
        v = torch.zeros_like(tp)
        curve = torch.zeros((steps, P + 1), dtype=torch.float32, device=dev)
        for k in range(steps):
            plan.gd_step([tp], tt, [m], [v], k + 1, 0.05, loss_out=curve[k])
        plan.sync()
    t64 = [t.astype(np.float64) for t in ts]
    l_ref, lp_ref, g_ref = ogd.loss_and_grad(phi.astype(np.float64), t64, cs)
    check_nmse(loss.cpu().numpy()[0], list(lp_ref) + [l_ref], rtol=1e-4)
    assert rel_l2(grad.cpu().numpy(), g_ref) <= 1e-4
    ref = ogd.gd_run(phi.astype(np.float64), t64, cs, steps, 0.05)
    check_nmse(curve.cpu().numpy()[:, P], ref["loss"])


SIZES = [(1024, 1280), (90, 100), (64, 64), (720, 1280), (90, 100), (27, 125), (512, 512), (3, 5)]


def _batch(hg, dev, sizes, n_iter, levels, graph=False, first=0):
    """Items first, first + 1, ... of SIZES' inputs (target seed 50 + index, start seed 60 + index)."""
    import torch

    targets = [synth.blur_target(h, w, 1.5, seed=50 + first + i) for i, (h, w) in enumerate(sizes)]
    phases = [synth.uniform_phase(h, w, seed=60 + first + i) for i, (h, w) in enumerate(sizes)]
    with hg.Plan([s[0] for s in sizes], [s[1] for s in sizes], quant_levels=levels) as plan:
        if graph:
            plan.set_graph(True)
        ta = [torch.from_numpy(t).to(dev) for t in targets]
        tp = [torch.from_numpy(p).to(dev) for p in phases]
        lv = [torch.zeros(s, dtype=torch.uint8, device=dev) for s in sizes]
        nm = torch.zeros((len(sizes), n_iter + 1), dtype=torch.float32, device=dev)
        for _ in range(2 if graph else 1):
            plan.gs(ta, n_iter, init_phase=tp, level_out=lv, nmse_out=nm)
        plan.sync()
        return [x.cpu().numpy() for x in lv], nm.cpu().numpy(), targets, phases


@pytest.mark.gpu
def test_batch_mixing_generic_and_compiled_lengths():
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    lv, nm, targets, phases = _batch(hg, dev, SIZES, 4, 4)
    for i in range(len(SIZES)):
        l1, n1, _, _ = _batch(hg, dev, [SIZES[i]], 4, 4, first=i)
        assert np.array_equal(l1[0], lv[i]), SIZES[i]
        assert np.array_equal(n1[0], nm[i]), SIZES[i]
    for i in (1, 5):  # two generic items against the oracle's curve
        ref = ogs.gs(targets[i].astype(np.float64), phases[i].astype(np.float64), 4, 4)
        check_nmse(nm[i], ref["nmse"])
    lg, ng, _, _ = _batch(hg, dev, SIZES, 4, 4, graph=True)
    assert all(np.array_equal(x, y) for x, y in zip(lg, lv))
    assert np.array_equal(ng, nm)


@pytest.mark.gpu
def test_generic_length_noalloc_matches_plan():
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    h, w = 750, 1200
    a = torch.from_numpy(synth.blur_target(h, w, 2.0, seed=71)).to(dev)
    p = torch.from_numpy(synth.uniform_phase(h, w, seed=72)).to(dev)
    ph = torch.zeros((h, w), dtype=torch.float32, device=dev)
    nm = torch.zeros((6,), dtype=torch.float32, device=dev)
    hg.hg_gs_run_noalloc(h, w, 0, a, p, 0, 5, ph, None, nm)
    ph2 = torch.zeros_like(ph)
    nm2 = torch.zeros((1, 6), dtype=torch.float32, device=dev)
    with hg.Plan([h], [w]) as plan:
        plan.gs([a], 5, init_phase=[p], phase_out=[ph2], nmse_out=nm2)
        plan.sync()
    assert torch.equal(ph, ph2) and torch.equal(nm, nm2[0])
