"""Strip widths of the tiled GS field and the autotuner that picks them.

Every width a size class allows (2, 4, 8 or 16 columns, the row-major field, or -1, the whole run in
one thread-block cluster per item) runs the same FFTs on the same values, so quantised levels and
phases must be bitwise equal across widths; only the
grouping of the NMSE partial sums changes, so NMSE agrees to float rounding.  The autotuner must
pick one of the allowed widths and leave results unchanged.
"""
import numpy as np
import pytest

import synth
from tests.helpers import cuda_device

SIZES = [(512, 512), (2048, 1024), (1080, 1920), (256, 256)]


def _inputs(h, w, seed):
    return synth.blur_target(h, w, 2.0, seed=seed), synth.uniform_phase(h, w, seed=seed + 1)


def _run(hg, dev, plan, a, p, n_iter, levels):
    import torch

    h, w = a.shape
    ta, tp = torch.from_numpy(a).to(dev), torch.from_numpy(p).to(dev)
    ph = torch.zeros((h, w), dtype=torch.float32, device=dev)
    lv = torch.zeros((h, w), dtype=torch.uint8, device=dev) if levels else None
    nm = torch.zeros((1, n_iter + 1), dtype=torch.float32, device=dev)
    plan.gs([ta], n_iter, init_phase=[tp], phase_out=[ph], level_out=None if lv is None else [lv], nmse_out=nm)
    plan.sync()
    return ph.cpu().numpy(), None if lv is None else lv.cpu().numpy(), nm.cpu().numpy()[0]


@pytest.mark.gpu
@pytest.mark.parametrize("h, w", SIZES)
@pytest.mark.parametrize("levels", [0, 4])
def test_every_strip_width_gives_the_same_hologram(h, w, levels):
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    a, p = _inputs(h, w, 300 + h + levels)
    with hg.Plan([h], [w], quant_levels=levels) as plan:
        ref = _run(hg, dev, plan, a, p, 5, levels)
        tried = [plan.strip_width(0)]
        for width in (-1, 0, 2, 4, 8, 16):
            try:
                plan.set_strip_width(0, width)
            except hg.HologenError as e:
                assert e.status == hg.HG_ERR_INVALID_ARG
                continue
            tried.append(width)
            out = _run(hg, dev, plan, a, p, 5, levels)
            assert np.array_equal(out[0], ref[0]), width
            if levels:
                assert np.array_equal(out[1], ref[1]), width
            np.testing.assert_allclose(out[2], ref[2], rtol=1e-5, atol=1e-7)
        assert 0 in tried and len(set(tried)) >= 2


@pytest.mark.gpu
def test_autotune_picks_an_allowed_width_and_keeps_results():
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    sizes = [(512, 512), (1024, 1024), (864, 1536)]
    with hg.Plan([s[0] for s in sizes], [s[1] for s in sizes], quant_levels=4) as plan:
        defaults = [plan.strip_width(i) for i in range(len(sizes))]
        plan.autotune()
        tuned = [plan.strip_width(i) for i in range(len(sizes))]
    assert all(t in (-1, 0, 2, 4, 8, 16) for t in tuned)
    # the flag runs the same tuning at creation (cached choices: identical)
    with hg.Plan([s[0] for s in sizes], [s[1] for s in sizes], quant_levels=4, flags=hg.HG_PLAN_AUTOTUNE) as plan:
        assert [plan.strip_width(i) for i in range(len(sizes))] == tuned
        a, p = _inputs(512, 512, 77)
        out = _run_item(hg, dev, plan, sizes, 0, a, p)
    with hg.Plan([s[0] for s in sizes], [s[1] for s in sizes], quant_levels=4) as plan:
        ref = _run_item(hg, dev, plan, sizes, 0, a, p)
    assert np.array_equal(out[0], ref[0])
    np.testing.assert_allclose(out[1], ref[1], rtol=1e-5, atol=1e-7)
    assert len(defaults) == len(tuned)


def _run_item(hg, dev, plan, sizes, item, a, p):
    import torch

    ta = [torch.from_numpy(synth.blur_target(h, w, 2.0, seed=900 + i)).to(dev) for i, (h, w) in enumerate(sizes)]
    tp = [torch.from_numpy(synth.uniform_phase(h, w, seed=950 + i)).to(dev) for i, (h, w) in enumerate(sizes)]
    ta[item] = torch.from_numpy(a).to(dev)
    tp[item] = torch.from_numpy(p).to(dev)
    lv = [torch.zeros(s, dtype=torch.uint8, device=dev) for s in sizes]
    nm = torch.zeros((len(sizes), 5), dtype=torch.float32, device=dev)
    plan.gs(ta, 4, init_phase=tp, level_out=lv, nmse_out=nm)
    plan.sync()
    return lv[item].cpu().numpy(), nm[item].cpu().numpy()


@pytest.mark.gpu
def test_strip_widths_of_multiplane_plans():
    """Multi-plane GS tiles its field in strips of 2, 4 or 8 columns (or keeps it row-major); the
    16-column strips and the whole-run cluster kernel are single-plane only."""
    import paper_2006_10509_gb300 as hg

    with hg.Plan([256], [256], propagation=hg.HG_FRESNEL, wavelength_m=532e-9, pitch_m=8e-6,
                 z_m=[0.05, 0.1]) as plan:
        for w in (2, 4, 8, 0):
            plan.set_strip_width(0, w)
            assert plan.strip_width(0) == w
        for w in (16, hg.HG_STRIP_CLUSTER):
            with pytest.raises(hg.HologenError):
                plan.set_strip_width(0, w)
        plan.autotune()
        assert plan.strip_width(0) in (0, 2, 4, 8)


# ------------------------------------------------------------------ radix plans

PLAN_SIZES = [(2048, 2048, 0), (2048, 2048, 4), (1024, 1024, 8), (1080, 1920, 2), (864, 1536, 4)]


@pytest.mark.gpu
@pytest.mark.parametrize("h, w, levels", PLAN_SIZES)
def test_every_radix_plan_matches_the_oracle_one_step(h, w, levels):
    """Each (row plan, column plan) of a length pair with alternatives: one teacher-forced GS step
    against the FP64 oracle, and the NMSE of the start."""
    from oracle import gs as ogs
    from oracle import project
    from oracle.fft import fft2
    from oracle.metrics import nmse
    from tests.helpers import check_continuous_phase, check_levels, check_nmse

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    a = synth.blur_target(h, w, 2.0, seed=500 + levels)
    if levels:
        phi0 = (2 * np.pi * np.random.default_rng(501).integers(0, levels, (h, w)) / levels).astype(np.float32)
    else:
        phi0 = synth.uniform_phase(h, w, seed=502)
    a64 = a.astype(np.float64)
    h0, _ = project.slm_project(np.exp(1j * phi0.astype(np.float64)), levels)
    st = ogs.gs_step(h0, a64, levels)
    e0 = nmse(np.abs(fft2(h0)) ** 2, a64 * a64)
    with hg.Plan([h], [w], quant_levels=levels) as plan:
        assert plan.strip_width(0) > 0  # the default tiled field
        for pr in (0, 1):
            for pc in (0, 1):
                plan.set_radix_plan(0, pr, pc)
                assert plan.radix_plan(0) == (pr, pc)
                ph, lv, nm = _run(hg, dev, plan, a, phi0, 1, levels)
                if levels:
                    check_levels(lv, st["q"], st["g"], levels)
                else:
                    check_continuous_phase(ph, st["g"], st["h"])
                check_nmse(nm[:1], [e0], rtol=1e-3)


@pytest.mark.gpu
def test_radix_plan_choice_errors_and_autotune():
    import paper_2006_10509_gb300 as hg

    cuda_device()
    with hg.Plan([512, 2048], [512, 2048]) as plan:
        with pytest.raises(hg.HologenError) as e:
            plan.set_radix_plan(0, 1, 0)  # 512 has no alternative plan
        assert e.value.status == hg.HG_ERR_INVALID_ARG
        with pytest.raises(hg.HologenError) as e:
            plan.set_radix_plan(1, 2, 0)
        assert e.value.status == hg.HG_ERR_INVALID_ARG
        assert plan.radix_plan(1) == (0, 0)
        plan.autotune()
        assert plan.radix_plan(0) == (0, 0)
        assert plan.radix_plan(1)[0] in (0, 1) and plan.radix_plan(1)[1] in (0, 1)
