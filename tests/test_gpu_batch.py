"""Mixed-size batched GS: one plan, many holograms of several sizes, size classes run concurrently,
optionally captured into one CUDA graph.

Every item of the batch must give exactly what a one-item plan gives for it (same kernels, same
reduction order: bitwise-equal levels and NMSE), the small items must match the FP64 oracle's NMSE
curve, graph replays must reproduce the first run, and the per-item latency stamps must be sane.
"""
import numpy as np
import pytest

import synth
from oracle import gs as ogs
from tests.helpers import check_nmse, cuda_device

SIZES = [(64, 64), (128, 256), (64, 64), (256, 128), (864, 1536), (128, 256), (512, 512), (512, 512)] + [(16, 16)] * 40


def _batch_inputs():
    targets = [synth.blur_target(h, w, 2.0, seed=700 + i) for i, (h, w) in enumerate(SIZES)]
    phases = [synth.uniform_phase(h, w, seed=900 + i) for i, (h, w) in enumerate(SIZES)]
    return targets, phases


def _run_plan(hg, dev, sizes, targets, phases, n_iter, levels, graph=False, repeat=1):
    import torch

    with hg.Plan([s[0] for s in sizes], [s[1] for s in sizes], quant_levels=levels) as plan:
        if graph:
            plan.set_graph(True)
        ta = [torch.from_numpy(t).to(dev) for t in targets]
        tp = [torch.from_numpy(p).to(dev) for p in phases]
        lv = [torch.zeros(s, dtype=torch.uint8, device=dev) for s in sizes]
        nm = torch.zeros((len(sizes), n_iter + 1), dtype=torch.float32, device=dev)
        outs = []
        for _ in range(repeat):
            plan.gs(ta, n_iter, init_phase=tp, level_out=lv, nmse_out=nm)
            plan.sync()
            outs.append(([x.cpu().numpy() for x in lv], nm.cpu().numpy().copy()))
        lat = plan.item_latency_ms()
        launches = plan.launch_count()
    return outs, lat, launches


@pytest.mark.gpu
def test_batch_matches_single_item_plans_and_oracle():
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    targets, phases = _batch_inputs()
    n_iter, levels = 6, 4
    (outs,), lat, _ = _run_plan(hg, dev, SIZES, targets, phases, n_iter, levels)
    lv_b, nm_b = outs
    for i in [0, 1, 3, 4, 6, 7, 8, 47]:
        (single,), _, _ = _run_plan(hg, dev, [SIZES[i]], [targets[i]], [phases[i]], n_iter, levels)
        assert np.array_equal(single[0][0], lv_b[i]), i
        assert np.array_equal(single[1][0], nm_b[i]), i
    for i in [0, 1, 3]:
        ref = ogs.gs(targets[i].astype(np.float64), phases[i].astype(np.float64), n_iter, levels)
        check_nmse(nm_b[i], ref["nmse"])
    assert all(x > 0 for x in lat) and max(lat) < 10_000


@pytest.mark.gpu
def test_batch_graph_replay_is_identical():
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    targets, phases = _batch_inputs()
    outs_g, lat, launches = _run_plan(hg, dev, SIZES, targets, phases, 5, 2, graph=True, repeat=3)
    (outs_s,), _, _ = _run_plan(hg, dev, SIZES, targets, phases, 5, 2)
    for lv, nm in outs_g:
        assert all(np.array_equal(a, b) for a, b in zip(lv, outs_s[0]))
        assert np.array_equal(nm, outs_s[1])
    assert launches > 0


@pytest.mark.gpu
def test_timed_graph_replay_reports_one_replay_and_same_results():
    """Graph mode with timing on: the timed graph (event nodes around every kernel) gives the same
    results as the untimed one, and the timing totals hold exactly the latest replay's launches."""
    import torch
    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    a = torch.from_numpy(synth.blur_target(512, 512, 2.0, seed=11)).to(dev)
    nm_plain = torch.zeros((1, 9), device=dev)
    nm_timed = torch.zeros((1, 9), device=dev)
    with hg.Plan([512], [512]) as plan:
        plan.set_graph(True)
        plan.gs([a], 8, seed=5, nmse_out=nm_plain)
        plan.set_timing(True)
        for _ in range(3):
            plan.gs([a], 8, seed=5, nmse_out=nm_timed)
        kt = plan.kernel_times()
        plan.set_timing(False)
        plan.gs([a], 8, seed=5, nmse_out=nm_plain)
        plan.sync()
    assert torch.equal(nm_plain, nm_timed)
    # one replay: 8 column passes + 8 row passes (+ init, final NMSE pass, finalise, target re-layout)
    assert kt["col_gs"][1] == 8 and kt["row_gs"][1] == 8
    assert all(ms > 0 for ms, _ in kt.values())


@pytest.mark.gpu
def test_batch_with_2048_and_4096_items():
    """A batch holding the two largest sizes of the mixed-size serving workload (and a 512^2 item):
    bitwise what one-item plans give, and one teacher-forced 4-level step of each large item
    against the FP64 oracle."""
    from oracle import project
    from tests.helpers import check_levels

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    sizes = [(4096, 4096), (2048, 2048), (512, 512), (2048, 2048)]
    levels = 4
    targets = [synth.blur_target(h, w, 2.0, seed=1700 + i) for i, (h, w) in enumerate(sizes)]
    rng = np.random.default_rng(1800)
    phases = [(2 * np.pi * rng.integers(0, levels, s) / levels).astype(np.float32) for s in sizes]
    (outs,), _, _ = _run_plan(hg, dev, sizes, targets, phases, 2, levels)
    for i in range(3):
        (single,), _, _ = _run_plan(hg, dev, [sizes[i]], [targets[i]], [phases[i]], 2, levels)
        assert np.array_equal(single[0][0], outs[0][i]), i
        assert np.array_equal(single[1][0], outs[1][i]), i
    (one,), _, _ = _run_plan(hg, dev, sizes, targets, phases, 1, levels)
    for i in (0, 1):
        a64 = targets[i].astype(np.float64)
        h0, _ = project.slm_project(np.exp(1j * phases[i].astype(np.float64)), levels)
        st = ogs.gs_step(h0, a64, levels)
        check_levels(one[0][i], st["q"], st["g"], levels)
