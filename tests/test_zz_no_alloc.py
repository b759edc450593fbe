"""hg_gs_run_noalloc: Gerchberg-Saxton without device allocation, checked against hg_gs_run and the
FP64 oracle.

Callers that cannot call cudaMalloc (code inside a memory arena it does not own, plug-ins whose host
forbids allocation after start-up, real-time loops where an allocation could stall the device)
cannot create a plan, because hg_plan_create allocates the workspace.  hg_gs_run_noalloc gives them
the same GS for one Fourier hologram with its scratch in a static device array of the library.

* Two calls in a row (two sizes, so the shared scratch is reused with new tables), each compared
  with hg_gs_run on a plan whose field is row-major: the same kernels and the same order of the
  NMSE partial sums, so phases, levels and NMSE must be bitwise equal.
* The full capacity (1024 x 1024 = 2^20 pixels, the whole field part of the array): one
  teacher-forced 4-level step against the FP64 oracle, and the run against hg_gs_run.
* The branches a plain run does not take: no iteration (the start's projection is the output),
  the start drawn from the seed, no NMSE output.
* No device memory is reserved by a call after a warm-up call of the same size.

The file sorts last so that a -x run reaches it after every other test.
"""
import numpy as np
import pytest

import synth
from oracle import gs as ogs
from oracle import project
from oracle.fft import fft2
from oracle.metrics import nmse
from tests.helpers import check_levels, check_nmse, cuda_device


def _inputs(h, w, seed):
    return synth.blur_target(h, w, 2.0, seed=seed), synth.uniform_phase(h, w, seed=seed + 1)


def _plan_run(hg, dev, h, w, levels, ta, tp, seed, n_iter, nmse=True):
    """hg_gs_run on a one-item plan with a row-major field (the kernels hg_gs_run_noalloc uses)."""
    import torch

    ph = torch.zeros((h, w), dtype=torch.float32, device=dev)
    lv = torch.zeros((h, w), dtype=torch.uint8, device=dev) if levels else None
    nm = torch.zeros((1, n_iter + 1), dtype=torch.float32, device=dev) if nmse else None
    with hg.Plan([h], [w], quant_levels=levels) as plan:
        plan.set_strip_width(0, 0)
        plan.gs([ta], n_iter, init_phase=None if tp is None else [tp], seed=seed, phase_out=[ph],
                level_out=None if lv is None else [lv], nmse_out=nm)
        plan.sync()
    return ph, lv, (nm[0] if nm is not None else None)


def _noalloc(hg, dev, h, w, levels, ta, tp, seed, n_iter, nmse=True):
    import torch

    ph = torch.zeros((h, w), dtype=torch.float32, device=dev)
    lv = torch.zeros((h, w), dtype=torch.uint8, device=dev) if levels else None
    nm = torch.zeros((n_iter + 1,), dtype=torch.float32, device=dev) if nmse else None
    hg.hg_gs_run_noalloc(h, w, levels, ta, tp, seed, n_iter, ph, lv, nm)
    return ph, lv, nm


def _assert_same(got, ref):
    for x, y in zip(got, ref):
        assert (x is None) == (y is None)
        if x is not None:
            assert torch_equal(x, y)


def torch_equal(x, y) -> bool:
    return bool(np.array_equal(x.cpu().numpy(), y.cpu().numpy()))


@pytest.mark.gpu
def test_noalloc_matches_plan_path_on_two_calls():
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    cases = [(512, 512, 4, 8, 21), (256, 1024, 0, 6, 31)]
    outs = []
    for h, w, levels, n_iter, seed in cases:
        a, phi = _inputs(h, w, seed)
        ta = torch.from_numpy(a).to(dev)
        tp = torch.from_numpy(phi).to(dev)
        outs.append((ta, tp, _noalloc(hg, dev, h, w, levels, ta, tp, 0, n_iter)))  # back-to-back calls
    torch.cuda.synchronize()
    for (h, w, levels, n_iter, _), (ta, tp, got) in zip(cases, outs):
        _assert_same(got, _plan_run(hg, dev, h, w, levels, ta, tp, 0, n_iter))


@pytest.mark.gpu
def test_noalloc_full_capacity_against_oracle_and_plan():
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    n, levels = 1024, 4  # 2^20 pixels: the field fills the whole field part of the scratch array
    a = synth.blur_target(n, n, 2.0, seed=41)
    q0 = np.random.default_rng(42).integers(0, levels, (n, n))
    phi0 = (2 * np.pi * q0 / levels).astype(np.float32)
    ta = torch.from_numpy(a).to(dev)
    tp = torch.from_numpy(phi0).to(dev)
    # one teacher-forced step from a start the projection leaves unchanged, against the oracle
    ph, lv, nm = _noalloc(hg, dev, n, n, levels, ta, tp, 0, 1)
    torch.cuda.synchronize()
    a64 = a.astype(np.float64)
    h0, _ = project.slm_project(np.exp(1j * phi0.astype(np.float64)), levels)
    st = ogs.gs_step(h0, a64, levels)
    q1 = lv.cpu().numpy()
    check_levels(q1, st["q"], st["g"], levels)
    e1 = nmse(np.abs(fft2(project.level_field(q1, levels))) ** 2, a64 * a64)  # of the GPU's own h_1
    check_nmse(nm.cpu().numpy(), [nmse(np.abs(fft2(h0)) ** 2, a64 * a64), e1], rtol=1e-3)
    # a longer run, bitwise against the plan path
    got = _noalloc(hg, dev, n, n, levels, ta, tp, 0, 5)
    _assert_same(got, _plan_run(hg, dev, n, n, levels, ta, tp, 0, 5))


@pytest.mark.gpu
def test_noalloc_branches_no_iteration_seeded_start_no_nmse():
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    h, w = 256, 512
    a, phi = _inputs(h, w, 51)
    ta = torch.from_numpy(a).to(dev)
    tp = torch.from_numpy(phi).to(dev)
    for levels, tp_in, seed, n_iter, with_nmse in [(4, tp, 0, 0, True),     # h_0 is the output
                                                   (0, None, 77, 4, True),  # start drawn from the seed
                                                   (2, tp, 0, 3, False),    # no NMSE: no finalise
                                                   (0, None, 5, 0, False)]:
        got = _noalloc(hg, dev, h, w, levels, ta, tp_in, seed, n_iter, with_nmse)
        ref = _plan_run(hg, dev, h, w, levels, ta, tp_in, seed, n_iter, with_nmse)
        _assert_same(got, ref)


@pytest.mark.gpu
def test_noalloc_call_reserves_no_device_memory():
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    h, w = 512, 1024
    a, phi = _inputs(h, w, 61)
    ta = torch.from_numpy(a).to(dev)
    tp = torch.from_numpy(phi).to(dev)
    ph = torch.zeros((h, w), dtype=torch.float32, device=dev)
    nm = torch.zeros((9,), dtype=torch.float32, device=dev)
    hg.hg_gs_run_noalloc(h, w, 0, ta, tp, 0, 8, ph, None, nm)  # warm-up: loads this size's kernels
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    hg.hg_gs_run_noalloc(h, w, 0, ta, tp, 0, 8, ph, None, nm)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0


@pytest.mark.gpu
def test_noalloc_rejects_oversize_and_host_buffers():
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    big = torch.zeros((2048, 2048), dtype=torch.float32, device=dev)
    with pytest.raises(hg.HologenError) as e:
        hg.hg_gs_run_noalloc(2048, 2048, 0, big, None, 0, 1)
    assert e.value.status == hg.HG_ERR_UNSUPPORTED_SIZE
    host = torch.zeros((64, 64), dtype=torch.float32)
    with pytest.raises(hg.HologenError) as e:
        hg.hg_gs_run_noalloc(64, 64, 0, host, None, 0, 1)
    assert e.value.status == hg.HG_ERR_INVALID_ARG
