"""GPU parity of the bare Fourier / Fresnel transforms (hg_propagate) against the FP64 oracle.

Sizes span one tile, several tiles, ragged tails (widths not a multiple of the column strip, heights
not a multiple of the row tile), mixed radices and the largest supported lengths, and lengths that run
on the generic kernels (any 2^a 3^b 5^c up to 4096, down to length 1).  Bar: relative L2
error <= 1e-4 on identical inputs.
"""
import numpy as np
import pytest

from oracle import optics
from tests.helpers import FIELD_TOL, cuda_device, rel_l2

LAM, PITCH = 532e-9, 8e-6

SIZES = [(8, 8), (16, 32), (64, 64), (256, 256), (12, 15), (30, 60), (120, 64), (15, 8), (60, 1920),
         (864, 1536), (1080, 1920), (2048, 2048), (4096, 256), (512, 4096),
         # common SLM sizes (compiled since), then lengths without a compiled instance (the generic
         # kernels), alone and mixed with compiled ones: odd and degenerate sizes, the longest ones
         (1024, 1280), (720, 1280), (2160, 3840), (1000, 1200), (1500, 2000), (1000, 1125), (1, 1), (1, 8),
         (3, 5), (27, 125), (243, 100), (2, 4000), (4050, 6), (3125, 18)]


def _field(h, w, seed):
    r = np.random.default_rng(seed)
    return (r.standard_normal((h, w)) + 1j * r.standard_normal((h, w))).astype(np.complex64)


@pytest.mark.gpu
@pytest.mark.parametrize("hw", SIZES)
@pytest.mark.parametrize("fresnel", [False, True])
def test_propagate_matches_oracle(hw, fresnel):
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    h, w = hw
    x = _field(h, w, h * 7 + w)
    z = 0.1
    kw = dict(propagation=hg.HG_FRESNEL, wavelength_m=LAM, pitch_m=PITCH, z_m=[z]) if fresnel else {}
    c = optics.chirp(h, w, LAM, PITCH, z) if fresnel else None
    with hg.Plan([h], [w], **kw) as plan:
        xin = torch.from_numpy(x).to(dev)
        for direction in (1, -1):
            out = torch.empty_like(xin)
            plan.propagate([xin], [out], direction=direction)
            torch.cuda.synchronize()
            ref = optics.propagate(x.astype(np.complex128), c, inverse=direction < 0)
            err = rel_l2(out.cpu().numpy(), ref)
            assert err <= FIELD_TOL, f"{hw} dir {direction}: rel L2 {err:.3e}"
        # in place, round trip
        y = xin.clone()
        plan.propagate([y], [y], direction=1)
        plan.propagate([y], [y], direction=-1)
        torch.cuda.synchronize()
        assert rel_l2(y.cpu().numpy(), x) <= FIELD_TOL


@pytest.mark.gpu
def test_propagate_mixed_size_batch():
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    sizes = [(64, 64), (256, 256), (64, 64), (30, 120), (64, 64)] + [(16, 16)] * 40  # > one launch chunk
    xs = [_field(h, w, 100 + i) for i, (h, w) in enumerate(sizes)]
    with hg.Plan([s[0] for s in sizes], [s[1] for s in sizes]) as plan:
        xin = [torch.from_numpy(x).to(dev) for x in xs]
        outs = [torch.empty_like(t) for t in xin]
        plan.propagate(xin, outs, direction=1)
        torch.cuda.synchronize()
    for x, o in zip(xs, outs):
        assert rel_l2(o.cpu().numpy(), optics.propagate(x.astype(np.complex128))) <= FIELD_TOL


@pytest.mark.gpu
def test_propagate_rejects_host_buffers_and_bad_direction():
    import torch

    import paper_2006_10509_gb300 as hg

    dev = cuda_device()
    with hg.Plan([64], [64]) as plan:
        host = torch.zeros((64, 64), dtype=torch.complex64)
        dev_t = torch.zeros((64, 64), dtype=torch.complex64, device=dev)
        with pytest.raises(hg.HologenError) as e:
            plan.propagate([host], [dev_t])
        assert e.value.status == hg.HG_ERR_INVALID_ARG
        with pytest.raises(hg.HologenError):
            plan.propagate([dev_t], [dev_t], direction=0)
