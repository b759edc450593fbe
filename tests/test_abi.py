"""Boundary tests that need no GPU: the library builds and loads, exports exactly the entry points
declared in include/hologen.h, and rejects bad arguments on the host before touching a device."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hg():
    from __graft_entry__ import build

    build()
    import paper_2006_10509_gb300 as m

    m.load()
    return m


def _declared():
    with open(os.path.join(ROOT, "include", "hologen.h")) as f:
        text = f.read()
    return set(re.findall(r"HG_API\s+[\w\s\*]+?\b(hg_\w+)\s*\(", text))


def test_exports_match_header(hg):
    declared = _declared()
    assert {"hg_plan_create", "hg_plan_destroy", "hg_propagate", "hg_gs_run"} <= declared
    out = subprocess.run(["nm", "-D", "--defined-only", hg.lib_path()], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.split()[-1].startswith("hg_")}
    assert exported == declared
    for name in declared:
        assert hasattr(hg.load(), name)


def test_status_strings_and_lengths(hg):
    assert hg.hg_status_string(0) == "HG_OK"
    assert hg.hg_status_string(2) == "HG_ERR_UNSUPPORTED_SIZE"
    assert hg.hg_status_string(99) == "HG_ERR_UNKNOWN"
    for n in (8, 16, 256, 1080, 1920, 2048, 4096, 15, 864):
        assert hg.hg_supported_length(n)
    for n in (0, 7, 4097, 8192, -4, 14, 4095):
        assert not hg.hg_supported_length(n)


def test_supported_lengths_are_every_235_smooth_length_up_to_4096(hg):
    # compiled instances and the generic kernels together: exactly n = 2^a 3^b 5^c, 1 <= n <= 4096
    def smooth(n):
        for p in (2, 3, 5):
            while n % p == 0:
                n //= p
        return n == 1

    got = [n for n in range(0, 4200) if hg.hg_supported_length(n)]
    want = [n for n in range(1, 4097) if smooth(n)]
    assert got == want and len(want) == 137


@pytest.mark.parametrize(
    "kwargs, status",
    [
        (dict(heights=[], widths=[]), 1),
        (dict(heights=[64], widths=[112]), 2),
        (dict(heights=[7], widths=[64]), 2),
        (dict(heights=[64], widths=[64], propagation=5), 1),
        (dict(heights=[64], widths=[64], quant_levels=1), 1),
        (dict(heights=[64], widths=[64], quant_levels=300), 1),
        (dict(heights=[64], widths=[64], propagation=1, wavelength_m=0.0, pitch_m=8e-6, z_m=[0.1]), 1),
        (dict(heights=[64], widths=[64], propagation=1, wavelength_m=5e-7, pitch_m=8e-6, z_m=[-0.1]), 1),
        (dict(heights=[64], widths=[64], z_m=[0.1, 0.2]), 1),
        (dict(heights=[64], widths=[64], flags=4), 1),
    ],
)
def test_create_rejects_bad_descriptors(hg, kwargs, status):
    with pytest.raises(hg.HologenError) as e:
        hg.hg_plan_create(**kwargs)
    assert e.value.status == status


def test_null_plan_calls(hg):
    lib = hg.load()
    assert lib.hg_plan_destroy(None) == 0
    assert lib.hg_plan_sync(None) == 1
    assert lib.hg_propagate(None, 0, 1, None, None, None) == 1
    assert lib.hg_gs_run(None, None, None, 0, 1, None, None, None, None) == 1
    assert lib.hg_ospr_run(None, None, 1, 0, 0, None, None, None) == 1
    assert "NULL" in hg.hg_last_error()
    assert lib.hg_mraf_run(None, None, None, 0.5, None, 0, 1, None, None, None, None) == 1
    assert lib.hg_hio_run(None, None, None, 0.7, None, 0, 1, None, None, None, None) == 1
    assert lib.hg_dbs_run(None, None, None, 0, 1, None, None, None, None) == 1
    assert lib.hg_sa_run(None, None, None, 0, 1, 1e-3, 0.9, None, None, None, None) == 1
    assert lib.hg_plan_set_slm_levels(None, None, 0) == 1
    assert lib.hg_plan_set_illumination(None, None) == 1
    assert lib.hg_plan_set_strip_width(None, 0, 2) == 1
    assert lib.hg_plan_autotune(None, None) == 1
    assert "NULL" in hg.hg_last_error()
    assert lib.hg_gs_run_noalloc(4096, 4096, 0, None, None, 0, 1, None, None, None, None) == 2
    assert "1048576" in hg.hg_last_error()


def test_product_path_has_no_oracle_or_fallback():
    pkg = os.path.join(ROOT, "paper_2006_10509_gb300")
    for dirpath, _, files in os.walk(pkg):
        for name in files:
            if name.endswith(".py"):
                with open(os.path.join(dirpath, name)) as f:
                    src = f.read()
                assert "oracle" not in src.replace("no CPU fallback", ""), name
                assert "torch.fft" not in src, name
