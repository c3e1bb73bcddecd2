"""Host-side pieces of bench.py that need no GPU: the source hash that retires
a recorded ncu traffic figure when a kernel's translation unit changes, the
algorithmic bytes per sphere behind the roofline, the clock record's parsing
(which decides whether a run is rejected) and the peak fallback."""
import os
import shutil

import pytest

import bench


@pytest.fixture
def tree(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2307_13802_gb300", "csrc")
    dst = tmp_path / "paper_2307_13802_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return dst


def test_source_hash_follows_every_included_header(tree):
    h0 = bench._src_hash("k_mixed.cu")
    assert h0 == bench._src_hash("k_mixed.cu")
    # a file the unit does not include leaves the hash alone
    with open(tree / "k_neighbors.cu", "a") as f:
        f.write("\n// unrelated\n")
    assert bench._src_hash("k_mixed.cu") == h0
    # a header the unit includes changes it
    with open(tree / "susp_internal.h", "a") as f:
        f.write("\n// changed\n")
    h1 = bench._src_hash("k_mixed.cu")
    assert h1 != h0
    # so does one reached only through another header
    (tree / "extra.cuh").write_text("// nested\n")
    dc = tree / "device_common.cuh"
    dc.write_text(dc.read_text().replace('#include "susp_internal.h"',
                                         '#include "susp_internal.h"\n#include "extra.cuh"', 1))
    h2 = bench._src_hash("k_mixed.cu")
    (tree / "extra.cuh").write_text("// nested, changed\n")
    assert bench._src_hash("k_mixed.cu") not in (h0, h1, h2)
    h1 = bench._src_hash("k_mixed.cu")
    # and so does the unit itself
    with open(tree / "k_mixed.cu", "a") as f:
        f.write("\n// changed\n")
    assert bench._src_hash("k_mixed.cu") not in (h0, h1)


def test_algorithmic_bytes_per_sphere():
    # the method's work per sphere: mixed pair 100 + 4K + 48c, FP64 pair
    # 128 + 4K + 48c; integrators 244 (mixed) and 196 (FP64)
    K, c = 3.943, 1.894
    assert bench.algorithmic_bytes("pair", "mixed", K, c, True) == pytest.approx(
        100 + 4 * K + 48 * c)
    assert bench.algorithmic_bytes("pair", "mixed", K, c, False) == pytest.approx(
        100 + 4 * K)
    assert bench.algorithmic_bytes("pair", "fp64", K, c, True) == pytest.approx(
        128 + 4 * K + 48 * c)
    assert bench.algorithmic_bytes("integrate", "mixed", K, c, True) == 244.0
    assert bench.algorithmic_bytes("integrate", "fp64", K, c, True) == 196.0
    # the library's own layout: mixed pair 64 + 4 + 4K + 32 + 16 + 48c
    assert bench.layout_bytes("pair", "mixed", K, c, True) == pytest.approx(
        64 + 4 + 4 * K + 32 + 16 + 48 * c)
    # integrator: state 96 + forces 32 + cell and tag 8 read, state 96 +
    # position and velocity mirrors 48 + cleared forces 32 written
    assert bench.layout_bytes("integrate", "mixed", K, c, True) == 312.0


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_record_median_maximum_and_active_reasons():
    ck = bench.Clocks(0)
    ck.proc = _Proc()
    # sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    ck.tmp.write("2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "garbage line\n")
    out = ck.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}
    ck = bench.Clocks(0)
    ck.proc = _Proc()
    ck.tmp.write("1500, 2070, 700.0, 0x8, Active, Not Active, Active, Not Active\n")
    out = ck.stop()
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    ck = bench.Clocks(0)
    assert ck.stop() is None            # nvidia-smi never started
    os.unlink(ck.tmp.name)


def test_peak_falls_back_without_a_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6795.8}')
    assert bench.peaks() == (6795.8, "measured")
