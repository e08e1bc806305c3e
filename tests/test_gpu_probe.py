"""The issue-rate probe (bf_measure_issue_rates), the denominator of the walk kernels' roofline.

Each rate is lane-instructions per clock per SM of one instruction class.  The checks are
bounds any Blackwell SM satisfies: four sub-partitions of 16 to 32 integer lanes and 32
FP32 lanes each, and the SM count of the device query."""
from __future__ import annotations

import pytest

pytestmark = pytest.mark.gpu


def test_issue_rates_are_plausible():
    import torch
    from paper_1904_03621_gb300 import build
    build.build()
    from paper_1904_03621_gb300 import api
    r = api.issue_rates()
    props = torch.cuda.get_device_properties(0)
    assert r["sms"] == props.multi_processor_count
    for k in ("iadd3_lanes_per_clk", "lop3_lanes_per_clk", "vmnmx_lanes_per_clk"):
        assert 16.0 <= r[k] <= 132.0, (k, r[k])
    assert 32.0 <= r["ffma_lanes_per_clk"] <= 260.0, r
    assert 300.0 <= r["sm_clock_mhz"] <= 3000.0, r
    # the probe is repeatable within a few per cent
    r2 = api.issue_rates()
    assert abs(r2["lop3_lanes_per_clk"] - r["lop3_lanes_per_clk"]) <= 0.05 * r["lop3_lanes_per_clk"]


def test_issue_rates_rejects_small_workspace():
    import ctypes
    import torch
    from paper_1904_03621_gb300 import _lib
    lib = _lib.load()
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    r = _lib.IssueRates()
    assert lib.bf_measure_issue_rates(ws.data_ptr(), 16, ctypes.byref(r), None) == _lib.BF_EWORKSPACE
