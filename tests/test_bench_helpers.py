"""Host logic of bench.py's roofline fields (no GPU): the measured-ceiling
fraction and its failure path, and the planner byte counts in the line."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


class _Props:
    multi_processor_count = 152


class _Cuda:
    @staticmethod
    def get_device_properties(device):
        return _Props()


class _Torch:
    cuda = _Cuda()


RATES = {"max_u16x2": 3.8, "viaddmax_u16x2": 1.97, "vimax3_u16x2": 1.93, "prmt": 2.0, "lop3": 2.0,
         "imad": 2.0, "step_cells_per_clk_sm": 6.0, "warps_per_sm_step": 48}


class _MP:
    def __init__(self, fail=False):
        self.fail = fail

    def mp_dp_op_rates(self, device):
        if self.fail:
            raise RuntimeError("no device")
        assert device == 0
        return dict(RATES)


def _m(waves=1):
    return {"clocks": {"sm_mhz": 2000.0}, "dp_ms": [10.0], "tot_ms": [20.0], "waves": waves,
            "code_bytes": 3_000, "moved": {"record_bytes": 10, "record_read_bytes": 40, "boundary_bytes": 20}}


def test_step_ceiling_fraction():
    cells = 6.0 * 152 * 2000e6 * 0.010 / 2        # half the ceiling's cells in 10 ms
    r = bench.with_ceilings({}, _MP(), _m(), cells, _Torch(), 0)["alu_ceilings"]
    assert abs(r["step_ceiling_gcups"] - 6.0 * 152 * 2.0) < 1e-6
    assert abs(r["frac_of_step_ceiling"] - 0.5) < 1e-9
    # several waves: the whole pipeline's time
    r = bench.with_ceilings({}, _MP(), _m(waves=3), cells, _Torch(), 0)["alu_ceilings"]
    assert abs(r["frac_of_step_ceiling"] - 0.25) < 1e-9


def test_ceiling_failure_is_reported_not_fatal():
    roof = bench.with_ceilings({"frac": 0.4}, _MP(fail=True), _m(), 1.0, _Torch(), 0)
    assert roof["frac"] == 0.4 and "error" in roof["alu_ceilings"]


def test_roofline_reports_planner_bytes():
    r = bench.roofline(_m(), 1500.0, _Torch(), 0, {})
    b = r["bytes_by_construction"]
    assert b["stream_written"] == 3_000 and b["stream_per_cell"] == 2.0
    assert b["records_written"] == 10 and b["records_read_by_strips"] == 40 and b["boundary_rows"] == 20
    assert r["bound"] == "alu" and r["ops_per_cell"] == 28
