"""Host logic of bench.py, without a GPU: the reference arm's JSON line, the
roofline bookkeeping (bound selection, per-launch figures, measured traffic)
on a synthetic kernel profile, and the traffic table against the summaries it
cites."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_prints_one_line_with_the_contract_keys():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "heat1d_63", "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert str(d["cpu_baseline"]["cores"]) + " processes at once" in d["cpu_baseline"]["sample"]
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "heat1d_63"


class _FakeSolver:
    """Stands in for stmg.Solver: a level count and per-level class totals."""

    def __init__(self, levels, per_level):
        self.num_levels = levels
        self._pl = per_level

    def profile_level(self, cls, L):
        return self._pl.get((cls, L), {"launches": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0})


def _prof(**classes):
    return {k: {"launches": v[0], "ms": v[1], "bytes": v[2], "flops": v[3]} for k, v in classes.items()}


def test_roofline_takes_the_dominant_class_on_the_finest_level():
    from paper_1411_0519_gb300 import workloads
    w = workloads.WORKLOADS["heat2d_255"]
    pk = {"hbm_gbs": 6790.3, "src": "measured"}
    # finest level: 10 launches, 6 ms, 3.2 GB and 0.55 GFLOP each
    fs = _FakeSolver(11, {("smooth", 10): {"launches": 10, "ms": 6.0, "bytes": 3.2e10, "flops": 5.5e9}})
    prof = _prof(smooth=(40, 8.0, 3.6e10, 6.0e9), dst=(6, 7.0, 6.4e9, 1.2e10), residual=(10, 5.0, 1e10, 1e9))
    rf = bench.roofline(fs, prof, False, pk, w)
    assert rf["level"] == "finest" and rf["launches"] == 10
    assert rf["avg_launch_ms"] == pytest.approx(0.6)
    gbs = 3.2e10 / 6e-3 / 1e9
    assert rf["bound"] == "hbm" and rf["achieved"] == pytest.approx(gbs, rel=1e-3)
    assert rf["frac"] == pytest.approx(gbs / 6790.3, rel=1e-3)
    assert rf["alg_bytes_per_launch"] == pytest.approx(3.2e9)
    # measured traffic of the finest-level smoother, scaled from the profiled case to a launch here
    t = bench.traffic_table()["smooth/fp64/d2_n255_q2"]
    ndof = w["N"] * (w["p_t"] + 1) * w["n"] ** w["d"]
    assert rf["traffic"] == pytest.approx(t["bytes_per_dof"] * ndof)
    assert rf["traffic_gbs"] == pytest.approx(t["bytes_per_dof"] * ndof / 0.6e-3 / 1e9, rel=1e-3)
    assert rf["kernel"] == t["kernel"]
    # excluding the dominant class moves to the next one; with flops dominating the bound is the ALU
    fs2 = _FakeSolver(11, {("residual", 10): {"launches": 5, "ms": 4.0, "bytes": 1e8, "flops": 4.0e9}})
    rf2 = bench.roofline(fs2, prof, False, pk, w, exclude=("smooth", "dst"))
    assert rf2["bound"] == "alu" and rf2["unit"] == "TFLOP/s"
    assert rf2["frac"] == pytest.approx(4.0e9 / 4e-3 / 1e12 / bench.FP64_PEAK_TFLOPS, rel=1e-3)


def test_traffic_table_entries_cite_existing_summaries():
    table = bench.traffic_table()
    assert table, "profiles/traffic_per_dof.json is missing"
    kernel_of = {"smooth": "k_fsmooth", "residual": "k_fresidual", "dst": "k_dst_rows_reg"}
    for key, t in table.items():
        cls, prec, case = key.split("/")
        assert prec in ("fp64", "fp32") and case.startswith("d")
        assert t["bytes_per_dof"] > 0
        assert t["kernel"].startswith(kernel_of[cls]), (key, t["kernel"])
        assert os.path.exists(os.path.join(ROOT, t["summary"])), t["summary"]
        assert "dram__bytes_read.sum + dram__bytes_write.sum" in t["measured"]


def test_vcycle_times_leave_out_the_boundary_transforms():
    fs = _FakeSolver(3, {("smooth", 2): {"launches": 8, "ms": 12.0, "bytes": 0.0, "flops": 0.0},
                         ("residual", 2): {"launches": 4, "ms": 6.0, "bytes": 0.0, "flops": 0.0},
                         ("dst", 2): {"launches": 2, "ms": 9.0, "bytes": 0.0, "flops": 0.0}})
    prof = _prof(smooth=(10, 14.0, 6e9, 0), residual=(6, 7.0, 3e9, 0), dst=(2, 9.0, 5e9, 0))
    v = bench.vcycle_times(fs, prof, steps=3, iters=2, per_step_ms=20.0, pk={"hbm_gbs": 1000.0})
    ms = (20.0 - 9.0 / 3) / 2
    assert v["ms_per_cycle_without_transforms"] == pytest.approx(ms)
    assert v["finest_level_kernel_ms_per_cycle"] == pytest.approx((12.0 + 6.0) / 3 / 2)
    # the cycle's algorithmic bytes leave out the transforms too
    assert v["alg_bytes_per_cycle"] == pytest.approx(9e9 / 3 / 2)
    assert v["achieved_gbs"] == pytest.approx(9e9 / 3 / 2 / (ms / 1e3) / 1e9, rel=1e-3)
    assert v["frac"] == pytest.approx(v["achieved_gbs"] / 1000.0, rel=1e-3)


def test_vcycle_times_leave_out_both_transform_classes():
    """With the tensor-core transforms the boundary work is two classes (split pass 'dst' and tensor
    pass 'dst_tc'); neither counts toward the cycle."""
    fs = _FakeSolver(3, {("smooth", 2): {"launches": 8, "ms": 12.0, "bytes": 0.0, "flops": 0.0},
                         ("residual", 2): {"launches": 4, "ms": 6.0, "bytes": 0.0, "flops": 0.0}})
    prof = _prof(smooth=(10, 14.0, 6e9, 0), residual=(6, 7.0, 3e9, 0), dst=(2, 3.0, 5e9, 0),
                 dst_tc=(2, 6.0, 5e9, 1e15))
    v = bench.vcycle_times(fs, prof, steps=3, iters=2, per_step_ms=20.0, pk={"hbm_gbs": 1000.0})
    assert v["ms_per_cycle_without_transforms"] == pytest.approx((20.0 - 9.0 / 3) / 2)
    assert v["alg_bytes_per_cycle"] == pytest.approx(9e9 / 3 / 2)


def test_transform_note_reports_the_tensor_rate_against_the_measured_peak():
    prof = _prof(smooth=(10, 14.0, 6e9, 0), dst=(4, 2.0, 4e9, 0), dst_tc=(4, 6.0, 4e9, 9.0e12))
    note = bench.transform_note(prof, {}, {"bf16_tflops_sustained": 1500.0})
    assert note["tensor_tflops"] == pytest.approx(1500.0, rel=1e-6)      # 9e12 flop in 6 ms
    assert note["tensor_frac"] == pytest.approx(1.0, rel=1e-6)
    assert note["split_gbs"] == pytest.approx(4e9 / 2e-3 / 1e9, rel=1e-6)
    assert note["share_of_kernel_time"] == pytest.approx(8.0 / 22.0, abs=1e-3)
    # the FFT form (no tensor pass) keeps the double-float description
    fft = bench.transform_note(_prof(smooth=(10, 14.0, 6e9, 0), dst=(4, 8.0, 4e9, 1e9)), {})
    assert fft["arithmetic"].startswith("double-float")


def test_windowed_load_equals_the_slice_of_the_full_load():
    """The CPU baseline's workers draw only their own time steps of f."""
    import numpy as np
    from paper_1411_0519_gb300 import workloads
    full = workloads.uniform_load(2, 15, 1, 32, seed=4)
    for s0, s1 in [(0, 8), (8, 16), (24, 32), (5, 6)]:
        assert np.array_equal(workloads.uniform_load_steps(2, 15, 1, 32, s0, s1, seed=4), full[s0:s1])
