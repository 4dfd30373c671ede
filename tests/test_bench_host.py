"""Host arithmetic of bench.py's report (no GPU): the issue roofline, the all-cores oracle
throughput and the per-launch figures read from the committed ncu summaries."""
import os

import pytest

import bench
import workloads as W


def test_issue_roofline_arithmetic(monkeypatch):
    """achieved = warp instructions per launch / launch time; peak = 4 schedulers x SMs x clock."""
    monkeypatch.setattr(bench, "ncu_summary", lambda fam, wl, key: 5.0e6 if key == "warp_inst_per_launch" else None)
    r = bench.issue_roofline("k_pint", "w", 0.0125, {"sm_mhz": 2000.0}, 150)
    assert r["achieved"] == pytest.approx(5.0e6 / 12.5e-6)
    assert r["peak"] == pytest.approx(4 * 150 * 2000e6)
    assert r["frac"] == pytest.approx(round(4.0e11 / 1.2e12, 4))
    assert bench.issue_roofline("k_pint", "w", 0.0125, None, 150) is None  # no clock sample


def test_ncu_summary_ignores_a_stale_capture(tmp_path, monkeypatch):
    """A summary taken on other kernels (source hash differs) yields no figure."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic_k_x_w.txt").write_text("csrc_sha256_16: 0000000000000000\ndram_bytes_per_launch: 123\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("k_x", "w") is None
    (prof / "traffic_k_x_w.txt").write_text(f"csrc_sha256_16: {bench.csrc_hash()}\ndram_bytes_per_launch: 123 (note)\n"
                                            "warp_inst_per_launch: 7 (from a capture)\n")
    assert bench.ncu_traffic("k_x", "w") == 123.0
    assert bench.ncu_summary("k_x", "w", "warp_inst_per_launch") == 7.0


def test_oracle_all_cores_counts_independent_solves():
    P = W.heat1d_forced(63, 16, seed=1)
    r = bench.oracle_all_cores(P, "tiny", 0.2)
    assert r["cores"] == (os.cpu_count() or 1)
    assert r["value"] > 0 and r["unit"] == bench.UNIT


def test_work_bytes_counts_only_the_final_loop_path_taken():
    """Solves that form the final loop by linearity skip the shifted solves of the final
    pass (their launches do no work) and run the elementwise pass; the others the reverse."""
    import bench

    def table():
        return [{"name": "pint_store_f32", "bytes": 100.0}, {"name": "final_comb", "bytes": 60.0},
                {"name": "pint_dots_f32", "bytes": 10.0}]

    all_lin = bench.work_bytes(table(), {"final_by_linearity": 4, "refine_sweeps": 4})
    assert [r["bytes"] for r in all_lin] == [0.0, 60.0, 10.0]
    none = bench.work_bytes(table(), {"final_by_linearity": 0, "refine_sweeps": 3})
    assert [r["bytes"] for r in none] == [100.0, 0.0, 10.0]
    half = bench.work_bytes(table(), {"final_by_linearity": 1, "refine_sweeps": 2})
    assert [r["bytes"] for r in half] == [50.0, 30.0, 10.0]
