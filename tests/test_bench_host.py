"""Host logic of bench.py (no GPU): the mapping from kernel names to solve passes and
the per-launch counts it reads back from an ncu launch list."""
import csv
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture()
def bench(tmp_path, monkeypatch):
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    monkeypatch.setattr(mod, "COUNTS_FILE", str(tmp_path / "ncu_counts.txt"))
    return mod


def test_pass_names(bench):
    assert bench._pass_name("void k2_z_fwd<df32, double, 512>(ZArgs2)", {}) == "z_forward"
    assert bench._pass_name("void k2_z_inv<float, float, 512>(ZArgs2)", {}) == "z_inverse"
    assert bench._pass_name("void k2_line<df32, 512, 2, 3>(LArgs)", {}) == "x_multiply"
    assert bench._pass_name("void k2_line<df32, 512, 0, -1>(LArgs)", {}) == "y_forward"
    assert bench._pass_name("void k3_line<float, 512, 1>(PArgs)", {}) == "y_inverse"
    assert bench._pass_name("void k_twiddles(int, cpx<double> *)", {}) is None


def test_ingest_averages_per_launch_and_tags_source(bench, tmp_path, capsys):
    path = tmp_path / "launches_256_df32.csv"
    rows = []
    for i, (kern, t, rd, wr, fadd, fadd2) in enumerate([
            ("void k2_line<df32, 512, 2, 3>(LArgs)", 1000.0, 800.0, 500.0, 10.0, 20.0),
            ("void k2_line<df32, 512, 2, 3>(LArgs)", 1200.0, 820.0, 480.0, 10.0, 20.0)]):
        for m, v in (("gpu__time_duration.sum", t), ("dram__bytes_read.sum", rd), ("dram__bytes_write.sum", wr),
                     ("smsp__sass_thread_inst_executed_op_fadd_pred_on.sum", fadd),
                     ("smsp__sass_thread_inst_executed_op_fadd2_pred_on.sum", fadd2)):
            rows.append({"ID": str(i), "Kernel Name": kern, "Metric Name": m, "Metric Value": f"{v:,.0f}"})
    with open(path, "w", newline="") as f:
        f.write("==PROF== Connected to process 1\n")
        w = csv.DictWriter(f, fieldnames=["ID", "Kernel Name", "Metric Name", "Metric Value"])
        w.writeheader()
        w.writerows(rows)
    assert bench.ingest_ncu([str(path)]) == 0
    assert "x_multiply" in capsys.readouterr().out
    assert bench.ncu_count("x_multiply", "n256_df32", "dram_bytes") == pytest.approx(1300.0)
    assert bench.ncu_count("x_multiply", "n256_df32", "fp32_lane_ops") == pytest.approx(50.0)
    assert bench.ncu_count("y_forward", "n256_df32", "dram_bytes") is None
    # a row taken on other sources is ignored
    text = open(bench.COUNTS_FILE).read().replace(bench.source_hash(), "0123456789ab")
    open(bench.COUNTS_FILE, "w").write(text)
    assert bench.ncu_count("x_multiply", "n256_df32", "dram_bytes") is None
