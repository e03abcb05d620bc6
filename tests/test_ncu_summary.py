"""The ncu summary writer (no GPU): kernel names are shortened without
losing parenthesised template arguments, a raw-page capture gives the
per-kernel lookup lines bench.py reads, and a launch list gives the shares."""
import csv

from paper_1810_00615_gb300 import ncu_summary as ns


def test_short_names_keep_template_arguments():
    assert ns.short_name("void aao::<unnamed>::k_matvec_fx<3, 0, 1, double, 0, (int)-1>"
                         "(const T4 *, double *, int)") == "k_matvec_fx<3, 0, 1, double, 0, (int)-1>"
    assert ns.short_name("void aao::fft::<unnamed>::k_fft4_inverseB<4096, 32, double>"
                         "(const aao::cx<float> *, T3 *, int)") == "k_fft4_inverseB<4096, 32, double>"
    assert ns.short_name("k_finish") == "k_finish"


def _write(path, rows):
    with open(path, "w", newline="") as f:
        csv.writer(f).writerows(rows)


def test_capture_summary_lines(tmp_path):
    hdr = ["Kernel Name", "gpu__time_duration.sum", "dram__bytes_read.sum", "dram__bytes_write.sum",
           "sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active",
           "sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active"]
    units = ["", "us", "Mbyte", "Kbyte", "%", "%"]
    row = ["void aao::<unnamed>::k_x<4096, 32>(float *)", "40.0", "72.5", "500", "29.2", "71.4"]
    _write(tmp_path / "raw.csv", [hdr, units, row])
    text = ns.capture_md(ns.read_raw(tmp_path / "raw.csv"), "t", "cmd", "abc", [("k_x<4096", "kx")])
    assert "source_digest: abc" in text and "## `k_x<4096, 32>` (launch 1)" in text
    assert "dram_bytes_per_launch: kx 73000000" in text
    assert "busiest_pipe_name: kx fp64" in text and "busiest_pipe_pct: kx 71.40" in text


def test_launch_list_shares(tmp_path):
    hdr = ["ID", "Kernel Name", "Block Size", "Grid Size", "Metric Name", "Metric Unit",
           "Metric Value"]
    rows = [hdr,
            ["0", "void k_a<1>(int)", "(128,1,1)", "(4,1,1)", "gpu__time_duration.sum", "nsecond", "3000"],
            ["1", "void k_b(int)", "(128,1,1)", "(4,1,1)", "gpu__time_duration.sum", "usecond", "1"],
            ["2", "void k_a<1>(int)", "(128,1,1)", "(4,1,1)", "gpu__time_duration.sum", "nsecond", "1000"]]
    _write(tmp_path / "l.csv", rows)
    text = ns.launches_md(tmp_path / "l.csv", "t", "cmd", "abc")
    assert "| `k_a<1>` | 2 | 4.0 | 2.0 | 80.0% |" in text
    assert "| `k_b` | 1 | 1.0 | 1.0 | 20.0% |" in text
