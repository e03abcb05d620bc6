"""Host-side pieces of bench.py, no GPU: figures from committed ncu summaries
are used only for the kernel code they were measured on, the nvidia-smi
clock samples are parsed into a median clock and the set of throttle
reasons, and the reference arm does no work on ranks other than 0 and
reports the steps it actually ran."""
import argparse
import io
import os
import tempfile
from contextlib import redirect_stdout

import pytest

import bench


def test_profile_figures_are_taken_only_for_the_current_kernel_code(tmp_path, monkeypatch):
    """A figure from an ncu summary is used only when the summary's
    source_digest line names the library sources built now; a summary of
    other kernel code gives None (no stale traffic in the bench line)."""
    from paper_1810_00615_gb300 import _build
    prof = tmp_path / "profiles"
    prof.mkdir()
    digest = _build._digest()
    (prof / "current.md").write_text(
        f"source_digest: {digest}\n\ndram_bytes_per_launch: kern_a 123456\n"
        "busiest_pipe_name: kern_a fp64\n")
    (prof / "stale.md").write_text(
        "source_digest: 0123abcd\n\ndram_bytes_per_launch: kern_b 999\n")
    (prof / "unstamped.md").write_text("dram_bytes_per_launch: kern_c 777\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("kern_a") == 123456.0
    assert bench._profile_value_text("busiest_pipe_name", "kern_a") == "fp64"
    assert bench._traffic("kern_b") is None
    assert bench._traffic("kern_c") is None
    assert bench._profile_value("dram_bytes_per_launch", "no_such_kernel") is None


def test_roofline_kernel_is_read_from_the_current_launch_list(tmp_path, monkeypatch):
    """The kernel shares that pick the roofline line come from a launch list
    of the current kernel code only."""
    from paper_1810_00615_gb300 import _build
    prof = tmp_path / "profiles"
    prof.mkdir()
    table = ("| kernel | launches | total us | mean us | share |\n|---|---|---|---|---|\n"
             "| `k_matvec_fx<2, 0, 1, double, 0, 1>` | 2 | 324.5 | 162.2 | 11.3% |\n"
             "| `k_fft4_inverseA_correct<4096, 32>` | 8 | 318.8 | 39.8 | 11.1% |\n")
    (prof / "launches_x.md").write_text(f"source_digest: {_build._digest()}\n\n" + table)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench._launch_list_shares()
    assert got == {"k_matvec_fx<2, 0, 1, double, 0, 1>": pytest.approx(0.113),
                   "k_fft4_inverseA_correct<4096, 32>": pytest.approx(0.111)}
    (prof / "launches_x.md").write_text("source_digest: 0123abcd\n\n" + table)
    assert bench._launch_list_shares() == {}


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler_with(lines):
    # a sample file beside this test; ClockSampler.stop() deletes it
    fd, path = tempfile.mkstemp(suffix=".csv", dir=os.path.dirname(os.path.abspath(__file__)))
    with os.fdopen(fd, "w") as f:
        f.write("".join(line + "\n" for line in lines))
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.path = path
    return s


def test_clock_samples_give_median_and_reasons():
    row = "0, {sm}, 2070, 900.1, 0x{act:x}, {hw}, Not Active, Not Active, {pc}"
    lines = [row.format(sm=sm, act=0, hw="Not Active", pc="Not Active")
             for sm in (2070, 2055, 2040)]
    lines.append(row.format(sm=1965, act=4, hw="Not Active", pc="Active"))
    lines.append("garbage line")
    sampler = _sampler_with(lines)
    got = sampler.stop()
    assert got["samples"] == 4
    assert got["sm_mhz"] == pytest.approx((2040 + 2055) / 2)
    assert got["sm_max_mhz"] == 2070
    assert got["reasons"] == ["sw_power_cap"]
    assert not os.path.exists(sampler.path)


def test_clock_samples_flag_hardware_slowdown():
    lines = ["0, 1500, 2070, 1300, 0x8, Active, Not Active, Active, Not Active"]
    got = _sampler_with(lines).stop()
    assert got["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_samples():
    got = _sampler_with([]).stop()
    assert got["sm_mhz"] is None and got["reasons"] == ["no samples"]
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]


def test_reference_arm_is_silent_on_other_ranks(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    def boom():
        raise AssertionError("rank 1 must not run the oracle")
    monkeypatch.setattr(bench, "_oracle_solve_seconds", boom)
    args = argparse.Namespace(gpus=2, steps=3, warmup=3, impl="reference")
    out = io.StringIO()
    with redirect_stdout(out):
        assert bench.run_reference(args) == 0
    assert out.getvalue() == ""


def test_reference_arm_prints_one_contract_line(monkeypatch):
    """Rank 0 of the reference arm times the oracle solve (here on a tiny
    workload) and prints one JSON line with the contract's keys."""
    import json
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setattr(bench, "N_SPACE", 31)
    monkeypatch.setattr(bench, "ELL", 32)
    args = argparse.Namespace(gpus=1, steps=3, warmup=3, impl="reference")
    out = io.StringIO()
    with redirect_stdout(out):
        assert bench.run_reference(args) == 0
    lines = [ln for ln in out.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["value"] == d["value"] == d["e2e"]["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["iters"] <= 2
    # the steps and warm-up actually run (at most 5 and 1), and what was asked
    assert d["steps"] == 3 and d["warmup"] == 1
    assert d["steps_requested"] == 3 and d["warmup_requested"] == 3
    assert "preconditioner" in d["config"]


def test_solution_error_against_time_stepping(monkeypatch):
    import synthetic as syn
    from oracle import system
    monkeypatch.setattr(bench, "N_SPACE", 31)
    monkeypatch.setattr(bench, "ELL", 16)
    u0 = syn.heat_initial(31, modes=8)
    S = system.heat(31, 16, 1.0 / 16)
    U = system.forward_substitution(S, system.rhs_heat(S, u0))
    assert bench._solution_error(u0, U)["rel_max_err"] == 0.0
    got = bench._solution_error(u0, U * (1 + 1e-9))
    assert 0.5e-9 <= got["rel_max_err"] <= 2e-9
    assert "error" in bench._solution_error(u0, U[:3])       # wrong shape: reported
