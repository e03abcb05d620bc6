"""Host-side pieces of bench.py, no GPU: the roofline line's inputs exist in
the committed ncu summaries, the nvidia-smi clock samples are parsed into a
median clock and the set of throttle reasons, and the reference arm does no
work on ranks other than 0."""
import argparse
import io
import os
import tempfile
from contextlib import redirect_stdout

import pytest

import bench


def test_roofline_inputs_are_in_the_committed_summaries():
    # ALU-pipe instructions and DRAM bytes per launch of the dominant kernel
    alu = bench._profile_value("alu_inst_per_launch", bench.ROOFLINE_KEY)
    dram = bench._traffic(bench.ROOFLINE_KEY)
    assert alu is not None and alu > 0
    assert dram is not None and dram > 0
    # the fused matvec reads z, v, v0 and writes w (32 B per element of the
    # 4095 x 4096 workload); its DRAM traffic cannot be below that by more
    # than what L2 keeps between launches, nor far above it
    algo = 32 * bench.N_SPACE * bench.ELL
    assert 0.5 * algo <= dram <= 1.5 * algo
    assert bench._profile_value("alu_inst_per_launch", "no_such_kernel") is None


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
