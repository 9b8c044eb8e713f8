"""Host-side arithmetic of bench.py: the flop counts behind the roofline figures, the FP32 peak
from unit counts, the parsing of the clock samples taken during the timed region, and the
reference arm's JSON line (with the oracle sample replaced by a stand-in, so that no oracle work
runs here); the precision study's medium step count against the oracle's, and the DFT16 study's
column count."""
import importlib.util
import json
import os
from types import SimpleNamespace

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_flop_counts_and_peak():
    b = _bench()
    # two DSTs of 5 N log2 N + 12 N, kinetic 6 N, two half-steps 12 N each, norm 4 N
    assert b.algorithmic_flops_per_step(4096) == 729_088
    for N in (16, 1024, 4096, 16384):
        lg = N.bit_length() - 1
        assert b.algorithmic_flops_per_step(N) == 10 * N * lg + 58 * N
        # the odd-extended length-2N pair: 10 (2N) log2(2N) plus 30 N pointwise
        assert b.nominal_flops_per_step(N) == 20 * N * (lg + 1) + 30 * N
    assert b.nominal_flops_per_step(4096) == 1_187_840
    # 152 SMs x 128 lanes x 2 flops x 2070 MHz
    assert abs(b.fp32_peak_tflops(152) - 80.548) < 1e-3


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_parsed():
    b = _bench()
    cs = b.ClockSampler()
    cs.proc = _FakeProc()
    cs.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
                "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
                "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                "garbage line",
                "0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    clk = cs.stop()
    assert clk["samples"] == 3 and clk["sm_mhz"] == 2070.0 and clk["sm_max_mhz"] == 2070.0
    assert clk["reasons"] == ["sw_power_cap"]
    cs = b.ClockSampler()
    cs.proc = _FakeProc()
    cs.lines = ["0, 1500, 2070, 1200, 0x40, Not Active, Active, Not Active, Not Active"]
    assert cs.stop()["reasons"] == ["hw_thermal_slowdown"]
    cs = b.ClockSampler()
    assert cs.stop()["reasons"] == ["nvidia-smi unavailable"]    # never started


def test_reference_arm_line(monkeypatch, capsys):
    b = _bench()
    import oracle
    monkeypatch.setattr(oracle, "build", lambda: None)
    calls = []

    def sample(n_traj, prefix_steps=2500, seed_offset=0):
        calls.append((n_traj, prefix_steps, seed_offset))
        return n_traj * prefix_steps, 0.5, n_traj

    monkeypatch.setattr(b, "oracle_sample", sample)
    monkeypatch.delenv("RANK", raising=False)
    b.run_reference(SimpleNamespace(steps=2, warmup=1, gpus=1))
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["metric"] == b.METRIC and line["unit"] == b.UNIT
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    cores = calls[-1][0]
    assert line["value"] == round(cores * 2500 / 0.5, 1) == line["e2e"]["value"] == line["cpu_baseline"]["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == cores
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    # one warm-up sample, then one timed sample per step with fresh seeds
    assert [c[1] for c in calls] == [300, 2500, 2500] and calls[1][2] != calls[2][2]
    # other ranks of a torchrun launch print nothing
    monkeypatch.setenv("RANK", "1")
    b.run_reference(SimpleNamespace(steps=1, warmup=0, gpus=2))
    assert capsys.readouterr().out == ""


def test_precision_study_step_count_matches_oracle():
    """precision.medium_step_count (the error model's step count for rMin-shortcut records) agrees
    with the oracle's own step count for Bjorken media, including the two workloads' 11,899 and 23,797."""
    import oracle as o
    from paper_2107_06147_gb300 import precision
    assert precision.medium_step_count(0.425, 0.6, 0.25, 0.001) == 11899
    assert precision.medium_step_count(0.425, 0.6, 0.25, 0.0005) == 23797
    rng = np.random.default_rng(3)
    for _ in range(20):
        T0 = float(rng.uniform(0.3, 0.6)); Tf = T0 * float(rng.uniform(0.4, 0.95)); dt = float(rng.choice([0.001, 0.0005]))
        g = o.Grid(N=64, L=5.0, dt=dt)
        assert precision.medium_step_count(T0, 0.6, Tf, dt) == o.n_steps(g, o.medium(T0, 0.6, Tf, 5.0, 0.0))


def test_dft16_study_column_count():
    """A trajectory-step runs 2 transforms x log16(N) radix-16 passes x N/16 columns."""
    from paper_2107_06147_gb300 import tcstudy
    assert tcstudy.columns_per_traj_step(4096) == 2 * 3 * 256
    assert tcstudy.columns_per_traj_step(65536) == 2 * 4 * 4096
