"""Host-side helpers of bench.py on CPU: the CPU model recorded beside the oracle baseline, and
the reference arm's JSON line (the oracle timed on the host cores) at a tiny sample."""
import io
import json
import os
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench

    return bench


def test_cpu_model_x86_and_arm(tmp_path):
    bench = _bench()
    x86 = tmp_path / "x86"
    x86.write_text("processor\t: 0\nvendor_id\t: GenuineIntel\nmodel name\t: Some Xeon @ 2.70GHz\n")
    assert bench._cpu_model(str(x86)) == "Some Xeon @ 2.70GHz"
    arm = tmp_path / "arm"
    arm.write_text("processor\t: 0\nBogoMIPS\t: 2000.00\nCPU implementer\t: 0x41\nCPU part\t: 0xd4f\n")
    m = bench._cpu_model(str(arm))
    assert "CPU implementer 0x41" in m and "part 0xd4f" in m
    assert bench._cpu_model(str(tmp_path / "missing"))  # never empty, never raises


def test_reference_arm_line(monkeypatch):
    bench = _bench()
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        rc = bench.main(["--impl", "reference", "--steps", "1", "--warmup", "0", "--ref-rows", "8"])
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert rc == 0 and line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cpu_model"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["higher_is_better"] is True and line["unit"] == "pair-evals/s"


def test_roofline_arithmetic():
    """The lane-peak fractions the bench line reports: pairs x operations per pair / launch time
    against SMs x lanes x clock, and the profile averages they start from."""
    bench = _bench()
    # 1.113e12 pairs/s at 30 FP32 operations per pair on 152 SMs x 128 lanes x 2070 MHz
    launch_s = 12.06e-3
    pairs = 1.113e12 * launch_s
    achieved, peak, frac = bench.alu_fraction(launch_s, pairs, 30, 128, 152, 2070.0)
    assert abs(peak - 152 * 128 * 2070e6) < 1.0
    assert abs(achieved - 1.113e12 * 30) / achieved < 1e-12
    assert abs(frac - 1.113e12 * 30 / (152 * 128 * 2070e6)) < 1e-12 and 0.82 < frac < 0.84
    # FP64: 44 operations per pair against 2 lanes per SM
    _, peak64, frac64 = bench.alu_fraction(1.0, 1.29e10, bench.FP64_OPS_PER_PAIR, bench.FP64_LANES_PER_SM, 152, 2070.0)
    assert abs(peak64 - 152 * 2 * 2070e6) < 1.0 and 0.89 < frac64 < 0.91
    # profile averages: summed milliseconds and pairs over the launch count; no launches -> no division by zero
    s, p = bench.ff_launch_rate({"farfield_ms": 24.0, "launches": 2, "pairs": 4.0e10})
    assert abs(s - 12e-3) < 1e-15 and p == 2.0e10
    s0, p0 = bench.ff_launch_rate({"farfield_ms": 0.0, "launches": 0, "pairs": 0.0})
    assert s0 == 0.0 and p0 == 0.0
