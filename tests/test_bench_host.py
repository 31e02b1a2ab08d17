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
