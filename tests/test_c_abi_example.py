"""The C ABI used from C: tests/c/hobi_c_example.c includes only include/hobi.h and links
libhobi.so. On the CPU it must compile and link; on the GPU its FP64 and FP32 solves of a
refined-octahedron sphere must reproduce the Born energy (Sec. 3.2, Table 2)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build(tmp_path):
    from paper_1301_5914_gb300 import build

    lib = build.build()
    exe = str(tmp_path / "hobi_c_example")
    libdir = os.path.dirname(lib)
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c", "hobi_c_example.c"), "-L", libdir, "-lhobi",
                           "-Wl,-rpath," + libdir, "-lm", "-o", exe])
    return exe


def test_c_example_compiles_and_links(tmp_path):
    exe = _build(tmp_path)
    assert os.path.exists(exe)
    out = subprocess.run(["ldd", exe], capture_output=True, text=True).stdout
    assert "libhobi.so" in out and "not found" not in out


@pytest.mark.gpu
def test_c_example_born_sphere(tmp_path):
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    exe = _build(tmp_path)
    r = subprocess.run([exe, "4", "2.0"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    rows = re.findall(r"(fp64|fp32) vertices (\d+) faces (\d+) iterations (\d+) E_sol (\S+) born (\S+)", r.stdout)
    assert [x[0] for x in rows] == ["fp64", "fp32"]
    e64, e32, born = float(rows[0][4]), float(rows[1][4]), float(rows[0][5])
    assert abs(e64 - born) <= 2e-3 * abs(born)
    assert abs(e32 - e64) <= 1e-5 * abs(e64)
    # the energy is (1/2) 4 pi C q phi_reac at the charge (the centre); inside a sphere with a centred
    # charge the reaction potential is constant, so the field vanishes up to the discretisation error
    pots = re.findall(r"(fp64|fp32) phi_reac (\S+) (\S+) field (.*)", r.stdout)
    assert [x[0] for x in pots] == ["fp64", "fp32"]
    for (prec, p0, p1, fld), e in zip(pots, (e64, e32)):
        p0, p1 = float(p0), float(p1)
        f = [float(v) for v in fld.split()]
        # FP32: the energy's and the potential's far-field plans chunk the sources differently
        assert abs(0.5 * 4 * 3.141592653589793 * 332.0716 * p0 - e) <= (1e-9 if prec == "fp64" else 1e-6) * abs(e)
        assert abs(p1 - p0) <= 5e-3 * abs(p0)
        assert max(abs(v) for v in f) * 2.0 <= 1e-2 * abs(p0), (prec, f, p0)
