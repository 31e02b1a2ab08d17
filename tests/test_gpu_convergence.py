"""Convergence of the surface potential under icosphere refinement, on the GPU in both
precisions, against the Kirkwood series (paper Sec. 3.1-3.2: the error e_phi of Eq. (24), the
order of Eq. (25) measured in the vertex density d, vertices per A^2).

C2 workload: sphere of radius 10 A, 10 seeded charges in the r <= 8 A ball, eps1 = 1, eps2 = 80,
kappa = 0.1257, icosphere levels 4, 5, 6 (d = 2.0, 8.2, 32.6; each level 4x the density). Plain
FP64 and FP32-bulk solves of each level are compared with the series; the FP32-bulk solution with
the FP64 one (1e-4 relative L2 in phi, 1e-5 in E); and the GPU FP64 solve of level 5 with the
oracle's full solve (1e-10, same Krylov iterations).

Measured on GB300 (FP64, GMRES to 1e-8): e_phi 9.4e-4, 2.5e-4, 6.5e-5 and E_sol errors 3.3e-3,
8.3e-4, 2.1e-4: order 0.96 (phi) and 1.0 (E) in d, i.e. second order in the mesh size h. The
paper's Table 2 reports orders 1.3-1.8 for a centred charge on MSMS spheres; the centred-charge
ladder below converges at order 0.5 in d on icospheres (see tests/test_oracle_convergence.py for
the cause: the fixed 4-point rule on faces next to the incident ones).
"""
import numpy as np
import pytest

import oracle
from oracle import kirkwood as kw
from paper_1301_5914_gb300 import hobi, synth

pytestmark = pytest.mark.gpu

A, EPS1, EPS2, KAPPA = 10.0, 1.0, 80.0, 0.1257
LEVELS = (4, 5, 6)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)


def _errors(phi, dphi, E, phi_k, dphi_k, E_k):
    return {"e_phi": np.max(np.abs(phi - phi_k)) / np.max(np.abs(phi_k)),
            "l2_phi": np.linalg.norm(phi - phi_k) / np.linalg.norm(phi_k),
            "e_dphi": np.max(np.abs(dphi - dphi_k)) / np.max(np.abs(dphi_k)),
            "e_E": abs(E - E_k) / abs(E_k)}


def _order(d, e):
    """Least-squares slope of -log e against log d (Eq. (25) over more than two levels)."""
    return -np.polyfit(np.log(d), np.log(e), 1)[0]


@pytest.fixture(scope="module")
def c2_ladder():
    Q = synth.ball_charges(10, 8.0, 2)
    E_k = kw.solvation_energy(Q, A, EPS1, EPS2, KAPPA)
    out = {}
    for L in LEVELS:
        V, F, N = synth.icosphere(L, A)
        phi_k, dphi_k = kw.surface_potential(V, Q, A, EPS1, EPS2, KAPPA)
        rec = {"d": V.shape[0] / (4 * np.pi * A * A)}
        s = hobi.Solver(V, F, N, Q, EPS1, EPS2, KAPPA, precision="fp64")
        p64, d64, i64 = s.solve(1e-8, 400)
        E64 = s.energy()
        s.set_precision("fp32")
        p32, d32, i32 = s.solve(1e-6, 400)
        E32 = s.energy()
        s.close()
        assert i64["converged"] and i32["converged"]
        rec["fp64"] = _errors(p64, d64, E64, phi_k, dphi_k, E_k)
        rec["fp32"] = _errors(p32, d32, E32, phi_k, dphi_k, E_k)
        rec["fp32_vs_fp64"] = {"phi": np.linalg.norm(p32 - p64) / np.linalg.norm(p64),
                               "dphi": np.linalg.norm(d32 - d64) / np.linalg.norm(d64),
                               "E": abs(E32 - E64) / abs(E64)}
        out[L] = rec
    for L in LEVELS:
        r = out[L]
        print(f"C2 L{L} d={r['d']:.2f}: FP64 e_phi {r['fp64']['e_phi']:.3e} l2 {r['fp64']['l2_phi']:.3e} "
              f"e_dphi {r['fp64']['e_dphi']:.3e} E {r['fp64']['e_E']:.2e} | FP32 e_phi {r['fp32']['e_phi']:.3e} "
              f"E {r['fp32']['e_E']:.2e} | FP32 vs FP64 phi {r['fp32_vs_fp64']['phi']:.2e} E {r['fp32_vs_fp64']['E']:.2e}")
    return out


def test_c2_errors_fall_at_first_order_in_density(c2_ladder):
    d = np.array([c2_ladder[L]["d"] for L in LEVELS])
    for prec in ("fp64", "fp32"):
        e_phi = np.array([c2_ladder[L][prec]["e_phi"] for L in LEVELS])
        e_E = np.array([c2_ladder[L][prec]["e_E"] for L in LEVELS])
        assert np.all(np.diff(e_phi) < 0) and np.all(np.diff(e_E) < 0), (prec, e_phi, e_E)
        # measured 0.96 (phi) and 1.0 (E) in FP64; the FP32-bulk max-norm error carries its own
        # ~1e-5 floor at level 6 (0.88 measured)
        lo = 0.9 if prec == "fp64" else 0.8
        assert _order(d, e_phi) >= lo, (prec, _order(d, e_phi))
        assert _order(d, e_E) >= 0.9, (prec, _order(d, e_E))
        assert e_phi[-1] <= 1e-4 and e_E[-1] <= 3e-4
    e_dphi = np.array([c2_ladder[L]["fp64"]["e_dphi"] for L in LEVELS])
    assert _order(d, e_dphi) >= 0.85


def test_c2_fp32_bulk_within_its_tolerances_of_fp64(c2_ladder):
    for L in LEVELS:
        r = c2_ladder[L]["fp32_vs_fp64"]
        assert r["phi"] <= 1e-4 and r["dphi"] <= 1e-4 and r["E"] <= 1e-5, (L, r)


def test_c2_level5_gpu_fp64_solve_equals_oracle_solve():
    """The GPU FP64 solve of level 5 (10,242 vertices) against the oracle's full GMRES solve: the
    same number of Krylov iterations and solutions within 1e-10."""
    V, F, N = synth.icosphere(5, A)
    Q = synth.ball_charges(10, 8.0, 2)
    orc = oracle.Problem(V, F, N, Q, EPS1, EPS2, KAPPA)
    u_ref, it_ref, conv, _ = orc.gmres(1e-6)
    assert conv
    s = hobi.Solver(V, F, N, Q, EPS1, EPS2, KAPPA, precision="fp64")
    phi, dphi, info = s.solve(1e-6, 400)
    assert info["converged"] and info["iterations"] == it_ref
    u = np.concatenate([phi, dphi])
    assert np.linalg.norm(u - u_ref) <= 1e-10 * np.linalg.norm(u_ref)
    e_ref = orc.energy(u_ref)
    assert abs(s.energy() - e_ref) <= 1e-10 * abs(e_ref)


def test_centred_charge_ladder_converges_at_half_order_in_density():
    """Table 2's case (radius 2 A, +1 e at the centre, eps = 80, kappa = 0) on icospheres: the
    exact surface values are constant, phi = 1/(4 pi eps2 a) and dphi/dnu = -1/(4 pi eps1 a^2).
    Measured e_phi 2.0e-5, 1.15e-5, 6.0e-6, 3.0e-6 at levels 3-6 (d = 12.8, 51, 204, 815): order
    0.48 in d, first order in h; E_sol within 1.1e-6 of the Born energy at level 6."""
    a, q = 2.0, 1.0
    phi_ex = q / (4 * np.pi * 80.0 * a)
    dphi_ex = -q / (4 * np.pi * 1.0 * a * a)
    E_born = kw.born_energy(q, a, 1.0, 80.0, 0.0)
    d, e_phi, e_dphi, e_E = [], [], [], []
    for L in (3, 4, 5, 6):
        V, F, N = synth.icosphere(L, a)
        s = hobi.Solver(V, F, N, synth.point_charge(0.0, 0.0, 0.0, q), 1.0, 80.0, 0.0, precision="fp64")
        phi, dphi, info = s.solve(1e-12, 400)
        assert info["converged"]
        d.append(V.shape[0] / (4 * np.pi * a * a))
        e_phi.append(np.max(np.abs(phi - phi_ex)) / abs(phi_ex))
        e_dphi.append(np.max(np.abs(dphi - dphi_ex)) / abs(dphi_ex))
        e_E.append(abs(s.energy() - E_born) / abs(E_born))
        s.close()
    print("centred charge: d", np.round(d, 1), "e_phi", e_phi, "e_dphi", e_dphi, "e_E", e_E)
    assert np.all(np.diff(e_phi) < 0) and np.all(np.diff(e_E) < 0)
    order = _order(np.array(d[1:]), np.array(e_phi[1:]))
    assert 0.35 <= order <= 0.7, order
    assert e_phi[-1] <= 4e-6 and e_E[-1] <= 2e-6
