"""GPU parity at full workload sizes: the synthetic 1000-atom molecule (the stand-in for the
paper's protein workload, ~40k curved triangles, eps1 = 2) and the level-6 Kirkwood sphere that
bench.py times, in the same launch configuration. The oracle evaluates sampled matvec rows one
by one; whole-vector properties (solve agreement, residual, energy) are checked at full size.
"""
import numpy as np
import pytest

import oracle
from oracle import kirkwood as kw
from paper_1301_5914_gb300 import hobi, synth
from rowsample import boundary_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.fixture(scope="module")
def molecule():
    V, F, N, Q = synth.synthetic_molecule(1000, 3)
    return V, F, N, Q, 2.0, 80.0, 0.1257


def _rows(nv, k, seed):
    return np.sort(np.random.default_rng(seed).choice(nv, size=k, replace=False))


def _check_rows(Au, orc, u, rows, tol):
    r1, r2 = orc.matvec_rows(u, rows)
    nv = orc.nv
    got1, got2 = Au[rows], Au[nv + rows]
    s1 = np.max(np.abs(r1)) + 1e-300
    s2 = np.max(np.abs(r2)) + 1e-300
    assert np.max(np.abs(got1 - r1)) <= tol * s1, np.max(np.abs(got1 - r1)) / s1
    assert np.max(np.abs(got2 - r2)) <= tol * s2, np.max(np.abs(got2 - r2)) / s2


def test_molecule_tables_match_oracle(molecule):
    V, F, N, Q, e1, e2, ka = molecule
    assert 36000 < F.shape[0] < 44000
    orc = oracle.Problem(V, F, N, Q, e1, e2, ka)
    s = hobi.Solver(V, F, N, Q, e1, e2, ka, precision="fp64")
    y, nu, W = s.nodes()
    oy, onu, oW = orc.nodes()
    assert np.max(np.abs(y - oy)) <= 1e-12 * np.max(np.abs(oy))
    assert np.max(np.abs(nu - onu)) <= 1e-10
    assert np.max(np.abs(W - oW)) <= 1e-11 * np.max(np.abs(oW))
    b = s.rhs()
    assert np.linalg.norm(b - orc.rhs()) <= 1e-12 * np.linalg.norm(b)


def test_molecule_matvec_sampled_rows(molecule):
    V, F, N, Q, e1, e2, ka = molecule
    orc = oracle.Problem(V, F, N, Q, e1, e2, ka)
    s = hobi.Solver(V, F, N, Q, e1, e2, ka, precision="fp64")
    rng = np.random.default_rng(4)
    u = rng.normal(size=2 * s.nv)
    rows = boundary_rows(s.nv, 64, 1)
    assert rows.size >= 300
    _check_rows(s.matvec(u), orc, u, rows, 1e-10)
    # FP32 bulk on a smooth density (the FP64 solution) and on the random vector
    phi, dphi, info = s.solve(1e-6, 200)
    usol = np.concatenate([phi, dphi])
    s.set_precision("fp32")
    _check_rows(s.matvec(usol), orc, usol, rows, 2e-5)
    _check_rows(s.matvec(u), orc, u, rows, 1e-4)


def test_molecule_rhs_matches_oracle(molecule):
    """Eq. (11) at 19,944 vertices with 1,000 charges (two-float Coulomb sums) against the oracle."""
    V, F, N, Q, e1, e2, ka = molecule
    ref = oracle.Problem(V, F, N, Q, e1, e2, ka).rhs()
    b = hobi.Solver(V, F, N, Q, e1, e2, ka, precision="fp64").rhs()
    assert np.linalg.norm(b - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.max(np.abs(b - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_molecule_solve_fp32_vs_fp64_and_energy(molecule):
    V, F, N, Q, e1, e2, ka = molecule
    s = hobi.Solver(V, F, N, Q, e1, e2, ka, precision="fp64")
    p64, d64, i64 = s.solve(1e-6, 200)
    E64 = s.energy()
    assert i64["converged"] and i64["iterations"] <= 20
    # GMRES on the plain system (no diagonal scaling) needs at least twice the iterations
    su = hobi.Solver(V, F, N, Q, e1, e2, ka, precision="fp64", gmres_scaling=False)
    pu, du, iu = su.solve(1e-6, 200)
    assert iu["converged"] and iu["iterations"] >= 2 * i64["iterations"]
    assert np.linalg.norm(np.concatenate([pu, du]) - np.concatenate([p64, d64])) <= 1e-4 * np.linalg.norm(
        np.concatenate([p64, d64]))
    u64 = np.concatenate([p64, d64])
    # the oracle's energy of the same surface potential (all N_c x N_n pairs)
    orc = oracle.Problem(V, F, N, Q, e1, e2, ka)
    assert abs(E64 - orc.energy(u64)) <= 1e-10 * abs(E64)
    # residual of the GPU solution on oracle rows is at the GMRES tolerance level
    b = orc.rhs()
    rows = _rows(s.nv, 32, 7)
    r1, r2 = orc.matvec_rows(u64, rows)
    res = np.concatenate([r1 - b[rows], r2 - b[s.nv + rows]])
    assert np.max(np.abs(res)) <= 1e-5 * np.max(np.abs(b))
    s.set_precision("fp32")
    p32, d32, i32 = s.solve(1e-6, 200)
    E32 = s.energy()
    assert abs(i32["iterations"] - i64["iterations"]) <= 1
    assert np.linalg.norm(p32 - p64) <= 1e-4 * np.linalg.norm(p64)
    assert np.linalg.norm(d32 - d64) <= 1e-4 * np.linalg.norm(d64)
    assert abs(E32 - E64) <= 1e-5 * abs(E64)


def test_bench_workload_full_size_fp32():
    """The bench workload (icosphere level 6, radius 10, 40,962 x 327,680 pairs) through the same
    library calls bench.py makes: sampled FP32 matvec rows vs the oracle, and the solved energy
    and surface potential vs the Kirkwood series."""
    V, F, N = synth.icosphere(6, 10.0)
    Q = synth.ball_charges(10, 8.0, 2)
    s = hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.1257, precision="fp32")
    orc = oracle.Problem(V, F, N, Q, 1.0, 80.0, 0.1257)
    phi, dphi, info = s.solve(1e-6, 200)
    assert info["converged"]
    u = np.concatenate([phi, dphi])
    rows = boundary_rows(s.nv, 128, 2)
    assert rows.size >= 512
    _check_rows(s.matvec(u), orc, u, rows, 2e-5)
    E = s.energy()
    e_ex = kw.solvation_energy(Q, 10.0, 1.0, 80.0, 0.1257)
    assert abs(E - e_ex) <= 1e-3 * abs(e_ex)
    phi_ex, _ = kw.surface_potential(V, Q, 10.0, 1.0, 80.0, 0.1257)
    assert np.max(np.abs(phi - phi_ex)) <= 2e-3 * np.max(np.abs(phi_ex))
