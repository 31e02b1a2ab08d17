"""FP32 and FP64 far fields in both of their coordinate modes against the FP64 oracle.

For kappa at or above 1e-6 1/A the far-field tables (FP32 and FP64 alike) hold coordinates
multiplied by kappa (the pair formula then needs no kappa r product); below it, kappa = 0
included, they are unscaled. Both modes must give the same operator (Eqs. (17)-(18)), reaction
potential and energy (Sec. 2.5) as the oracle, on either side of the switch, for single
molecules, LOBI-PB and batches: FP32 within its bulk tolerances, FP64 within 1e-10.
"""
import numpy as np
import pytest

import oracle
from paper_1301_5914_gb300 import hobi, synth

pytestmark = pytest.mark.gpu

# below the switch, just above it, the paper's values, and a strongly screened case
KAPPAS = [0.0, 5e-7, 1e-6, 0.1257, 3.0]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.fixture(scope="module")
def sphere():
    V, F, N = synth.icosphere(3, 4.0)
    return V, F, N, synth.ball_charges(5, 3.0, 11)


@pytest.mark.parametrize("kappa", KAPPAS)
def test_fp32_matvec_and_energy_both_modes(sphere, kappa):
    V, F, N, Q = sphere
    orc = oracle.Problem(V, F, N, Q, 1.0, 80.0, kappa)
    s = hobi.Solver(V, F, N, Q, 1.0, 80.0, kappa, precision="fp32")
    u = np.random.default_rng(21).normal(size=2 * s.nv)
    assert _rel(s.matvec(u), orc.matvec(u)) <= 1e-5
    u_sol, it_ref, _, _ = orc.gmres(1e-8)
    assert _rel(s.matvec(u_sol), orc.matvec(u_sol)) <= 2e-6
    # energy and off-surface potential of the oracle's solution through the FP32 row-1 kernel
    s.set_solution(u_sol)
    e_ref = orc.energy(u_sol)
    assert abs(s.energy() - e_ref) <= 1e-5 * abs(e_ref)
    pts = np.array([[0.3, -0.2, 0.1], [1.0, 1.5, -0.5], [0.0, 0.0, 2.5]])
    got = s.reaction_potential(pts)
    ref = orc.reaction_potential(u_sol, pts)
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))
    phi, dphi, info = s.solve(1e-6)
    assert info["converged"]


@pytest.mark.parametrize("kappa", [0.0, 0.1257])
def test_lobi_fp32_both_modes(sphere, kappa):
    """LOBI-PB skips the zero-distance self pair: the skip must hold in both modes."""
    V, F, N, Q = sphere
    orc = oracle.LobiProblem(V, F, N, Q, 1.0, 80.0, kappa)
    s = hobi.Solver(V, F, N, Q, 1.0, 80.0, kappa, precision="fp32", scheme="lobi")
    u = np.random.default_rng(22).normal(size=2 * s.npts)
    assert _rel(s.matvec(u), orc.matvec(u)) <= 1e-5


@pytest.mark.parametrize("kappa", [0.0, 0.1257])
def test_batch_fp32_both_modes(kappa):
    mols = []
    for k, (lvl, rad) in enumerate([(2, 3.0), (3, 5.0), (1, 2.0)]):
        V, F, N = synth.icosphere(lvl, rad)
        mols.append((V, F, N, synth.ball_charges(3, 0.6 * rad, 30 + k)))
    b = hobi.BatchSolver(mols, 1.0, 80.0, kappa, precision="fp32")
    u = np.random.default_rng(40).normal(size=2 * b.nv_total)
    Au = b.matvec(u)
    off = 0
    for m in mols:
        n = 2 * m[0].shape[0]
        orc = oracle.Problem(*m, 1.0, 80.0, kappa)
        assert _rel(Au[off:off + n], orc.matvec(u[off:off + n])) <= 1e-5
        off += n


@pytest.mark.parametrize("kappa", KAPPAS)
def test_fp64_matvec_energy_and_potential_both_modes(sphere, kappa):
    V, F, N, Q = sphere
    orc = oracle.Problem(V, F, N, Q, 1.0, 80.0, kappa)
    s = hobi.Solver(V, F, N, Q, 1.0, 80.0, kappa, precision="fp64")
    u = np.random.default_rng(23).normal(size=2 * s.nv)
    ref = orc.matvec(u)
    assert np.max(np.abs(s.matvec(u) - ref)) <= 1e-10 * np.max(np.abs(ref))
    u_sol, _, _, _ = orc.gmres(1e-8)
    s.set_solution(u_sol)
    e_ref = orc.energy(u_sol)
    assert abs(s.energy() - e_ref) <= 1e-10 * abs(e_ref)
    pts = np.array([[0.3, -0.2, 0.1], [1.0, 1.5, -0.5], [0.0, 0.0, 2.5]])
    ref_p = orc.reaction_potential(u_sol, pts)
    assert np.max(np.abs(s.reaction_potential(pts) - ref_p)) <= 1e-10 * np.max(np.abs(ref_p))


@pytest.mark.parametrize("kappa", [0.0, 5e-7, 0.1257])
def test_lobi_fp64_both_modes(sphere, kappa):
    V, F, N, Q = sphere
    orc = oracle.LobiProblem(V, F, N, Q, 1.0, 80.0, kappa)
    s = hobi.Solver(V, F, N, Q, 1.0, 80.0, kappa, precision="fp64", scheme="lobi")
    u = np.random.default_rng(24).normal(size=2 * s.npts)
    ref = orc.matvec(u)
    assert np.max(np.abs(s.matvec(u) - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("kappa", [0.0, 5e-7, 0.1257])
def test_batch_fp64_both_modes(kappa):
    mols = []
    for k, (lvl, rad) in enumerate([(2, 3.0), (3, 5.0), (1, 2.0)]):
        V, F, N = synth.icosphere(lvl, rad)
        mols.append((V, F, N, synth.ball_charges(3, 0.6 * rad, 50 + k)))
    b = hobi.BatchSolver(mols, 1.0, 80.0, kappa, precision="fp64")
    u = np.random.default_rng(41).normal(size=2 * b.nv_total)
    Au = b.matvec(u)
    off = 0
    for m in mols:
        n = 2 * m[0].shape[0]
        ref = oracle.Problem(*m, 1.0, 80.0, kappa).matvec(u[off:off + n])
        assert np.max(np.abs(Au[off:off + n] - ref)) <= 1e-10 * np.max(np.abs(ref))
        off += n
