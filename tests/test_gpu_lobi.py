"""LOBI-PB (Sec. 2.4, Eqs. (21)/(22)) on the GPU against the oracle's LOBI scheme: flat-face
geometry, right-hand side, matvec (self pair skipped), GMRES and energy, both precisions."""
import numpy as np
import pytest

import oracle
from paper_1301_5914_gb300 import hobi, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")


CASES = {
    "sphere_l3": lambda: (*synth.icosphere(3, 2.0), synth.point_charge(0.5, 0, 0, 1.0), 1.0, 80.0, 0.1257),
    "sphere_l4_r10": lambda: (*synth.icosphere(4, 10.0), synth.ball_charges(10, 8.0, 2), 1.0, 80.0, 0.1257),
    "molecule_60": lambda: (*synth.synthetic_molecule(60, 7), 2.0, 80.0, 0.1257),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    V, F, N, Q, e1, e2, ka = CASES[request.param]()
    return V, F, N, Q, e1, e2, ka, oracle.LobiProblem(V, F, N, Q, e1, e2, ka)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def test_lobi_geometry_and_rhs(case):
    V, F, N, Q, e1, e2, ka, orc = case
    s = hobi.Solver(V, F, N, Q, e1, e2, ka, precision="fp64", scheme="lobi")
    assert s.npts == len(F) and s.n_nodes == len(F)
    y, nu, W = s.nodes()
    x, n, A = orc.geometry()
    assert np.max(np.abs(y - x)) <= 1e-13 * np.max(np.abs(x))
    assert np.max(np.abs(nu - n)) <= 1e-12
    assert np.max(np.abs(W[:, 0] - A)) <= 1e-13 * A.max() and not W[:, 1:].any()
    assert _rel(s.rhs(), orc.rhs()) <= 1e-12


def test_lobi_matvec(case):
    V, F, N, Q, e1, e2, ka, orc = case
    s = hobi.Solver(V, F, N, Q, e1, e2, ka, precision="fp64", scheme="lobi")
    u = np.random.default_rng(1).normal(size=2 * s.npts)
    ref = orc.matvec(u)
    assert np.max(np.abs(s.matvec(u) - ref)) <= 1e-10 * np.max(np.abs(ref))
    s.set_precision("fp32")
    assert _rel(s.matvec(u), ref) <= 1e-5


def test_lobi_unscaled_gmres_matches_oracle(case):
    """LOBI-PB with gmres_scaling off: the oracle's iterations and solution on the plain system."""
    V, F, N, Q, e1, e2, ka, orc = case
    u_ref, it_ref, conv, hist_ref = orc.gmres(1e-6, scaled=False)
    s = hobi.Solver(V, F, N, Q, e1, e2, ka, precision="fp64", scheme="lobi", gmres_scaling=False)
    phi, dphi, info = s.solve(1e-6, history=64)
    assert conv and info["iterations"] == it_ref
    assert _rel(np.concatenate([phi, dphi]), u_ref) <= 1e-10
    assert np.allclose(info["history"], hist_ref, rtol=1e-8, atol=0)


def test_lobi_solve_and_energy(case):
    V, F, N, Q, e1, e2, ka, orc = case
    u_ref, it_ref, conv, _ = orc.gmres(1e-6)
    E_ref = orc.energy(u_ref)
    s = hobi.Solver(V, F, N, Q, e1, e2, ka, precision="fp64", scheme="lobi")
    phi, dphi, info = s.solve(1e-6)
    assert info["iterations"] == it_ref
    assert _rel(np.concatenate([phi, dphi]), u_ref) <= 1e-10
    assert abs(s.energy() - E_ref) <= 1e-10 * abs(E_ref)
    s.set_precision("fp32")
    phi, dphi, info = s.solve(1e-6)
    assert abs(info["iterations"] - it_ref) <= 1
    assert _rel(phi, u_ref[: s.npts]) <= 1e-4 and _rel(dphi, u_ref[s.npts:]) <= 1e-4
    assert abs(s.energy() - E_ref) <= 1e-5 * abs(E_ref)
