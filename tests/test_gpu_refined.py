"""Mixed-precision solve (hobi_solve_refined): FP32-bulk GMRES corrections with FP64 residuals
must reach FP64-level tolerances on the FP64 operator, and agree with the oracle's solution."""
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


@pytest.fixture(scope="module")
def sphere():
    V, F, N = synth.icosphere(4, 10.0)
    Q = synth.ball_charges(10, 8.0, 2)
    orc = oracle.Problem(V, F, N, Q, 1.0, 80.0, 0.1257)
    return V, F, N, Q, orc


def _fp64_residual(V, F, N, Q, u):
    s = hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.1257, precision="fp64")
    b = s.rhs()
    return np.linalg.norm(b - s.matvec(u)) / np.linalg.norm(b)


@pytest.mark.parametrize("fast", [0, 5])
def test_refined_reaches_fp64_tolerance(sphere, fast):
    V, F, N, Q, orc = sphere
    s = hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.1257, precision="fp32", fast_degree=fast)
    phi, dphi, info = s.solve_refined(1e-10, history=10)
    assert info["converged"] and info["rel_residual"] <= 1e-10
    hist = info["history"]
    assert hist[0] == 1.0 and np.all(np.diff(hist[hist > 0]) < 0)   # the FP64 residual falls each step
    u = np.concatenate([phi, dphi])
    assert _fp64_residual(V, F, N, Q, u) <= 1.5e-10
    u_ref = orc.gmres(1e-12)[0]
    assert np.linalg.norm(u - u_ref) <= 1e-8 * np.linalg.norm(u_ref)
    # the handle keeps its precision (FP32-bulk: the energy's pair sums carry ~1e-7) and the solution
    assert abs(s.energy() - orc.energy(u_ref)) <= 1e-6 * abs(orc.energy(u_ref))
    Au = s.matvec(u)  # still the FP32-bulk operator
    b = s.rhs()
    assert np.linalg.norm(b - Au) / np.linalg.norm(b) > 1e-9


def test_refined_not_converged_status(sphere):
    V, F, N, Q, orc = sphere
    s = hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.1257, precision="fp32")
    phi, dphi, info = s.solve_refined(1e-14, max_refine=1, raise_on_fail=False)
    assert info["status"] == hobi.HOBI_ERR_NOT_CONVERGED and not info["converged"]
    assert 1e-14 < info["rel_residual"] < 1e-4
