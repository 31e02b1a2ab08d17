"""Reaction field -grad phi_reac at off-surface points (hobi_reaction_field) against the oracle,
through the C ABI: FP64 to 1e-10 and FP32 bulk to 5e-5 of the largest component, on a point set
that spans several 256-target blocks with a ragged tail, kappa-scaled and unscaled, host and
device pointers; plus the argument and state checks."""
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
    # radius-2 icosphere (642 vertices), one off-centre charge
    "sphere_l3": lambda: (*synth.icosphere(3, 2.0), synth.point_charge(0.5, 0.2, -0.1, 1.0), 1.0, 80.0, 0.1257),
    "sphere_l3_k0": lambda: (*synth.icosphere(3, 2.0), synth.point_charge(0.5, 0.2, -0.1, 1.0), 1.0, 80.0, 0.0),
    # a 60-atom synthetic molecule, eps1 = 2
    "molecule_60": lambda: (*synth.synthetic_molecule(60, 7), 2.0, 80.0, 0.1257),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    V, F, N, Q, e1, e2, ka = CASES[request.param]()
    orc = oracle.Problem(V, F, N, Q, e1, e2, ka)
    u = orc.gmres(1e-8)[0]
    # 785 points (3 blocks of 256 and a ragged tail): inside the charges' ball and outside the surface
    rng = np.random.default_rng(31)
    c = V.mean(axis=0)
    R = np.linalg.norm(V - c, axis=1)
    inner = c + synth.ball_charges(600, 0.5 * R.min(), 32)[:, :3]
    d = rng.normal(size=(185, 3))
    outer = c + d / np.linalg.norm(d, axis=1)[:, None] * (R.max() + 1.0 + rng.random((185, 1)))
    pts = np.ascontiguousarray(np.concatenate([inner, outer]))
    return V, F, N, Q, e1, e2, ka, orc, u, pts


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 5e-5)])
def test_field_matches_oracle(case, prec, tol):
    V, F, N, Q, e1, e2, ka, orc, u, pts = case
    ref = orc.reaction_field(u, pts)
    s = hobi.Solver(V, F, N, Q, e1, e2, ka, precision=prec)
    s.set_solution(u)
    f = s.reaction_field(pts)
    assert f.shape == (pts.shape[0], 3)
    assert np.max(np.abs(f - ref)) <= tol * np.max(np.abs(ref)), np.max(np.abs(f - ref)) / np.max(np.abs(ref))
    s.close()


def test_field_is_minus_the_gradient_of_the_gpu_reaction_potential(case):
    V, F, N, Q, e1, e2, ka, orc, u, pts = case
    s = hobi.Solver(V, F, N, Q, e1, e2, ka, precision="fp64")
    s.set_solution(u)
    x = pts[:64]
    f = s.reaction_field(x)
    h = 1e-4
    fd = np.zeros_like(f)
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        fd[:, c] = -(s.reaction_potential(x + e) - s.reaction_potential(x - e)) / (2 * h)
    assert np.max(np.abs(f - fd)) <= 1e-6 * np.max(np.abs(f))


def test_field_device_pointers_equal_host(case):
    import torch

    V, F, N, Q, e1, e2, ka, orc, u, pts = case
    dev = torch.device("cuda:0")
    t = lambda a, dt=torch.float64: torch.as_tensor(a, dtype=dt, device=dev)
    for prec in ("fp64", "fp32"):
        sh = hobi.Solver(V, F, N, Q, e1, e2, ka, precision=prec)
        sd = hobi.Solver(t(V), t(F, torch.int32), t(N), t(Q), e1, e2, ka, precision=prec)
        sh.set_solution(u)
        sd.set_solution(t(u))
        a = sh.reaction_field(pts)
        b = sd.reaction_field(t(pts))
        assert isinstance(b, torch.Tensor) and b.shape == (pts.shape[0], 3)
        assert np.array_equal(a, b.cpu().numpy())
        fd = sd.reaction_forces()
        assert isinstance(fd, torch.Tensor) and np.array_equal(sh.reaction_forces(), fd.cpu().numpy())


def test_field_arguments_and_state():
    import ctypes as C

    V, F, N = synth.icosphere(2, 2.0)
    Q = synth.point_charge(0, 0, 0, 1.0)
    s = hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.0, precision="fp64")
    with pytest.raises(hobi.HobiError) as ei:
        s.reaction_field(np.zeros((4, 3)))
    assert ei.value.code == hobi.HOBI_ERR_STATE
    s.solve(1e-8)
    assert s.reaction_field(np.zeros((0, 3))).shape == (0, 3)
    lib = hobi.load_library()
    assert lib.hobi_reaction_field(s._h, None, 4, None) == hobi.HOBI_ERR_ARG
    assert lib.hobi_reaction_field(s._h, None, -1, None) == hobi.HOBI_ERR_ARG
    lo = hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.0, precision="fp64", scheme="lobi")
    lo.solve(1e-8)
    with pytest.raises(hobi.HobiError) as ei:
        lo.reaction_field(np.zeros((4, 3)))
    assert ei.value.code == hobi.HOBI_ERR_ARG


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 5e-5)])
def test_reaction_forces_match_oracle(case, prec, tol):
    """4 pi C q_k times the reaction field at each charge (kcal/(mol A)) against the oracle's."""
    V, F, N, Q, e1, e2, ka, orc, u, pts = case
    ref = orc.reaction_forces(u)
    s = hobi.Solver(V, F, N, Q, e1, e2, ka, precision=prec)
    s.set_solution(u)
    f = s.reaction_forces()
    assert f.shape == (Q.shape[0], 3)
    assert np.max(np.abs(f - ref)) <= tol * np.max(np.abs(ref)), np.max(np.abs(f - ref)) / np.max(np.abs(ref))
    s.close()


def test_reaction_forces_without_charges_or_solution():
    V, F, N = synth.icosphere(2, 2.0)
    s = hobi.Solver(V, F, N, np.zeros((0, 4)), 1.0, 80.0, 0.1, precision="fp64")
    with pytest.raises(hobi.HobiError) as ei:
        s.reaction_forces()
    assert ei.value.code == hobi.HOBI_ERR_STATE
    s.solve(1e-8, 50, raise_on_fail=False)
    assert s.reaction_forces().shape == (0, 3)


def test_field_of_a_fast_summation_handle_is_the_direct_sum():
    """The reaction field always sums every node directly: a handle whose matvec uses the treecode
    gives the same field as a direct handle from the same solution."""
    V, F, N = synth.icosphere(5, 10.0)
    Q = synth.ball_charges(10, 8.0, 2)
    u = np.random.default_rng(4).normal(size=2 * V.shape[0])
    pts = synth.ball_charges(300, 7.0, 5)[:, :3]
    d = hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.1257, precision="fp32")
    f = hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.1257, precision="fp32", fast_degree=5, fast_theta=0.7)
    d.set_solution(u)
    f.set_solution(u)
    assert np.array_equal(d.reaction_field(pts), f.reaction_field(pts))
    assert np.array_equal(d.reaction_forces(), f.reaction_forces())
