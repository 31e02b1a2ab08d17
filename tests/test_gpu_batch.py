"""Batched solve (one far-field launch per GMRES step for all molecules) against the
single-molecule path and the oracle: every molecule's result must equal its own solve."""
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


EPS1, EPS2, KAPPA = 2.0, 80.0, 0.1257


@pytest.fixture(scope="module")
def molecules():
    """Uneven sizes: three icospheres (42, 642, 2562 vertices) and two small synthetic molecules."""
    mols = []
    for lvl, R, seed in ((1, 1.5, 11), (3, 4.0, 12), (4, 8.0, 13)):
        V, F, N = synth.icosphere(lvl, R)
        mols.append((V, F, N, synth.ball_charges(5, 0.6 * R, seed)))
    for n_atoms, seed in ((40, 1001), (90, 1002)):
        mols.append(synth.synthetic_molecule(n_atoms, seed))
    return mols


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_batch_matches_single_solves(molecules, prec, tol):
    """FP64: same arithmetic up to the order of FP64 chunk sums. FP32: the batch uses the
    128-node tile shape in 32-tile tasks while a single solve may use another autotuned shape
    (other FP32 tile sums) -- differences far below the FP32-bulk tolerance (1e-4)."""
    bs = hobi.BatchSolver(molecules, EPS1, EPS2, KAPPA, precision=prec)
    phis, dphis, info = bs.solve(1e-6, 200)
    assert info["converged"] and np.all(info["mol_status"] == 0)
    E = bs.energy()
    for i, (V, F, N, Q) in enumerate(molecules):
        s = hobi.Solver(V, F, N, Q, EPS1, EPS2, KAPPA, precision=prec)
        p, d, inf = s.solve(1e-6, 200)
        assert info["iterations"][i] == inf["iterations"]
        assert _rel(phis[i], p) <= tol and _rel(dphis[i], d) <= tol
        assert abs(E[i] - s.energy()) <= tol * abs(E[i])
        s.close()
    assert info["steps"] == max(info["iterations"])
    bs.close()


def test_batch_fp64_against_oracle(molecules):
    bs = hobi.BatchSolver(molecules[:4], EPS1, EPS2, KAPPA, precision="fp64")
    phis, dphis, info = bs.solve(1e-6, 200)
    E = bs.energy()
    for i, (V, F, N, Q) in enumerate(molecules[:4]):
        orc = oracle.Problem(V, F, N, Q, EPS1, EPS2, KAPPA)
        u_ref, it_ref, conv, _ = orc.gmres(1e-6)
        assert info["iterations"][i] == it_ref
        assert _rel(np.concatenate([phis[i], dphis[i]]), u_ref) <= 1e-10
        assert abs(E[i] - orc.energy(u_ref)) <= 1e-10 * abs(E[i])


def test_batch_unscaled_gmres_against_oracle(molecules):
    """gmres_scaling off: each molecule takes the oracle's iterations on the plain system."""
    bs = hobi.BatchSolver(molecules[:3], EPS1, EPS2, KAPPA, precision="fp64", gmres_scaling=False)
    phis, dphis, info = bs.solve(1e-6, 200)
    for i, (V, F, N, Q) in enumerate(molecules[:3]):
        orc = oracle.Problem(V, F, N, Q, EPS1, EPS2, KAPPA)
        u_ref, it_ref, conv, _ = orc.gmres(1e-6, scaled=False)
        assert info["iterations"][i] == it_ref
        assert _rel(np.concatenate([phis[i], dphis[i]]), u_ref) <= 1e-10


def test_batch_matvec_and_device_mode(molecules):
    import torch

    bh = hobi.BatchSolver(molecules, EPS1, EPS2, KAPPA, precision="fp64")
    bd = hobi.BatchSolver(molecules, EPS1, EPS2, KAPPA, precision="fp64", device_mode=True)
    u = np.random.default_rng(0).normal(size=2 * bh.nv_total)
    Au = bh.matvec(u)
    assert np.array_equal(Au, bd.matvec(torch.as_tensor(u, device="cuda")).cpu().numpy())
    # block m of A u is molecule m's own operator on its block
    off = 0
    for (V, F, N, Q) in molecules:
        n = 2 * V.shape[0]
        s = hobi.Solver(V, F, N, Q, EPS1, EPS2, KAPPA, precision="fp64")
        assert np.max(np.abs(Au[off:off + n] - s.matvec(u[off:off + n]))) <= 1e-12 * np.max(np.abs(Au[off:off + n]))
        off += n


def test_batch_restart_and_not_converged(molecules):
    bs = hobi.BatchSolver(molecules[:3], EPS1, EPS2, KAPPA, precision="fp64", restart=3)
    phis, dphis, info = bs.solve(1e-8, 300)
    assert info["converged"]
    for i, (V, F, N, Q) in enumerate(molecules[:3]):
        s = hobi.Solver(V, F, N, Q, EPS1, EPS2, KAPPA, precision="fp64", restart=3)
        p, d, inf = s.solve(1e-8, 300)
        assert info["iterations"][i] == inf["iterations"]
        assert _rel(phis[i], p) <= 1e-10
    phis, dphis, info = bs.solve(1e-14, 4, raise_on_fail=False)
    assert info["status"] == hobi.HOBI_ERR_NOT_CONVERGED
    assert np.all(info["mol_status"] == hobi.HOBI_ERR_NOT_CONVERGED)


def test_batch_reports_bad_member():
    V, F, N = synth.icosphere(2, 2.0)
    Q = synth.point_charge(0, 0, 0, 1.0)
    with pytest.raises(hobi.HobiError) as ei:
        hobi.BatchSolver([(V, F, N, Q), (V, F[:-1], N, Q)], 1.0, 80.0, 0.0)
    assert ei.value.code == hobi.HOBI_ERR_MESH and "molecule 1" in str(ei.value)


def test_concurrent_member_setup_is_deterministic(molecules):
    """Members are built by several host threads on their own streams and carve their tables from
    one shared arena (in whatever order the threads reach it): two set-ups of the same batch give
    bit-identical solutions and energies."""
    mols = molecules * 3  # 15 members: more than the set-up threads
    out = []
    for _ in range(2):
        bs = hobi.BatchSolver(mols, EPS1, EPS2, KAPPA, precision="fp32")
        phis, dphis, info = bs.solve(1e-6, 200)
        out.append((np.concatenate(phis + dphis), bs.energy(), info["iterations"].copy()))
        bs.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
    # the copies of one molecule in the batch give the same result as each other
    n = len(molecules)
    assert np.array_equal(out[0][1][:n], out[0][1][n:2 * n])


def test_batch_reports_first_bad_member_in_index_order():
    """With several invalid members built concurrently, the error names the first one."""
    V, F, N = synth.icosphere(2, 2.0)
    Q = synth.point_charge(0, 0, 0, 1.0)
    good, bad = (V, F, N, Q), (V, F[:-1], N, Q)
    mols = [good] * 12
    mols[3] = bad
    mols[9] = bad
    for _ in range(3):
        with pytest.raises(hobi.HobiError) as ei:
            hobi.BatchSolver(mols, 1.0, 80.0, 0.0)
        assert ei.value.code == hobi.HOBI_ERR_MESH and "molecule 3:" in str(ei.value)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_batch_reaction_forces_equal_single_handles(molecules, prec, tol):
    """hobi_reaction_forces_batch: per molecule the forces a single handle computes from the same
    solution (the members queue their field kernels on their own streams)."""
    bs = hobi.BatchSolver(molecules, EPS1, EPS2, KAPPA, precision=prec)
    phis, dphis, info = bs.solve(1e-8, 200)
    forces = bs.reaction_forces()
    assert len(forces) == len(molecules)
    for i, (V, F, N, Q) in enumerate(molecules):
        s = hobi.Solver(V, F, N, Q, EPS1, EPS2, KAPPA, precision=prec)
        s.set_solution(np.concatenate([phis[i], dphis[i]]))
        ref = s.reaction_forces()
        assert forces[i].shape == ref.shape == (Q.shape[0], 3)
        assert np.max(np.abs(forces[i] - ref)) <= tol * np.max(np.abs(ref))
        s.close()
    bs.close()
