"""Parity at the full sizes of the two largest workloads, in the launch configurations bench.py
times: the C5 two-globule complex (59,888 vertices x 479,088 nodes; 1,061 sampled rows, plus the
reaction field at 96 points and the forces on 64 of its charges) and the
C4 batch of 64 molecules (at least 32 rows of every molecule), on rows the oracle evaluates one
by one: the edges of every 256-target block (first and last row, both sides of the first thread
stride) plus seeded random rows; and the empty-charge edge case.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
from paper_1301_5914_gb300 import hobi, synth
from rowsample import boundary_rows

pytestmark = pytest.mark.gpu

KAPPA = 0.1257


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _rows(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))


def _check_rows(Au, ref, rows, nv, tol):
    r1, r2 = ref
    e1 = np.max(np.abs(Au[rows] - r1)) / np.max(np.abs(r1))
    e2 = np.max(np.abs(Au[nv + rows] - r2)) / np.max(np.abs(r2))
    assert e1 <= tol and e2 <= tol, (e1, e2, tol)


def test_c5_complex_sampled_rows():
    V, F, N, Q = synth.two_globule_complex(3000, 51, 52, n_faces=120000)
    s = hobi.Solver(V, F, N, Q, 2.0, 80.0, KAPPA, precision="fp32")
    assert s.nv > 55000 and s.n_nodes > 450000
    phi, dphi, info = s.solve(1e-6, 400)
    assert info["converged"]
    u = np.concatenate([phi, dphi])
    orc = oracle.Problem(V, F, N, Q, 2.0, 80.0, KAPPA)
    rows = boundary_rows(s.nv, 128, 1)
    assert rows.size >= 1000
    ref = orc.matvec_rows(u, rows)
    # FP32 pair terms carry ~1e-7 relative error each; over 479,088 nodes the K3/K4 row cancels
    # more than at smaller sizes (sum of |terms| / |sum| grows), so the bound is 5e-5 of max |row|
    _check_rows(s.matvec(u), ref, rows, s.nv, 5e-5)
    s.set_precision("fp64")
    _check_rows(s.matvec(u), ref, rows, s.nv, 1e-10)
    # the solved energy against the oracle's energy of the same surface potential
    s.set_precision("fp32")
    s.set_solution(u)
    e_ref = orc.energy(u)
    assert abs(s.energy() - e_ref) <= 1e-5 * abs(e_ref)
    # reaction field at 96 points (inside and outside the surface) and the forces on 64 of the
    # 6,000 charges, at full size, against the oracle
    rng = np.random.default_rng(9)
    c = V.mean(axis=0)
    pts = np.concatenate([Q[rng.choice(Q.shape[0], 64, replace=False), :3] + 0.3 * rng.normal(size=(64, 3)),
                          c + rng.normal(size=(32, 3)) * 40.0])
    f_ref = orc.reaction_field(u, pts)
    assert np.max(np.abs(s.reaction_field(pts) - f_ref)) <= 5e-5 * np.max(np.abs(f_ref))
    k = np.sort(rng.choice(Q.shape[0], 64, replace=False))
    fk_ref = 4 * np.pi * 332.0716 * Q[k, 3:4] * orc.reaction_field(u, Q[k, :3])
    assert np.max(np.abs(s.reaction_forces()[k] - fk_ref)) <= 5e-5 * np.max(np.abs(fk_ref))
    # fast summation at full size: on this smooth u the far (approximated) part carries more of
    # each row than on a random vector, so the treecode's deviation from the direct operator is
    # larger here (measured 1.2e-5 relative L2, against 7.8e-7 on a random u); energy within 1e-5
    f = hobi.Solver(V, F, N, Q, 2.0, 80.0, KAPPA, precision="fp32", fast_degree=5, fast_theta=0.7)
    d_au = s.matvec(u)
    assert np.linalg.norm(f.matvec(u) - d_au) <= 3e-5 * np.linalg.norm(d_au)
    f.solve(1e-6, 400)
    assert abs(f.energy() - e_ref) <= 1e-5 * abs(e_ref)


def _c4_member(m):
    n_atoms = int(round(np.exp(np.random.default_rng(1000 + m).uniform(np.log(50), np.log(2000)))))
    return synth.synthetic_molecule(n_atoms, 1000 + m)


def test_c4_batch_sampled_rows():
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        mols = pool.map(_c4_member, range(64))
    b = hobi.BatchSolver(mols, 2.0, 80.0, KAPPA, precision="fp32")
    phis, dphis, info = b.solve(1e-6, 400)
    assert info["converged"]
    E = b.energy()
    # the batch's operator applied to every molecule's solution at once
    uc = np.zeros(2 * b.nv_total)
    for k in range(len(mols)):
        o = 2 * int(b.vert_off[k])
        nv = mols[k][0].shape[0]
        uc[o:o + nv], uc[o + nv:o + 2 * nv] = np.asarray(phis[k]), np.asarray(dphis[k])
    Auc = b.matvec(uc)
    checked = 0
    for k in range(len(mols)):
        V, F, N, Q = mols[k]
        orc = oracle.Problem(V, F, N, Q, 2.0, 80.0, KAPPA)
        o = 2 * int(b.vert_off[k])
        u = uc[o:o + 2 * orc.nv]
        rows = boundary_rows(orc.nv, 32, 2 + k)
        assert rows.size >= 32
        _check_rows(Auc[o:o + 2 * orc.nv], orc.matvec_rows(u, rows), rows, orc.nv, 5e-5)
        e_ref = orc.energy(u)
        assert abs(E[k] - e_ref) <= 1e-5 * abs(e_ref), k
        checked += rows.size
    assert checked >= 64 * 32


def test_no_charges_gives_zero_solution_and_energy():
    V, F, N = synth.icosphere(3, 5.0)
    s = hobi.Solver(V, F, N, np.zeros((0, 4)), 1.0, 80.0, KAPPA, precision="fp32")
    assert np.all(s.rhs() == 0.0)
    phi, dphi, info = s.solve(1e-6, 50, raise_on_fail=False)
    assert np.all(phi == 0.0) and np.all(dphi == 0.0)
    assert s.energy() == 0.0
