"""Pins of the oracle's low-order LOBI-PB scheme (Sec. 2.4, eqdbef1/eqdbef2): flat triangles,
centroid collocation, self triangle dropped."""
import numpy as np

import oracle
from oracle import kirkwood as kw
from paper_1301_5914_gb300 import synth


def _born(L):
    V, F, N = synth.icosphere(L, 2.0)
    Q = synth.point_charge(0, 0, 0, 1.0)
    p = oracle.LobiProblem(V, F, N, Q, 1.0, 80.0, 0.0)
    u, it, conv, _ = p.gmres(1e-8)
    assert conv
    x, n, A = p.geometry()
    phi_ex = 1.0 / (4 * np.pi * 80 * 2.0)
    return p, u, abs(u[: p.nf] - phi_ex).max() / phi_ex, p.energy(u)


def test_lobi_geometry_is_flat_faces():
    V, F, N = synth.icosphere(1, 2.0)
    p = oracle.LobiProblem(V, F, N, np.zeros((0, 4)), 1.0, 80.0, 0.0)
    x, n, A = p.geometry()
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    assert np.allclose(x, (a + b + c) / 3)
    cr = np.cross(b - a, c - a)
    assert np.allclose(A, 0.5 * np.linalg.norm(cr, axis=1))
    assert np.allclose(n, cr / np.linalg.norm(cr, axis=1, keepdims=True))


def test_lobi_born_half_order_and_table1_band():
    """Table 1 (LOBI-PB column): surface-potential error converges at about half order in the
    density d, and E_sol approaches -81.98 from below (-83.41 at d = 5 ... -82.43 at d = 80)."""
    out = [_born(L) for L in (2, 3, 4)]
    e = [o[2] for o in out]
    E = [o[3] for o in out]
    orders = [np.log(e[k] / e[k + 1]) / np.log(4.0) for k in range(2)]
    assert all(0.35 < o < 0.8 for o in orders), orders
    assert E[0] < E[1] < E[2] < -81.98
    assert abs(E[2] - (-82.60)) < 0.3  # level 4 (d = 51) vs Table 1 at d = 40


def test_lobi_double_layer_identity_kappa0():
    """kappa = 0: A [1; 0] = [eps; 0]; the dropped self term is exact for the flat double layer
    (d . n_j = 0 on the own panel), so the residual is the centroid-rule error, falling with h."""
    errs = []
    for L in (2, 3):
        V, F, N = synth.icosphere(L, 2.0)
        p = oracle.LobiProblem(V, F, N, np.zeros((0, 4)), 1.0, 80.0, 0.0)
        u = np.zeros(2 * p.nf)
        u[: p.nf] = 1.0
        Au = p.matvec(u)
        assert np.max(np.abs(Au[p.nf:])) == 0.0
        errs.append(np.max(np.abs(Au[: p.nf] - 80.0)))
    assert errs[1] < errs[0] and errs[1] < 2.0


def test_lobi_gmres_matches_dense_lu_and_hobi_agrees():
    V, F, N = synth.icosphere(2, 2.0)
    Q = synth.ball_charges(3, 1.2, 3)
    p = oracle.LobiProblem(V, F, N, Q, 1.0, 80.0, 0.5)
    u, it, conv, _ = p.gmres(1e-12)
    u_lu = np.linalg.solve(p.dense(), p.rhs())
    assert conv and np.linalg.norm(u - u_lu) / np.linalg.norm(u_lu) < 1e-10
    # both schemes approach the Kirkwood energy; HOBI is the closer one
    e_ex = kw.solvation_energy(Q, 2.0, 1.0, 80.0, 0.5)
    ph = oracle.Problem(V, F, N, Q, 1.0, 80.0, 0.5)
    uh, _, _, _ = ph.gmres(1e-10)
    assert abs(ph.energy(uh) - e_ex) < abs(p.energy(u) - e_ex) < 0.1 * abs(e_ex)
