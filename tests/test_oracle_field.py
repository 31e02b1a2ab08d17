"""Pins of the oracle's reaction field (-grad phi_reac at off-surface points), on the CPU.

The field is written from the gradients of G0 and G_kappa (oracle/hobi_oracle.c,
or_reaction_field); each pin checks it against something computed another way:
- central differences of the oracle's reaction potential (its own kernels K1, K2), on random
  densities, for kappa = 0, a Debye length of 8 A and kappa = 1;
- inversion symmetry: a centred charge in an icosphere gives zero field at the centre;
- the Kirkwood series (a sphere with an off-centre charge): the field converges to the central
  differences of the analytic reaction potential as the mesh is refined.
"""
import numpy as np
import pytest

import oracle
from oracle import kirkwood as kw
from paper_1301_5914_gb300 import synth


def _fd_field(p, u, pts, h):
    g = np.zeros((pts.shape[0], 3))
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        g[:, c] = -(p.reaction_potential(u, pts + e) - p.reaction_potential(u, pts - e)) / (2 * h)
    return g


@pytest.mark.parametrize("kappa", [0.0, 0.1257, 1.0])
def test_field_is_minus_the_gradient_of_the_reaction_potential(kappa):
    V, F, N = synth.icosphere(2, 3.0)
    Q = synth.ball_charges(3, 1.5, 21)
    p = oracle.Problem(V, F, N, Q, 2.0, 80.0, kappa)
    u = np.random.default_rng(3).normal(size=2 * p.nv)
    pts = synth.ball_charges(8, 2.0, 22)[:, :3]
    f = p.reaction_field(u, pts)
    fd = _fd_field(p, u, pts, 1e-4)
    assert f.shape == (8, 3)
    # central differences: truncation ~h^2 phi''' and rounding ~1e-16 |phi| / h (measured 7e-9)
    assert np.max(np.abs(f - fd)) <= 1e-7 * np.max(np.abs(f)), np.max(np.abs(f - fd)) / np.max(np.abs(f))


def test_centred_charge_gives_zero_field_at_the_centre():
    V, F, N = synth.icosphere(3, 2.0)
    Q = synth.point_charge(0, 0, 0, 1.0)
    p = oracle.Problem(V, F, N, Q, 1.0, 80.0, 0.5)
    u = p.gmres(1e-12)[0]
    f = p.reaction_field(u, np.array([[0.0, 0.0, 0.0], [0.7, 0.2, -0.3]]))
    # the icosphere is symmetric under x -> -x, so the field at the centre vanishes
    assert np.max(np.abs(f[0])) <= 1e-9 * np.max(np.abs(f[1]))
    assert np.max(np.abs(f[1])) > 0


def test_field_converges_to_the_kirkwood_series():
    """Off-centre charge at (0.5, 0, 0) in a radius-2 sphere, kappa = 0.1257: the oracle's field at
    interior points against central differences of Kirkwood's reaction potential (Gaussian units,
    4 pi times the formulation's), at levels 2 and 3: measured 1.3e-2 -> 3.3e-3 (8.2e-4 at level 4),
    a factor 4 per level."""
    Q = synth.point_charge(0.5, 0, 0, 1.0)
    pts = np.array([[0.0, 0.0, 0.0], [0.8, 0.3, -0.2], [-1.0, 0.5, 0.4], [0.2, -1.2, 0.6]])
    h = 1e-4
    ex = np.zeros((4, 3))
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        ex[:, c] = -(kw.reaction_potential_at(pts + e, Q, 2.0, 1.0, 80.0, 0.1257) -
                     kw.reaction_potential_at(pts - e, Q, 2.0, 1.0, 80.0, 0.1257)) / (2 * h) / (4 * np.pi)
    errs = []
    for L in (2, 3):
        V, F, N = synth.icosphere(L, 2.0)
        p = oracle.Problem(V, F, N, Q, 1.0, 80.0, 0.1257)
        u = p.gmres(1e-10)[0]
        errs.append(np.abs(p.reaction_field(u, pts) - ex).max() / np.abs(ex).max())
    assert errs[1] < errs[0] / 3 and errs[1] < 4e-3, errs


@pytest.mark.parametrize("kappa", [0.0, 0.1257])
def test_reaction_forces_are_minus_the_energy_gradient(kappa):
    """The force on charge k, 4 pi C q_k times the reaction field at x_k, against central
    differences of the solvation energy when x_k moves (the surface fixed, a full solve per
    displaced position): the discrete operator keeps the reciprocity that makes these equal,
    measured 2.9e-7 relative for two charges in a level-3 sphere with kappa = 0.1257."""
    V, F, N = synth.icosphere(3, 3.0)
    Q = np.array([[0.6, 0.3, -0.2, 1.0], [-0.5, -0.4, 0.3, -0.7]])

    def solved(Qm):
        p = oracle.Problem(V, F, N, Qm, 2.0, 80.0, kappa)
        return p, p.gmres(1e-12, max_it=400)[0]

    p, u = solved(Q)
    f = p.reaction_forces(u)
    h = 1e-4
    fd = np.zeros((2, 3))
    for k in range(2):
        for c in range(3):
            Qp, Qn = Q.copy(), Q.copy()
            Qp[k, c] += h
            Qn[k, c] -= h
            pp, up = solved(Qp)
            pn, un = solved(Qn)
            fd[k, c] = -(pp.energy(up) - pn.energy(un)) / (2 * h)
    assert np.max(np.abs(f - fd)) <= 2e-6 * np.max(np.abs(fd)), np.max(np.abs(f - fd)) / np.max(np.abs(fd))
