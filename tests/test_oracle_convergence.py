"""Why the centred-charge potential converges slowly on icospheres (oracle, CPU).

For kappa = 0 the first row of A [1; 0] is (1/2)(1 + eps) - (eps - 1) * (double-layer integral),
and the double-layer integral of a closed surface at a smooth surface point is exactly 1/2
(Gauss), so the discrete row equals eps up to quadrature error. The centred-charge error e_phi is
this quadrature error (the exact surface values are constant). These pins show that it falls
as O(h) (order 1/2 in the vertex density d) and that it comes almost entirely from the regular
4-point rule on the faces next to the incident ones, with the 16-point singular rule on the
incident faces a much smaller part: refining those two rules on a few vertices (Gauss-Legendre
tensor rules under the Duffy map, 48 x 48 on incident faces, 12 x 12 on regular faces within
4 mesh sizes) removes nearly all of it. The paper's Table 2 rule (4-point "Gauss-Radau", nodes not
printed) may have a smaller error constant on such near faces; the reading used here is the
degree-3 collapsed rule.
"""
import numpy as np
import pytest

import oracle
from paper_1301_5914_gb300 import synth

A, EPS = 2.0, 80.0


def _problem(level):
    V, F, N = synth.icosphere(level, A)
    return V, F, N, oracle.Problem(V, F, N, synth.point_charge(0.0, 0.0, 0.0, 1.0), 1.0, EPS, 0.0)


def _identity_error(p, rows):
    u = np.zeros(2 * p.nv)
    u[: p.nv] = 1.0
    r1, _ = p.matvec_rows(u, rows)
    return (r1 - EPS) / (EPS - 1.0) / 0.5  # relative error of the discrete double-layer integral


def _generic_rows(F, nv, k, seed):
    """k vertices of valence 6 (the 12 original icosahedron vertices have valence 5)."""
    val = np.bincount(F.reshape(-1), minlength=nv)
    cand = np.where(val == 6)[0]
    return np.sort(np.random.default_rng(seed).choice(cand, size=k, replace=False))


def test_identity_error_falls_as_h():
    worst = []
    for L in (3, 4, 5):
        V, F, N, p = _problem(L)
        rows = _generic_rows(F, V.shape[0], 40, L)
        worst.append(np.max(np.abs(_identity_error(p, rows))))
    # measured 2.7e-5, 1.6e-5, 8.3e-6 (4.0e-6 at level 6): halves per level = first order in h
    assert 1.6 <= worst[1] / worst[2] <= 2.5, worst
    assert worst[2] <= 1.2e-5


def _dense_face(P, x, nx, n):
    """Integral over the curved element P of K2(x, y) L_k(y) dS (k = 1..3) by an n x n
    Gauss-Legendre rule under the Duffy map from the element's first corner."""
    g, w = np.polynomial.legendre.leggauss(n)
    g, w = 0.5 * (g + 1.0), 0.5 * w
    out = np.zeros(3)
    for a in range(n):
        for b in range(n):
            r, s, wt = (1 - g[b]) * g[a], g[b] * g[a], w[a] * w[b] * g[a]
            y, ny, J = oracle.element_eval(P, r, s)
            out += wt * J * np.array([1 - r - s, r, s]) * oracle.kernels(x, nx, y, ny, EPS, 0.0)[1]
    return out


def test_identity_error_is_the_near_face_regular_rule():
    V, F, N, p = _problem(3)
    y, nu, W = p.nodes()
    pts = p.element_points()
    h = np.mean(np.linalg.norm(V[F[:, 0]] - V[F[:, 1]], axis=1))
    cen = y.mean(axis=1)
    for i in _generic_rows(F, V.shape[0], 3, 0):
        err = _identity_error(p, np.array([i]))[0] * (EPS - 1.0) * 0.5  # in row-1 units
        x, nx = V[i], N[i] / np.linalg.norm(N[i])
        inc = np.where((F == i).any(axis=1))[0]
        d_sing = -sum(p.singular_coeffs_n(i, j, 48)[:, 1].sum() - p.singular_coeffs(i, j)[:, 1].sum() for j in inc)
        near = np.where((np.linalg.norm(cen - x, axis=1) < 4 * h) & ~(F == i).any(axis=1))[0]
        d_reg = 0.0
        for j in near:
            k2 = np.array([oracle.kernels(x, nx, y[j, m], nu[j, m], EPS, 0.0)[1] for m in range(4)])
            d_reg -= _dense_face(pts[j], x, nx, 12).sum() - (W[j] * k2[:, None]).sum()
        # refining both rules removes the error: what is left is below 10 % of it
        assert abs(err + d_sing + d_reg) <= 0.1 * abs(err), (i, err, d_sing, d_reg)
        # and the near-face regular rule is the larger part (measured 7-20x the singular part)
        assert abs(d_reg) >= 3 * abs(d_sing), (i, d_reg, d_sing)
