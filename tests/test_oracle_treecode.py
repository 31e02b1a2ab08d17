"""Pins of the oracle's treecode (oracle/treecode.py) to mathematics: exactness of the
barycentric interpolation on polynomials, the tree and batch invariants, the direct-sum limit,
and convergence with the interpolation degree."""
import numpy as np
import pytest

import oracle
from oracle import treecode as tc
from paper_1301_5914_gb300 import synth


def test_lagrange_basis_reproduces_polynomials():
    rng = np.random.default_rng(0)
    for n in (2, 5, 8):
        c = {"lo": np.array([-1.0, 2.0, 0.5]), "hi": np.array([3.0, 2.5, 0.9])}
        ax, half = tc.chebyshev_axes(c, n)
        for d in range(3):
            x = rng.uniform(c["lo"][d], c["hi"][d], size=50)
            L = tc.lagrange_basis(x, ax[d], half[d])
            assert np.allclose(L.sum(axis=1), 1.0, atol=1e-13)          # partition of unity
            for deg in range(n + 1):                                       # exact up to degree n
                p = np.polynomial.Polynomial(rng.normal(size=deg + 1))
                assert np.allclose(L @ p(ax[d]), p(x), rtol=1e-10, atol=1e-10)
            # at the Chebyshev points themselves the basis is the identity
            assert np.allclose(tc.lagrange_basis(ax[d], ax[d], half[d]), np.eye(n + 1))
        # points of the second kind: cos(pi k / n) mapped to the box
        assert np.allclose(ax[0], 1.0 + 2.0 * np.cos(np.pi * np.arange(n + 1) / n))


def test_tree_and_batch_invariants():
    rng = np.random.default_rng(1)
    P = rng.normal(size=(5000, 3)) * [3.0, 1.0, 0.2]
    cl, perm = tc.build_tree(P, 64)
    assert sorted(perm.tolist()) == list(range(len(P)))
    for c in cl:
        pts = P[perm[c["begin"]:c["end"]]]
        assert np.all(pts >= c["lo"] - 1e-15) and np.all(pts <= c["hi"] + 1e-15)
        if c["children"]:
            rng_ = [(cl[k]["begin"], cl[k]["end"]) for k in c["children"]]
            assert rng_[0][0] == c["begin"] and rng_[-1][1] == c["end"]
            assert all(a[1] == b[0] for a, b in zip(rng_, rng_[1:]))     # children partition the parent
        else:
            assert c["end"] - c["begin"] <= 64
    b, order = tc.kd_batches(P, 256)
    assert sorted(order.tolist()) == list(range(len(P)))
    sizes = [x["end"] - x["begin"] for x in b]
    assert max(sizes) <= 256 and sum(sizes) == len(P)
    assert sum(s == 256 for s in sizes) >= len(P) // 256 - 1


@pytest.fixture(scope="module")
def small_problem():
    V, F, N = synth.icosphere(3, 6.0)
    orc = oracle.Problem(V, F, N, synth.ball_charges(4, 4.0, 3), 1.0, 80.0, 0.3)
    u = np.random.default_rng(2).normal(size=2 * orc.nv)
    return orc, u, tc.direct_far(orc, u)


def test_treecode_reduces_to_direct_sum(small_problem):
    orc, u, (d1, d2) = small_problem
    st = {}
    t1, t2 = tc.treecode_far(orc, u, 4, 1e-3, leaf=64, batch=64, stats=st)
    assert st["approx_pairs"] == 0 and st["direct_pairs"] == orc.nv * 4 * orc.nf
    assert np.allclose(t1, d1, rtol=1e-12, atol=1e-12 * np.abs(d1).max())
    assert np.allclose(t2, d2, rtol=1e-12, atol=1e-12 * np.abs(d2).max())


def test_treecode_error_falls_with_degree(small_problem):
    orc, u, (d1, d2) = small_problem
    errs = []
    for n in (2, 4, 6):
        st = {}
        t1, t2 = tc.treecode_far(orc, u, n, 0.9, leaf=32, batch=64, stats=st)
        assert st["approx_pairs"] > 0
        errs.append(max(np.linalg.norm(t1 - d1) / np.linalg.norm(d1), np.linalg.norm(t2 - d2) / np.linalg.norm(d2)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-4 and errs[0] / errs[2] > 10


def test_direct_far_is_the_regular_rule_kernel_sum():
    """The module's pair formula and node densities against the oracle's kernels K1-K4 (pinned
    to finite differences of G0 and G_kappa) summed node by node with the regular-rule weights
    W_{j,m,n}; and the oracle's matvec rows rebuilt from that sum, the diagonal and the 16-point
    rule on the incident faces (Eqs. (17)-(20))."""
    V, F, N = synth.icosphere(1, 2.0)
    orc = oracle.Problem(V, F, N, synth.ball_charges(2, 1.2, 5), 1.0, 80.0, 0.3)
    u = np.random.default_rng(4).normal(size=2 * orc.nv)
    nv, eps = orc.nv, orc.eps
    y, nu, W = orc.nodes()
    nx = tc.target_normals(orc)
    d1, d2 = tc.direct_far(orc, u)
    Au = orc.matvec(u)
    for i in range(nv):
        K = np.array([[oracle.kernels(V[i], nx[i], y[j, m], nu[j, m], eps, orc.kappa) for m in range(4)]
                      for j in range(orc.nf)])                                # [face, node, kernel]
        R = np.einsum("jmn,jmq->jnq", W, K)                                   # regular-rule coefficients
        un, uu = u[nv + F], u[F]                                              # [face, corner]
        r1 = np.sum(R[:, :, 0] * un + R[:, :, 1] * uu)
        r2 = np.sum(R[:, :, 2] * un + R[:, :, 3] * uu)
        assert abs(d1[i] - r1) <= 1e-12 * max(1.0, abs(r1))
        assert abs(d2[i] - r2) <= 1e-12 * max(1.0, abs(r2))
        # incident faces: the 16-point rule replaces the regular rule
        c1 = c2 = 0.0
        for j in np.flatnonzero((F == i).any(axis=1)):
            S = orc.singular_coeffs(i, j) - R[j]
            c1 += np.sum(S[:, 0] * un[j] + S[:, 1] * uu[j])
            c2 += np.sum(S[:, 2] * un[j] + S[:, 3] * uu[j])
        assert abs(Au[i] - (0.5 * (1 + eps) * u[i] - r1 - c1)) <= 1e-10 * np.abs(Au[:nv]).max()
        assert abs(Au[nv + i] - (0.5 * (1 + 1 / eps) * u[nv + i] - r2 - c2)) <= 1e-10 * np.abs(Au[nv:]).max()
