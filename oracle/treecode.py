"""Barycentric Lagrange treecode for the HOBI-PB far-field sum, in plain numpy FP64
(test infrastructure only; the product path never imports this package).

The far field of one matvec (Sec. 2.2-2.3, the regular-rule sum of Eqs. (17)-(18) over
every node of every element, written with sigma = sum_n W u_{N_v+v_n}/4pi, mu = sum_n W u_{v_n}/4pi
and m = mu nu_y) is, for target vertex x with unit normal nu_x, d = x - y, r = |d|,
E = exp(-kappa r), P = E (1 + kappa r), Q = E (3 + 3 kappa r + kappa^2 r^2):

    row1(x) = sum_y (1 - E)/r sigma + (eps P - 1)/r^3 (d . m)
    row2(x) = sum_y (P - 1)/r^3 (nu_x . m) + [(P/eps - 1)/r^3 sigma - (Q - 3)/r^5 (d . m)] (nu_x . d)

The paper evaluates it directly and names fast summation as future work. This module writes out
the barycentric Lagrange treecode (Wang, Tlupova and Krasny, "A kernel-independent treecode based
on barycentric Lagrange interpolation", 2020) for it, with the tree, batch and admissibility
rules of this implementation:

* tree: a cluster is a set of points with its tight bounding box; a cluster of more than `leaf`
  points whose box is not a single point is split into the octants of its box midpoint
  (coordinate > midpoint goes to the upper half; octant index x + 2y + 4z; empty octants
  dropped). Points are listed depth first, so every cluster is a contiguous range.
* target batches: recursive splits of the targets along the longest axis of their tight box
  (sorted by that coordinate, ties by index), the first part holding floor(ceil(c/batch)/2)
  batches' worth, down to sets of at most `batch` targets; each batch's box is the tight box of
  its targets.
* admissibility: batch B and source cluster C interact through C's proxy points when C has more
  than (n+1)^3 points and r_B + r_C < theta |c_B - c_C| (c the box midpoint, r half its
  diagonal); otherwise a leaf C is summed directly and an inner C is opened.
* proxies: the (n+1)^3 tensor Chebyshev points of the second kind of C's box (each half-extent
  raised to at least 1e-3 of the largest), with proxy densities
  q_ijk = sum_{y in C} L_i(y_x) L_j(y_y) L_k(y_z) q_y for q in {sigma, m}, L the barycentric
  Lagrange basis (weights (-1)^i, halved at both ends; a coordinate within 1e-6 half-extents of
  a Chebyshev point takes the Kronecker value). The approximated interaction is the pair
  formula above with the proxies as sources.

The paper prints no fast summation to compare with. The tests pin this module to the direct sum
(a tiny theta gives it to rounding, the error falls with the degree), to polynomial reproduction
and partition of unity of the interpolation, and its pair formula and node densities to the
oracle's kernels K1-K4 (themselves pinned to finite differences of G0 and G_kappa) summed with the
regular-rule weights.
"""
from __future__ import annotations

import numpy as np

HIT_TOL = 1e-6      # in half-extents of the proxy box
MIN_HALF = 1e-3     # smallest half-extent, relative to the largest one


def build_tree(P: np.ndarray, leaf: int):
    """Clusters of the points P (n, 3) and the depth-first order `perm` (tree position -> index).

    Each cluster is a dict: begin, end (range in tree order), lo, hi (tight box), children."""
    P = np.asarray(P, dtype=np.float64)
    clusters, perm = [], []

    def visit(idx):
        pts = P[idx]
        lo, hi = pts.min(axis=0), pts.max(axis=0)
        ci = len(clusters)
        clusters.append({"begin": len(perm), "end": -1, "lo": lo, "hi": hi, "children": []})
        if len(idx) > leaf and np.any(hi > lo):
            mid = 0.5 * (lo + hi)
            code = (pts[:, 0] > mid[0]).astype(int) + 2 * (pts[:, 1] > mid[1]) + 4 * (pts[:, 2] > mid[2])
            for o in range(8):
                sub = idx[code == o]
                if len(sub):
                    clusters[ci]["children"].append(visit(sub))
        else:
            perm.extend(idx.tolist())
        clusters[ci]["end"] = len(perm)
        return ci

    visit(np.arange(len(P)))
    return clusters, np.asarray(perm, dtype=np.int64)


def kd_batches(x: np.ndarray, batch: int):
    """Target batches (dicts with begin, end, lo, hi) and the batch order of the targets.

    A set of c > batch targets is sorted along the longest axis of its tight box (ties by index)
    and split after floor(ceil(c / batch) / 2) * batch targets, so that every batch but the last
    of each split holds exactly `batch` targets."""
    x = np.asarray(x, dtype=np.float64)
    order, batches = [], []

    def visit(idx):
        pts = x[idx]
        lo, hi = pts.min(axis=0), pts.max(axis=0)
        c = len(idx)
        if c <= batch:
            batches.append({"begin": len(order), "end": len(order) + c, "lo": lo, "hi": hi, "children": []})
            order.extend(idx.tolist())
            return
        a = int(np.argmax(hi - lo))
        srt = idx[np.lexsort((idx, pts[:, a]))]
        cut = ((c + batch - 1) // batch // 2) * batch
        visit(srt[:cut])
        visit(srt[cut:])

    visit(np.arange(len(x)))
    return batches, np.asarray(order, dtype=np.int64)


def center_radius(c):
    return 0.5 * (c["lo"] + c["hi"]), 0.5 * float(np.linalg.norm(c["hi"] - c["lo"]))


def interaction_lists(batches, clusters, theta: float, degree: int):
    """Per batch: (direct source clusters, approximated source clusters), in traversal order."""
    n3 = (degree + 1) ** 3
    out = []
    for b in batches:
        cb, rb = center_radius(b)
        direct, approx = [], []

        def visit(ci):
            c = clusters[ci]
            cc, rc = center_radius(c)
            if c["end"] - c["begin"] > n3 and rb + rc < theta * np.linalg.norm(cc - cb):
                approx.append(ci)
            elif not c["children"]:
                direct.append(ci)
            else:
                for ch in c["children"]:
                    visit(ch)

        visit(0)
        out.append((direct, approx))
    return out


def chebyshev_axes(c, degree: int) -> np.ndarray:
    """(3, n+1) Chebyshev points of the second kind along each axis of the cluster's box."""
    mid = 0.5 * (c["lo"] + c["hi"])
    half = 0.5 * (c["hi"] - c["lo"])
    half = np.maximum(half, MIN_HALF * half.max())
    t = np.cos(np.pi * np.arange(degree + 1) / degree)
    return mid[:, None] + half[:, None] * t[None, :], half


def lagrange_basis(x: np.ndarray, s: np.ndarray, half: float) -> np.ndarray:
    """(m, n+1) barycentric Lagrange basis at x for the Chebyshev points s of one axis."""
    n = len(s) - 1
    w = (-1.0) ** np.arange(n + 1)
    w[0] *= 0.5
    w[n] *= 0.5
    diff = x[:, None] - s[None, :]
    hit = np.abs(diff) < HIT_TOL * half
    safe = np.where(hit, 1.0, diff)
    terms = w[None, :] / safe
    L = terms / terms.sum(axis=1, keepdims=True)
    rows = hit.any(axis=1)
    if rows.any():
        L[rows] = 0.0
        first = np.argmax(hit[rows], axis=1)
        L[np.flatnonzero(rows), first] = 1.0
    return L


def proxies(c, y, sigma, m, degree: int):
    """Proxy points (K, 3) and densities sigma (K,), m (K, 3) of cluster c; K = (n+1)^3,
    proxy (i, j, k) at index (i (n+1) + j)(n+1) + k."""
    ax, half = chebyshev_axes(c, degree)
    Lx = lagrange_basis(y[:, 0], ax[0], half[0])
    Ly = lagrange_basis(y[:, 1], ax[1], half[1])
    Lz = lagrange_basis(y[:, 2], ax[2], half[2])
    s_sig = np.einsum("yi,yj,yk,y->ijk", Lx, Ly, Lz, sigma).ravel()
    s_m = np.stack([np.einsum("yi,yj,yk,y->ijk", Lx, Ly, Lz, m[:, a]).ravel() for a in range(3)], axis=1)
    g = np.meshgrid(ax[0], ax[1], ax[2], indexing="ij")
    pts = np.stack([g[0].ravel(), g[1].ravel(), g[2].ravel()], axis=1)
    return pts, s_sig, s_m


def pair_sums(x, nx, y, sigma, m, eps: float, kappa: float):
    """Far-field row sums (row1, row2) at targets x (t, 3) with normals nx from sources y."""
    r1 = np.zeros(len(x))
    r2 = np.zeros(len(x))
    for a in range(0, len(x), 64):
        d = x[a:a + 64, None, :] - y[None, :, :]
        r = np.sqrt((d * d).sum(axis=2))
        E = np.exp(-kappa * r)
        P = E * (1.0 + kappa * r)
        Q = E * (3.0 + 3.0 * kappa * r + kappa * kappa * r * r)
        dm = (d * m[None, :, :]).sum(axis=2)
        r1[a:a + 64] = ((1.0 - E) / r * sigma[None, :] + (eps * P - 1.0) / r**3 * dm).sum(axis=1)
        nd = (d * nx[a:a + 64, None, :]).sum(axis=2)
        nm = m @ nx[a:a + 64].T
        r2[a:a + 64] = ((P - 1.0) / r**3 * nm.T + ((P / eps - 1.0) / r**3 * sigma[None, :]
                                                     - (Q - 3.0) / r**5 * dm) * nd).sum(axis=1)
    return r1, r2


def node_densities(problem, u):
    """Sources of the far field of u: nodes y (N_n, 3), sigma (N_n,), m (N_n, 3)."""
    y, nu, W = problem.nodes()
    F = problem.F
    nv = problem.nv
    c = 1.0 / (4.0 * np.pi)
    sig = np.einsum("jmn,jn->jm", W, u[nv + F]) * c
    mu = np.einsum("jmn,jn->jm", W, u[F]) * c
    return y.reshape(-1, 3), sig.ravel(), (mu[:, :, None] * nu).reshape(-1, 3)


def target_normals(problem):
    return problem.N / np.linalg.norm(problem.N, axis=1, keepdims=True)


def direct_far(problem, u):
    """Direct far field (row1, row2) of u over every node (the sum the treecode approximates)."""
    y, sig, m = node_densities(problem, u)
    return pair_sums(problem.V, target_normals(problem), y, sig, m, problem.eps, problem.kappa)


def treecode_far(problem, u, degree: int, theta: float, leaf: int = 256, batch: int = 256,
                 stats: dict | None = None):
    """Treecode far field (row1, row2) of u."""
    y, sig, m = node_densities(problem, u)
    x, nx = problem.V, target_normals(problem)
    eps, kappa = problem.eps, problem.kappa
    src, sperm = build_tree(y, leaf)
    batches, tperm = kd_batches(x, batch)
    lists = interaction_lists(batches, src, theta, degree)
    cache = {}
    r1 = np.zeros(len(x))
    r2 = np.zeros(len(x))
    n_direct = n_approx = 0
    for b, (direct, approx) in zip(batches, lists):
        ti = tperm[b["begin"]:b["end"]]
        for ci in direct:
            c = src[ci]
            si = sperm[c["begin"]:c["end"]]
            a1, a2 = pair_sums(x[ti], nx[ti], y[si], sig[si], m[si], eps, kappa)
            r1[ti] += a1
            r2[ti] += a2
            n_direct += len(ti) * len(si)
        for ci in approx:
            if ci not in cache:
                c = src[ci]
                si = sperm[c["begin"]:c["end"]]
                cache[ci] = proxies(c, y[si], sig[si], m[si], degree)
            pts, ps, pm = cache[ci]
            a1, a2 = pair_sums(x[ti], nx[ti], pts, ps, pm, eps, kappa)
            r1[ti] += a1
            r2[ti] += a2
            n_approx += len(ti) * len(pts)
    if stats is not None:
        stats.update(direct_pairs=n_direct, approx_pairs=n_approx, batches=len(batches),
                     clusters=len(src), proxy_clusters=len(cache))
    return r1, r2


def treecode_matvec(problem, u, degree: int, theta: float, **kw):
    """The oracle's matvec with its far field replaced by the treecode's:
    A u - (far_treecode - far_direct) for both rows."""
    t1, t2 = treecode_far(problem, u, degree, theta, **kw)
    d1, d2 = direct_far(problem, u)
    return problem.matvec(u) - np.concatenate([t1 - d1, t2 - d2])
