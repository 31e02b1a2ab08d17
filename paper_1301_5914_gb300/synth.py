"""Seeded synthetic inputs for the HOBI-PB solver: meshes, normals and charges.

This module only *makes inputs*. It holds none of the solver's arithmetic
(no quadrature, no kernels, no curved geometry), so both the CUDA library and
the FP64 CPU oracle can be fed from it without sharing method code.

Workloads (sizes and seeds are the ones the tests and the benchmark use):

* ``icosphere(level, radius)``: the uniform icosahedral triangulation the
  paper uses for spheres (Sec. 3.2, "ico"), with vertices projected exactly
  onto the sphere (the radial projection of Sec. 2) and exact unit normals.
  Level L has 20*4**L faces and 10*4**L + 2 vertices.
* ``ball_charges(n, r_max, seed)``: n point charges uniform in a ball with
  values uniform in [-1, 1] e (the Kirkwood multi-charge sphere test).
* ``synthetic_molecule(...)``: a globular "protein" stand-in for the paper's
  1ajj workload (Sec. 3.4): seeded atoms, a Gaussian-density isosurface
  extracted by marching tetrahedra, analytic density-gradient normals.

All arrays are float64 / int32, C-contiguous. Faces are counter-clockwise
seen from outside (outward normals by the right-hand rule).
"""
from __future__ import annotations

import math
import os

import numpy as np

__all__ = [
    "icosphere",
    "ball_charges",
    "point_charge",
    "synthetic_molecule",
    "two_globule_complex",
    "mesh_stats",
]


def _icosahedron():
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array(
        [
            [-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
            [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
            [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1],
        ],
        dtype=np.float64,
    )
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    return v, f


def _orient_outward(v: np.ndarray, f: np.ndarray) -> np.ndarray:
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    cr = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", cr, a + b + c) < 0.0
    f = f.copy()
    f[flip, 1], f[flip, 2] = f[flip, 2].copy(), f[flip, 1].copy()
    return f


def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Return (V[nv,3], F[nf,3] int32, N[nv,3]) of a subdivided icosahedron.

    Every vertex is projected onto the sphere of the given radius and its
    normal is the exact radial unit vector.
    """
    if level < 0:
        raise ValueError("level must be >= 0")
    v, f = _icosahedron()
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    f = _orient_outward(v, f)
    for _ in range(level):
        nv = v.shape[0]
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        key = np.minimum(e[:, 0], e[:, 1]) * (nv + 1) + np.maximum(e[:, 0], e[:, 1])
        uniq, inv = np.unique(key, return_inverse=True)
        a = uniq // (nv + 1)
        b = uniq % (nv + 1)
        mid = v[a] + v[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid], axis=0)
        nf = f.shape[0]
        m01 = nv + inv[:nf]
        m12 = nv + inv[nf:2 * nf]
        m20 = nv + inv[2 * nf:]
        f = np.concatenate(
            [
                np.stack([f[:, 0], m01, m20], 1),
                np.stack([f[:, 1], m12, m01], 1),
                np.stack([f[:, 2], m20, m12], 1),
                np.stack([m01, m12, m20], 1),
            ],
            axis=0,
        )
    n = v / np.linalg.norm(v, axis=1, keepdims=True)
    verts = n * float(radius) + np.asarray(center, dtype=np.float64)[None, :]
    return (
        np.ascontiguousarray(verts, dtype=np.float64),
        np.ascontiguousarray(f, dtype=np.int32),
        np.ascontiguousarray(n, dtype=np.float64),
    )


def point_charge(x: float, y: float, z: float, q: float = 1.0) -> np.ndarray:
    """One charge as an [1,4] array (x, y, z in Angstrom; q in e)."""
    return np.array([[x, y, z, q]], dtype=np.float64)


def ball_charges(n: int, r_max: float, seed: int, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """n charges uniform in the ball |x - center| <= r_max, q ~ U[-1, 1] e.

    Radius r_max * U**(1/3) and a uniformly random direction (normalised
    Gaussian vector), drawn from numpy's PCG64 generator.
    """
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = r_max * rng.random(n) ** (1.0 / 3.0)
    q = rng.uniform(-1.0, 1.0, n)
    out = np.empty((n, 4), dtype=np.float64)
    out[:, :3] = d * r[:, None] + np.asarray(center, dtype=np.float64)[None, :]
    out[:, 3] = q
    return out


# ---------------------------------------------------------------------------
# Synthetic molecules (stand-in for the paper's MSMS surfaces of 1ajj)
# ---------------------------------------------------------------------------

_BETA = 1.0  # Gaussian density sharpness: rho = sum exp(-beta (|x-c|^2/R^2 - 1))
_PROBE = 0.6  # radius inflation (A) that closes most inter-atom tunnels, like a solvent probe
_CUT2 = 20.0  # density terms beyond |x-c| = 4.47 R are dropped (exp(-19) relative)


def _place_atoms(n_atoms: int, ball_radius: float, rng) -> tuple[np.ndarray, np.ndarray]:
    """Sequential random packing: reject a candidate closer than 0.8 (Ri + Rj) to a placed atom."""
    centers = np.empty((n_atoms, 3))
    radii = np.empty(n_atoms)
    cell = 3.2  # >= 0.8 * (2.0 + 2.0): neighbours of a candidate sit in the 27 surrounding cells
    grid: dict = {}
    k = 0
    tries = 0
    while k < n_atoms:
        tries += 1
        if tries > 5000 * n_atoms:
            raise RuntimeError("atom packing failed; ball too small")
        c = rng.uniform(-ball_radius, ball_radius, 3)
        if c @ c > ball_radius * ball_radius:
            continue
        rad = rng.uniform(1.2, 2.0)
        key = tuple(np.floor(c / cell).astype(int))
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for idx in grid.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                        d = centers[idx] - c
                        if d @ d < (0.8 * (radii[idx] + rad)) ** 2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            continue
        centers[k] = c
        radii[k] = rad
        grid.setdefault(key, []).append(k)
        k += 1
    return centers, radii


def _charges_for(centers: np.ndarray, rng) -> np.ndarray:
    n = centers.shape[0]
    q = rng.normal(0.0, 0.4, n)
    q -= (q.sum() - np.round(q.sum())) / n
    out = np.empty((n, 4))
    out[:, :3] = centers
    out[:, 3] = q
    return out


def _density_grid(centers, radii, lo, shape, h):
    """rho - 1 on the grid lo + h*(i,j,k), each atom adding only inside its cutoff box."""
    rho = np.zeros(shape)
    for a in range(centers.shape[0]):
        R = radii[a]
        rc = R * np.sqrt(_CUT2)
        i0 = np.maximum(np.floor((centers[a] - rc - lo) / h).astype(int), 0)
        i1 = np.minimum(np.ceil((centers[a] + rc - lo) / h).astype(int) + 1, np.array(shape))
        xs = [lo[d] + h * np.arange(i0[d], i1[d]) - centers[a, d] for d in range(3)]
        t = (xs[0][:, None, None] ** 2 + xs[1][None, :, None] ** 2 + xs[2][None, None, :] ** 2) / (R * R)
        rho[i0[0]:i1[0], i0[1]:i1[1], i0[2]:i1[2]] += np.exp(-_BETA * (np.minimum(t, _CUT2) - 1.0))
    return rho - 1.0


def _density_points_chunk(P, centers, radii, atoms):
    from scipy.spatial import cKDTree


    rmax = float(radii.max()) * np.sqrt(_CUT2)
    # every (point, atom) pair within rmax, in point order and then atom order
    pairs = cKDTree(P).sparse_distance_matrix(atoms, rmax, output_type="ndarray")
    order = np.lexsort((pairs["j"], pairs["i"]))
    ip = pairs["i"][order].astype(np.int64)
    ia = pairs["j"][order].astype(np.int64)
    d = P[ip] - centers[ia]
    inv_r2 = 1.0 / radii[ia] ** 2
    t = np.einsum("ij,ij->i", d, d) * inv_r2
    g = np.exp(-_BETA * (np.minimum(t, _CUT2) - 1.0)) * (t < _CUT2)
    rho = np.bincount(ip, weights=g, minlength=P.shape[0])
    coef = -2.0 * _BETA * inv_r2 * g
    grad = np.stack([np.bincount(ip, weights=coef * d[:, k], minlength=P.shape[0]) for k in range(3)], 1)
    return rho, grad


def _density_points(P, centers, radii, chunk=4096):
    """rho(P) and grad rho(P) over the atoms within the cutoff (4 R) of each point. Points are
    processed in chunks on a thread pool; each point's sum runs over its atoms in index order, so
    the result does not depend on the chunking or the thread count."""
    import concurrent.futures as cf

    from scipy.spatial import cKDTree

    atoms = cKDTree(centers)
    n = P.shape[0]
    if n <= chunk:
        return _density_points_chunk(P, centers, radii, atoms)
    parts = [(a, min(n, a + chunk)) for a in range(0, n, chunk)]
    with cf.ThreadPoolExecutor(max_workers=min(len(parts), os.cpu_count() or 1)) as ex:
        res = list(ex.map(lambda ab: _density_points_chunk(P[ab[0]:ab[1]], centers, radii, atoms), parts))
    return np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res])


def _density(points: np.ndarray, centers: np.ndarray, radii: np.ndarray):
    return _density_points(points, centers, radii)


# The six tetrahedra of a cube that share the main diagonal 0-6 (cube corners
# numbered by bits x + 2y + 4z in the order below), each listed with positive
# orientation. The decomposition is conforming across neighbouring cubes.
_CUBE = np.array(
    [[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]],
    dtype=np.int64,
)
_TETS = np.array(
    [[0, 6, 1, 2], [0, 6, 2, 3], [0, 6, 3, 7], [0, 6, 7, 4], [0, 6, 4, 5], [0, 6, 5, 1]],
    dtype=np.int64,
)


def _marching_tets(field: np.ndarray, origin: np.ndarray, h: float):
    """Triangulate {field > 0} (inside) vs {field <= 0} on a regular grid.

    Vertices lie on grid edges (linear interpolation of the field) and are
    welded by global edge id, so the output is watertight wherever the
    isosurface stays inside the grid. Each triangle is oriented so that its
    right-hand normal points from inside (field > 0) to outside.
    """
    nx, ny, nz = field.shape
    idx = np.arange(nx * ny * nz, dtype=np.int64).reshape(nx, ny, nz)
    cx, cy, cz = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), np.arange(nz - 1), indexing="ij")
    cx, cy, cz = cx.ravel(), cy.ravel(), cz.ravel()
    corner_ids = np.stack(
        [idx[cx + o[0], cy + o[1], cz + o[2]] for o in _CUBE], axis=1
    )  # [ncell, 8]
    inside_c = field.ravel()[corner_ids] > 0.0
    anyin = inside_c.any(axis=1)
    allin = inside_c.all(axis=1)
    keep = anyin & ~allin
    corner_ids = corner_ids[keep]
    tris_a = []  # edge endpoints (global grid ids) of the 3 triangle vertices
    tris_b = []
    fl = field.ravel()
    for tet in _TETS:
        g = corner_ids[:, tet]  # [nc, 4]
        ins = fl[g] > 0.0
        cnt = ins.sum(axis=1)
        for case_cnt in (1, 2, 3):
            sel = cnt == case_cnt
            if not np.any(sel):
                continue
            gs = g[sel]
            ins_s = ins[sel]
            # sort the 4 corners: inside corners first, keeping the permutation parity
            order = np.argsort(~ins_s, axis=1, kind="stable")
            perm = gs[np.arange(gs.shape[0])[:, None], order]
            parity = _perm_parity(order)
            if case_cnt == 1:
                i0 = perm[:, 0]
                o1, o2, o3 = perm[:, 1], perm[:, 2], perm[:, 3]
                a = [np.stack([i0, o1], 1), np.stack([i0, o2], 1), np.stack([i0, o3], 1)]
                tris = [(a[0], a[1], a[2])]
            elif case_cnt == 3:
                i0, i1, i2, o0 = perm[:, 0], perm[:, 1], perm[:, 2], perm[:, 3]
                a = [np.stack([i0, o0], 1), np.stack([i1, o0], 1), np.stack([i2, o0], 1)]
                tris = [(a[0], a[2], a[1])]
            else:
                i0, i1, o0, o1 = perm[:, 0], perm[:, 1], perm[:, 2], perm[:, 3]
                e00 = np.stack([i0, o0], 1)
                e01 = np.stack([i0, o1], 1)
                e10 = np.stack([i1, o0], 1)
                e11 = np.stack([i1, o1], 1)
                tris = [(e00, e01, e11), (e00, e11, e10)]
            for (p, q, r) in tris:
                # orientation fixed below from the field gradient direction
                tris_a.append(np.stack([p, q, r], 1))
                tris_b.append(parity)
    if not tris_a:
        raise RuntimeError("empty isosurface")
    E = np.concatenate(tris_a, axis=0)  # [nt, 3, 2] (inside, outside) grid ids
    # weld: vertex id = unique undirected grid edge
    key = E[:, :, 0] * (nx * ny * nz) + E[:, :, 1]
    ukey, inv = np.unique(key.ravel(), return_inverse=True)
    ein = ukey // (nx * ny * nz)
    eout = ukey % (nx * ny * nz)
    fin, fout = fl[ein], fl[eout]
    t = fin / (fin - fout)
    pin = np.stack(np.unravel_index(ein, (nx, ny, nz)), 1).astype(np.float64)
    pout = np.stack(np.unravel_index(eout, (nx, ny, nz)), 1).astype(np.float64)
    verts = origin[None, :] + h * (pin + t[:, None] * (pout - pin))
    faces = inv.reshape(-1, 3)
    # orient: normal must point from the inside grid point toward the outside one
    a, b, c = verts[faces[:, 0]], verts[faces[:, 1]], verts[faces[:, 2]]
    cr = np.cross(b - a, c - a)
    outdir = (pout - pin)[inv.reshape(-1, 3)[:, 0]]
    flip = np.einsum("ij,ij->i", cr, outdir) < 0.0
    faces[flip, 1], faces[flip, 2] = faces[flip, 2].copy(), faces[flip, 1].copy()
    return verts, faces


def _perm_parity(order: np.ndarray) -> np.ndarray:
    o = order.copy()
    n = o.shape[1]
    par = np.zeros(o.shape[0], dtype=np.int64)
    for i in range(n):
        for j in range(i + 1, n):
            par += o[:, i] > o[:, j]
    return par & 1


def _clean_mesh(v: np.ndarray, f: np.ndarray, min_area_frac: float = 1e-6):
    """Collapse degenerate triangles, keep the largest edge-connected component."""
    # collapse vertices that coincide (zero-length edges from grid corners on the surface)
    q = np.round(v / 1e-9).astype(np.int64)
    _, first, inv = np.unique(q, axis=0, return_index=True, return_inverse=True)
    inv = inv.ravel()
    f = inv[f]
    v = v[first]
    ok = (f[:, 0] != f[:, 1]) & (f[:, 1] != f[:, 2]) & (f[:, 2] != f[:, 0])
    f = f[ok]
    # drop duplicate faces (same vertex set)
    srt = np.sort(f, axis=1)
    _, ui, cnt = np.unique(srt, axis=0, return_index=True, return_counts=True)
    dup_keys = set(map(tuple, np.unique(srt, axis=0)[cnt > 1]))
    if dup_keys:
        keep = np.array([tuple(s) not in dup_keys for s in srt])
        f = f[keep]
    # connected components over shared edges
    nf = f.shape[0]
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], 0)
    ek = np.minimum(e[:, 0], e[:, 1]) * (v.shape[0] + 1) + np.maximum(e[:, 0], e[:, 1])
    fid = np.tile(np.arange(nf), 3)
    order = np.argsort(ek, kind="stable")
    ek_s, fid_s = ek[order], fid[order]
    parent = np.arange(nf)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    same = np.nonzero(ek_s[1:] == ek_s[:-1])[0]
    for s in same:
        a, b = find(fid_s[s]), find(fid_s[s + 1])
        if a != b:
            parent[a] = b
    roots = np.array([find(i) for i in range(nf)])
    lab, counts = np.unique(roots, return_counts=True)
    big = lab[np.argmax(counts)]
    f = f[roots == big]
    used = np.unique(f)
    remap = -np.ones(v.shape[0], dtype=np.int64)
    remap[used] = np.arange(used.size)
    return v[used], remap[f]


def _is_closed_manifold(f: np.ndarray) -> bool:
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], 0)
    n = int(f.max()) + 1
    directed = e[:, 0] * n + e[:, 1]
    rev = e[:, 1] * n + e[:, 0]
    if np.unique(directed).size != directed.size:
        return False
    return bool(np.all(np.isin(rev, directed)))


def _face_normals(V, F):
    cr = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    return cr / np.maximum(np.linalg.norm(cr, axis=1, keepdims=True), 1e-300)


def _project(V, centers, radii, max_step):
    """Two Newton steps onto rho = 1 along grad rho, each step length-limited."""
    for _ in range(2):
        rho, g = _density_points(V, centers, radii)
        g2 = np.einsum("ij,ij->i", g, g)
        ok = g2 > 1e-20
        step = np.zeros_like(V)
        step[ok] = ((rho[ok] - 1.0) / g2[ok])[:, None] * g[ok]
        ln = np.linalg.norm(step, axis=1, keepdims=True)
        step *= np.minimum(1.0, max_step / np.maximum(ln, 1e-300))
        V = V - step
    return V


def _smooth_on_surface(V, F, centers, radii, iters=6, step=0.5):
    """Tangential Laplacian smoothing (step-limited) with projection back onto rho = 1."""
    nv = V.shape[0]
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]], 0)
    deg = np.bincount(e[:, 0], minlength=nv).astype(np.float64)
    h = float(np.median(np.linalg.norm(V[e[:, 0]] - V[e[:, 1]], axis=1)))
    for _ in range(iters):
        nb = np.stack([np.bincount(e[:, 0], weights=V[e[:, 1], k], minlength=nv) for k in range(3)], 1)
        lap = nb / deg[:, None] - V
        _, g = _density_points(V, centers, radii)
        n = g / np.maximum(np.linalg.norm(g, axis=1, keepdims=True), 1e-300)
        lap -= np.einsum("ij,ij->i", lap, n)[:, None] * n
        ln = np.linalg.norm(lap, axis=1, keepdims=True)
        lap *= np.minimum(1.0, 0.3 * h / np.maximum(ln, 1e-300))
        V = _project(V + step * lap, centers, radii, 0.3 * h)
    return V


def _surface(centers, radii, grid_h, pad=3.0, smooth_iters=6):
    R = radii + _PROBE
    lo = (centers - R[:, None]).min(axis=0) - pad
    hi = (centers + R[:, None]).max(axis=0) + pad
    lo = lo - 0.3183098861837907 * grid_h  # irrational offset: no grid point sits on the isosurface
    shape = tuple((np.ceil((hi - lo) / grid_h).astype(int) + 1).tolist())
    field = _density_grid(centers, R, lo, shape, grid_h)
    # keep grid values away from the isovalue so no surface vertex lands within 5% of a cell
    # corner (prevents sliver triangles); the crossing moves by at most that much
    eps = 0.05 * np.median(np.abs(np.diff(field, axis=0))) + 1e-12
    small = np.abs(field) < eps
    field[small] = np.where(field[small] >= 0.0, eps, -eps)
    v, f = _marching_tets(field, lo, grid_h)
    v, f = _clean_mesh(v, f)
    if smooth_iters:
        v = _smooth_on_surface(v, f, centers, R, iters=smooth_iters)
    _, grad = _density_points(v, centers, R)
    n = -grad / np.linalg.norm(grad, axis=1, keepdims=True)
    return v, f, n


def synthetic_molecule(n_atoms: int, seed: int, ball_radius: float | None = None, n_faces: int | None = None,
                       grid_h: float | None = None, centers=None, radii=None):
    """Seeded globular molecule and its Gaussian-density surface (stand-in for the paper's
    MSMS surfaces of protein 1ajj, Sec. 3.4).

    Atoms: sequential random packing in a ball (radius 20 A * (n_atoms/1000)**(1/3) by
    default), radii U[1.2, 2.0] A; charges N(0, 0.4) e shifted so the net charge is an integer.
    Surface: {rho = 1}, rho = sum_a exp(-(|x - c_a|^2/(R_a + 0.6)^2 - 1)), by marching
    tetrahedra; the largest component is kept, vertices are smoothed tangentially (6 passes) and
    projected back onto the isosurface, normals are -grad rho/|grad rho| (analytic). The grid spacing is
    grid_h, or chosen to give about n_faces triangles (default 40 per atom).

    Returns (V, F, N, charges[n,4]).
    """
    rng = np.random.default_rng(seed)
    if centers is None:
        if ball_radius is None:
            ball_radius = 20.0 * (n_atoms / 1000.0) ** (1.0 / 3.0)
        centers, radii = _place_atoms(n_atoms, ball_radius, rng)
    charges = _charges_for(centers, rng)
    if grid_h is None:
        # smoothing leaves the triangle count unchanged: search the spacing on raw extractions
        target = n_faces if n_faces is not None else 40 * centers.shape[0]
        grid_h = 1.0
        for _ in range(2):
            _, f, _ = _surface(centers, radii, grid_h, smooth_iters=0)
            if abs(f.shape[0] / target - 1.0) < 0.1:
                break
            grid_h = grid_h * np.sqrt(f.shape[0] / target)
    v, f, n = _surface(centers, radii, grid_h)
    return (
        np.ascontiguousarray(v, dtype=np.float64),
        np.ascontiguousarray(f, dtype=np.int32),
        np.ascontiguousarray(n, dtype=np.float64),
        np.ascontiguousarray(charges, dtype=np.float64),
    )


def two_globule_complex(n_atoms_each: int, seed_a: int, seed_b: int, n_faces: int | None = None):
    """Two seeded globules in contact (centres 2*R_g - 2 A apart), one surface."""
    rg = 20.0 * (n_atoms_each / 1000.0) ** (1.0 / 3.0)
    ca, ra = _place_atoms(n_atoms_each, rg, np.random.default_rng(seed_a))
    cb, rb = _place_atoms(n_atoms_each, rg, np.random.default_rng(seed_b))
    cb = cb + np.array([2.0 * rg - 2.0, 0.0, 0.0])
    centers = np.concatenate([ca, cb], 0)
    radii = np.concatenate([ra, rb], 0)
    return synthetic_molecule(2 * n_atoms_each, seed_a * 1000 + seed_b, centers=centers,
                              radii=radii, n_faces=n_faces)


def mesh_stats(V: np.ndarray, F: np.ndarray) -> dict:
    """Counts and closedness (a cheap host check used by the generators' tests)."""
    return {
        "n_v": int(V.shape[0]),
        "n_f": int(F.shape[0]),
        "closed_oriented": _is_closed_manifold(np.asarray(F, dtype=np.int64)),
        "euler": int(V.shape[0]) - int(F.shape[0]) * 3 // 2 + int(F.shape[0]),
    }
