"""FP64 CPU oracle for HOBI-PB (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / ``--impl reference`` legs may import this package. The
product path (the CUDA library under ``paper_1301_5914_gb300``) never calls
it; the two share no code.

The arithmetic lives in ``hobi_oracle.c`` (plain C, double precision, OpenMP
over independent rows) and ``kirkwood.py`` (the analytic sphere solution).
This module only loads the shared library and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hobi_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp, portable flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB)
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    lp = C.POINTER(C.c_int64)
    lib.or_create.restype = C.c_void_p
    lib.or_create.argtypes = [dp, C.c_int64, ip, C.c_int64, dp, dp, C.c_int64, C.c_double,
                              C.c_double, C.c_double]
    lib.or_destroy.argtypes = [C.c_void_p]
    lib.or_get_nodes.argtypes = [C.c_void_p, dp, dp, dp]
    lib.or_get_element_points.argtypes = [C.c_void_p, dp]
    lib.or_singular_coeffs.argtypes = [C.c_void_p, C.c_int64, C.c_int64, dp]
    lib.or_singular_coeffs.restype = C.c_int
    lib.or_singular_coeffs_n.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int, dp, dp, dp]
    lib.or_singular_coeffs_n.restype = C.c_int
    lib.or_matvec.argtypes = [C.c_void_p, dp, dp]
    lib.or_matvec_rows.argtypes = [C.c_void_p, dp, lp, C.c_int64, dp]
    lib.or_rhs.argtypes = [C.c_void_p, dp]
    lib.or_reaction_potential.argtypes = [C.c_void_p, dp, dp, C.c_int64, dp]
    lib.or_reaction_field.argtypes = [C.c_void_p, dp, dp, C.c_int64, dp]
    lib.or_energy.argtypes = [C.c_void_p, dp]
    lib.or_energy.restype = C.c_double
    lib.or_gmres.argtypes = [C.c_void_p, dp, C.c_double, C.c_int, C.c_int, C.c_int, dp, dp,
                             C.POINTER(C.c_int)]
    lib.or_gmres.restype = C.c_int
    lib.or_lobi_geometry.argtypes = [C.c_void_p, dp, dp, dp]
    lib.or_lobi_matvec.argtypes = [C.c_void_p, dp, dp]
    lib.or_lobi_matvec_rows.argtypes = [C.c_void_p, dp, lp, C.c_int64, dp]
    lib.or_lobi_rhs.argtypes = [C.c_void_p, dp]
    lib.or_lobi_energy.argtypes = [C.c_void_p, dp]
    lib.or_lobi_energy.restype = C.c_double
    lib.or_lobi_gmres.argtypes = [C.c_void_p, dp, C.c_double, C.c_int, C.c_int, C.c_int, dp, dp,
                                  C.POINTER(C.c_int)]
    lib.or_lobi_gmres.restype = C.c_int
    lib.or_regular_rule.argtypes = [dp, dp, dp]
    lib.or_gauss_legendre4.argtypes = [dp, dp]
    lib.or_singular_rule.argtypes = [dp, dp, dp]
    lib.or_p3_basis.argtypes = [C.c_double, C.c_double, dp, dp, dp]
    lib.or_edge_arc.argtypes = [dp, dp, dp, dp, C.c_double, dp, dp]
    lib.or_element_points.argtypes = [dp, dp, dp, dp, dp, dp, dp]
    lib.or_element_eval.argtypes = [dp, C.c_double, C.c_double, dp, dp, dp]
    lib.or_kernels.argtypes = [dp, dp, dp, dp, C.c_double, C.c_double, dp]
    lib.or_G.argtypes = [C.c_double] * 7
    lib.or_G.restype = C.c_double
    lib.or_num_threads.restype = C.c_int
    lib.or_set_num_threads.argtypes = [C.c_int]
    _lib = lib
    return lib


def _p(a: np.ndarray, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Rules and geometry primitives (exported for the pin tests)
# ---------------------------------------------------------------------------

def regular_rule():
    lib = _load()
    r, s, w = (np.zeros(4) for _ in range(3))
    lib.or_regular_rule(_p(r), _p(s), _p(w))
    return r, s, w


def gauss_legendre4():
    lib = _load()
    x, w = np.zeros(4), np.zeros(4)
    lib.or_gauss_legendre4(_p(x), _p(w))
    return x, w


def singular_rule():
    lib = _load()
    r, s, w = (np.zeros(16) for _ in range(3))
    lib.or_singular_rule(_p(r), _p(s), _p(w))
    return r, s, w


def p3_basis(r: float, s: float):
    lib = _load()
    N, Nr, Ns = (np.zeros(10) for _ in range(3))
    lib.or_p3_basis(float(r), float(s), _p(N), _p(Nr), _p(Ns))
    return N, Nr, Ns


def edge_arc(P, nP, Q, nQ, t: float):
    lib = _load()
    x, n = np.zeros(3), np.zeros(3)
    lib.or_edge_arc(_p(_f64(P)), _p(_f64(nP)), _p(_f64(Q)), _p(_f64(nQ)), float(t), _p(x), _p(n))
    return x, n


def element_points(X, N):
    """X, N: [3,3] vertex positions and normals -> [10,3] interpolation points."""
    lib = _load()
    X, N = _f64(X), _f64(N)
    out = np.zeros((10, 3))
    lib.or_element_points(_p(X[0]), _p(N[0]), _p(X[1]), _p(N[1]), _p(X[2]), _p(N[2]), _p(out))
    return out


def element_eval(pts, r: float, s: float):
    lib = _load()
    pts = _f64(pts)
    x, nu, J = np.zeros(3), np.zeros(3), np.zeros(1)
    lib.or_element_eval(_p(pts), float(r), float(s), _p(x), _p(nu), _p(J))
    return x, nu, float(J[0])


def kernels(x, nx, y, ny, eps: float, kappa: float) -> np.ndarray:
    lib = _load()
    K = np.zeros(4)
    lib.or_kernels(_p(_f64(x)), _p(_f64(nx)), _p(_f64(y)), _p(_f64(ny)), float(eps), float(kappa), _p(K))
    return K


def green(x, y, kappa: float) -> float:
    lib = _load()
    return float(lib.or_G(*map(float, x), *map(float, y), float(kappa)))


def num_threads() -> int:
    return int(_load().or_num_threads())


def set_num_threads(n: int) -> None:
    _load().or_set_num_threads(int(n))


# ---------------------------------------------------------------------------
# Problem object
# ---------------------------------------------------------------------------

class Problem:
    """One molecule: mesh, vertex normals, charges and dielectric parameters.

    Builds the curved elements and the regular-rule node table on creation.
    """

    def __init__(self, V, F, N, charges, eps1: float, eps2: float, kappa: float):
        lib = _load()
        self.V = _f64(V)
        self.F = np.ascontiguousarray(F, dtype=np.int32)
        self.N = _f64(N)
        self.charges = _f64(charges).reshape(-1, 4)
        self.eps1, self.eps2, self.kappa = float(eps1), float(eps2), float(kappa)
        self.eps = self.eps2 / self.eps1
        self.nv, self.nf, self.nc = self.V.shape[0], self.F.shape[0], self.charges.shape[0]
        self._h = lib.or_create(_p(self.V), self.nv, _p(self.F, C.c_int32), self.nf, _p(self.N),
                                _p(self.charges), self.nc, self.eps1, self.eps2, self.kappa)
        if not self._h:
            raise RuntimeError("oracle: or_create failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_destroy(h)
            self._h = None

    # tables -----------------------------------------------------------
    def nodes(self):
        """Regular-rule nodes: y[nf,4,3], nu[nf,4,3], W[nf,4,3] (W_{j,m,n})."""
        y, nu, W = (np.zeros((self.nf, 4, 3)) for _ in range(3))
        _lib.or_get_nodes(self._h, _p(y), _p(nu), _p(W))
        return y, nu, W

    def element_points(self):
        out = np.zeros((self.nf, 10, 3))
        _lib.or_get_element_points(self._h, _p(out))
        return out

    def singular_coeffs(self, i: int, j: int) -> np.ndarray:
        """[3,4] coefficients (K1..K4 sums) of face j for target vertex i, 16-point rule."""
        out = np.zeros((3, 4))
        if _lib.or_singular_coeffs(self._h, int(i), int(j), _p(out)) != 0:
            raise ValueError("vertex is not a corner of the face")
        return out

    def singular_coeffs_n(self, i: int, j: int, n: int) -> np.ndarray:
        """Same with an n x n Gauss-Legendre Duffy rule (brute force)."""
        x, w = np.polynomial.legendre.leggauss(n)
        x = 0.5 * (x + 1.0)
        w = 0.5 * w
        out = np.zeros((3, 4))
        if _lib.or_singular_coeffs_n(self._h, int(i), int(j), int(n), _p(_f64(x)), _p(_f64(w)), _p(out)) != 0:
            raise ValueError("vertex is not a corner of the face")
        return out

    # operators --------------------------------------------------------
    def rhs(self) -> np.ndarray:
        b = np.zeros(2 * self.nv)
        _lib.or_rhs(self._h, _p(b))
        return b

    def matvec(self, u) -> np.ndarray:
        u = _f64(u)
        assert u.shape == (2 * self.nv,)
        out = np.zeros(2 * self.nv)
        _lib.or_matvec(self._h, _p(u), _p(out))
        return out

    def matvec_rows(self, u, rows) -> tuple[np.ndarray, np.ndarray]:
        """({Au}_i, {Au}_{i+N_v}) for the selected vertex rows i."""
        u = _f64(u)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.zeros((rows.size, 2))
        _lib.or_matvec_rows(self._h, _p(u), _p(rows, C.c_int64), rows.size, _p(out))
        return out[:, 0].copy(), out[:, 1].copy()

    def dense(self) -> np.ndarray:
        """Assemble A column by column from unit vectors (small meshes only)."""
        n = 2 * self.nv
        A = np.zeros((n, n))
        e = np.zeros(n)
        for k in range(n):
            e[:] = 0.0
            e[k] = 1.0
            A[:, k] = self.matvec(e)
        return A

    def reaction_potential(self, u, points) -> np.ndarray:
        u = _f64(u)
        pts = _f64(points).reshape(-1, 3)
        out = np.zeros(pts.shape[0])
        _lib.or_reaction_potential(self._h, _p(u), _p(pts), pts.shape[0], _p(out))
        return out

    def reaction_field(self, u, points) -> np.ndarray:
        """-grad phi_reac at the points, [n, 3] (the gradient of reaction_potential)."""
        u = _f64(u)
        pts = _f64(points).reshape(-1, 3)
        out = np.zeros((pts.shape[0], 3))
        _lib.or_reaction_field(self._h, _p(u), _p(pts), pts.shape[0], _p(out))
        return out

    def reaction_forces(self, u) -> np.ndarray:
        """Reaction-field force on each charge, 4 pi C q_k (-grad phi_reac)(x_k) in kcal/(mol A),
        [n_c, 3]: the force of the polarised dielectric on the charge with the surface held fixed
        (the energy's units, 4 pi C with C = 332.0716, times q and the field)."""
        q = self.charges[:, 3:4]
        return 4.0 * np.pi * 332.0716 * q * self.reaction_field(u, self.charges[:, :3])

    def energy(self, u) -> float:
        """E_sol in kcal/mol from the solution u = [phi; dphi/dnu]."""
        return float(_lib.or_energy(self._h, _p(_f64(u))))

    def gmres(self, tol: float = 1e-6, max_it: int = 200, restart: int = 50, b=None, scaled: bool = True):
        """Returns (u, iterations, converged, residual history). scaled: GMRES on the unknowns
        scaled by the inverse diagonal coefficients (1/2)(1 + eps), (1/2)(1 + 1/eps) of the two
        row blocks (right preconditioning; the residual test is that of A u = b)."""
        if b is None:
            b = self.rhs()
        b = _f64(b)
        x = np.zeros(2 * self.nv)
        hist = np.zeros(max_it + 1)
        conv = C.c_int(0)
        it = _lib.or_gmres(self._h, _p(b), float(tol), int(max_it), int(restart), int(bool(scaled)), _p(x),
                           _p(hist), C.byref(conv))
        return x, int(it), bool(conv.value), hist[: it + 1].copy()


class LobiProblem(Problem):
    """The low-order LOBI-PB scheme (Sec. 2.4) on the same inputs: flat triangles, centroid
    collocation, self triangle dropped; 2 N_f unknowns (phi then dphi/dnu at centroids)."""

    def geometry(self):
        x, n, A = np.zeros((self.nf, 3)), np.zeros((self.nf, 3)), np.zeros(self.nf)
        _lib.or_lobi_geometry(self._h, _p(x), _p(n), _p(A))
        return x, n, A

    def rhs(self) -> np.ndarray:
        b = np.zeros(2 * self.nf)
        _lib.or_lobi_rhs(self._h, _p(b))
        return b

    def matvec(self, u) -> np.ndarray:
        u = _f64(u)
        assert u.shape == (2 * self.nf,)
        out = np.zeros(2 * self.nf)
        _lib.or_lobi_matvec(self._h, _p(u), _p(out))
        return out

    def matvec_rows(self, u, rows):
        u = _f64(u)
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.zeros((rows.size, 2))
        _lib.or_lobi_matvec_rows(self._h, _p(u), _p(rows, C.c_int64), rows.size, _p(out))
        return out[:, 0].copy(), out[:, 1].copy()

    def dense(self) -> np.ndarray:
        n = 2 * self.nf
        A = np.zeros((n, n))
        e = np.zeros(n)
        for k in range(n):
            e[:] = 0.0
            e[k] = 1.0
            A[:, k] = self.matvec(e)
        return A

    def energy(self, u) -> float:
        return float(_lib.or_lobi_energy(self._h, _p(_f64(u))))

    def gmres(self, tol: float = 1e-6, max_it: int = 200, restart: int = 50, b=None, scaled: bool = True):
        if b is None:
            b = self.rhs()
        b = _f64(b)
        x = np.zeros(2 * self.nf)
        hist = np.zeros(max_it + 1)
        conv = C.c_int(0)
        it = _lib.or_lobi_gmres(self._h, _p(b), float(tol), int(max_it), int(restart), int(bool(scaled)), _p(x),
                                _p(hist), C.byref(conv))
        return x, int(it), bool(conv.value), hist[: it + 1].copy()


def solve_dense(prob: Problem, b=None) -> np.ndarray:
    """Dense assembly + LU (numpy) for small meshes."""
    if b is None:
        b = prob.rhs()
    return np.linalg.solve(prob.dense(), b)


KCAL_PER_MOL_E = 4.0 * np.pi * 332.0716  # G-unit potential -> kcal/(mol e)
