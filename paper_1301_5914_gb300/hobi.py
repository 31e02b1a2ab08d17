"""Thin Python binding of libhobi (include/hobi.h): argument marshalling only.

Every step of the solver runs in the CUDA library. Inputs may be numpy arrays
(host pointers: the library copies them to and from the GPU) or CUDA torch
tensors (device pointers, work ordered on torch's current stream). PyTorch is
used only for device memory and streams.

If ``_build/libhobi.so`` is missing this module raises on first use: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libhobi.so")

HOBI_OK = 0
HOBI_ERR_ARG = -1
HOBI_ERR_MESH = -2
HOBI_ERR_CUDA = -3
HOBI_ERR_NOMEM = -4
HOBI_ERR_NOT_CONVERGED = -5
HOBI_ERR_BREAKDOWN = -6
HOBI_ERR_STATE = -7
HOBI_FP64 = 0
HOBI_FP32_BULK = 1
HOBI_SCHEME_HOBI = 0
HOBI_SCHEME_LOBI = 1
KCAL_PER_MOL_E = 4.0 * np.pi * 332.0716

EXPORTS = [
    "hobi_default_options", "hobi_setup", "hobi_set_precision", "hobi_sizes", "hobi_matvec", "hobi_rhs",
    "hobi_solve", "hobi_solve_from", "hobi_solve_refined", "hobi_set_solution", "hobi_get_solution", "hobi_reaction_potential",
    "hobi_reaction_potential_noalloc", "hobi_reaction_field", "hobi_reaction_forces", "hobi_reaction_forces_batch",
    "hobi_energy",
    "hobi_get_nodes", "hobi_get_correction", "hobi_profile_enable", "hobi_profile_read", "hobi_kernel_launches", "hobi_plan_info",
    "hobi_fast_info", "hobi_fast_plan_stats", "hobi_fp64_pair_functions", "hobi_check_tile_wait_timeout",
    "hobi_destroy", "hobi_last_error", "hobi_setup_batch", "hobi_batch_sizes", "hobi_batch_set_precision",
    "hobi_matvec_batch", "hobi_solve_batch", "hobi_energy_batch", "hobi_batch_kernel_launches", "hobi_destroy_batch",
    "hobi_batch_profile_enable", "hobi_batch_profile_read",
]


class HobiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hobi error {code}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("mem_device", C.c_int32), ("stream", C.c_void_p),
                ("restart", C.c_int32), ("use_graph", C.c_int32), ("device", C.c_int32), ("scheme", C.c_int32),
                ("autotune", C.c_int32), ("ff_shape", C.c_int32), ("fast_degree", C.c_int32),
                ("fast_theta", C.c_double), ("gmres_scaling", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("rel_residual", C.c_double),
                ("solve_ms", C.c_double), ("farfield_pairs", C.c_double),
                ("resid_history", C.POINTER(C.c_double)), ("resid_capacity", C.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libhobi.so and declare its signatures (fails loudly if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libhobi.so not found at {path}; build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    lib = C.CDLL(path)
    vp, dp, i64 = C.c_void_p, C.c_void_p, C.c_int64
    lib.hobi_default_options.argtypes = [C.POINTER(Options)]
    lib.hobi_default_options.restype = None
    lib.hobi_setup.argtypes = [dp, i64, dp, i64, dp, dp, i64, C.c_double, C.c_double, C.c_double,
                               C.POINTER(Options), C.POINTER(C.c_void_p)]
    lib.hobi_set_precision.argtypes = [vp, C.c_int32]
    lib.hobi_sizes.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64)]
    lib.hobi_matvec.argtypes = [vp, dp, dp]
    lib.hobi_rhs.argtypes = [vp, dp]
    lib.hobi_solve.argtypes = [vp, C.c_double, C.c_int32, dp, dp, C.POINTER(SolveInfo)]
    lib.hobi_solve_from.argtypes = [vp, dp, C.c_double, C.c_int32, dp, dp, C.POINTER(SolveInfo)]
    lib.hobi_solve_refined.argtypes = [vp, C.c_double, C.c_int32, C.c_int32, dp, dp, C.POINTER(SolveInfo)]
    lib.hobi_set_solution.argtypes = [vp, dp]
    lib.hobi_get_solution.argtypes = [vp, dp]
    lib.hobi_reaction_potential.argtypes = [vp, dp, i64, dp]
    lib.hobi_reaction_field.argtypes = [vp, dp, i64, dp]
    lib.hobi_reaction_forces.argtypes = [vp, dp]
    lib.hobi_reaction_forces_batch.argtypes = [vp, dp]
    lib.hobi_reaction_potential_noalloc.argtypes = [vp, dp, i64, dp]
    lib.hobi_energy.argtypes = [vp, C.POINTER(C.c_double)]
    lib.hobi_get_nodes.argtypes = [vp, dp, dp, dp]
    lib.hobi_get_correction.argtypes = [vp, C.POINTER(i64), dp, dp, dp]
    lib.hobi_profile_enable.argtypes = [vp, C.c_int32]
    lib.hobi_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(i64), C.POINTER(C.c_double)]
    lib.hobi_kernel_launches.argtypes = [vp, C.POINTER(i64)]
    lib.hobi_plan_info.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.hobi_fast_info.argtypes = [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32)]
    lib.hobi_fast_plan_stats.argtypes = [dp, i64, dp, i64, C.c_int32, C.c_double, C.POINTER(i64), C.POINTER(i64),
                                         C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.hobi_fp64_pair_functions.argtypes = [dp, i64, dp, dp]
    lib.hobi_check_tile_wait_timeout.argtypes = [vp, C.POINTER(C.c_double)]
    lib.hobi_destroy.argtypes = [vp]
    lib.hobi_destroy.restype = None
    lib.hobi_setup_batch.argtypes = [C.c_int32, dp, dp, dp, dp, dp, dp, dp, C.c_double, C.c_double, C.c_double,
                                     C.POINTER(Options), C.POINTER(C.c_void_p)]
    lib.hobi_batch_sizes.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(i64), C.POINTER(i64)]
    lib.hobi_batch_set_precision.argtypes = [vp, C.c_int32]
    lib.hobi_matvec_batch.argtypes = [vp, dp, dp]
    lib.hobi_solve_batch.argtypes = [vp, C.c_double, C.c_int32, dp, dp, dp, dp, C.POINTER(SolveInfo)]
    lib.hobi_energy_batch.argtypes = [vp, dp]
    lib.hobi_batch_kernel_launches.argtypes = [vp, C.POINTER(i64)]
    lib.hobi_batch_profile_enable.argtypes = [vp, C.c_int32]
    lib.hobi_batch_profile_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(i64), C.POINTER(C.c_double)]
    lib.hobi_destroy_batch.argtypes = [vp]
    lib.hobi_destroy_batch.restype = None
    lib.hobi_last_error.argtypes = []
    lib.hobi_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("hobi_default_options", "hobi_destroy", "hobi_last_error", "hobi_destroy_batch"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(code: int):
    if code != HOBI_OK:
        raise HobiError(code, _lib.hobi_last_error().decode())


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _is_cuda_tensor(x) -> bool:
    return _is_torch(x) and x.is_cuda


_PRECISIONS = {"fp32": HOBI_FP32_BULK, "fp64": HOBI_FP64}
_SCHEMES = {"hobi": HOBI_SCHEME_HOBI, "lobi": HOBI_SCHEME_LOBI}


def _precision(precision: str) -> int:
    if precision not in _PRECISIONS:
        raise ValueError(f"precision must be 'fp32' or 'fp64', not {precision!r}")
    return _PRECISIONS[precision]


def _scheme(scheme: str) -> int:
    if scheme not in _SCHEMES:
        raise ValueError(f"scheme must be 'hobi' or 'lobi', not {scheme!r}")
    return _SCHEMES[scheme]


def _check_mesh(V, F, N, Q=None):
    """Shapes the C ABI reads through its plain pointers: V, N [n_v, 3], F [n_f, 3], Q [n_c, 4]."""
    if len(V.shape) != 2 or V.shape[1] != 3:
        raise ValueError(f"vertices must have shape (n_v, 3), not {tuple(V.shape)}")
    if tuple(N.shape) != tuple(V.shape):
        raise ValueError(f"vertex normals must have the shape of the vertices {tuple(V.shape)}, not {tuple(N.shape)}")
    if len(F.shape) != 2 or F.shape[1] != 3:
        raise ValueError(f"faces must have shape (n_f, 3), not {tuple(F.shape)}")
    if Q is not None and (len(Q.shape) != 2 or Q.shape[1] != 4):
        raise ValueError(f"charges must have shape (n_c, 4), not {tuple(Q.shape)}")


def fast_plan_stats(nodes, targets, degree: int, theta: float):
    """Treecode plan statistics for FP64 source nodes and targets, built on the host (no GPU)."""
    lib = load_library()
    y = np.ascontiguousarray(nodes, dtype=np.float64).reshape(-1, 3)
    x = np.ascontiguousarray(targets, dtype=np.float64).reshape(-1, 3)
    d, a = C.c_int64(), C.c_int64()
    b, p = C.c_int32(), C.c_int32()
    _check(lib.hobi_fast_plan_stats(y.ctypes.data, y.shape[0], x.ctypes.data, x.shape[0], int(degree), float(theta),
                                    C.byref(d), C.byref(a), C.byref(b), C.byref(p)))
    return {"direct_pairs": d.value, "approx_pairs": a.value, "batches": b.value, "proxy_clusters": p.value}


def fp64_pair_functions(x):
    """The FP64 far field's own 1/sqrt(x) and exp(-x) at host points x >= 0 (on the current GPU)."""
    lib = load_library()
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    rs, ex = np.empty_like(x), np.empty_like(x)
    _check(lib.hobi_fp64_pair_functions(x.ctypes.data, x.size, rs.ctypes.data, ex.ctypes.data))
    return rs, ex


class Solver:
    """One molecule on one GPU (wraps a hobi_t handle).

    V [n_v,3], F [n_f,3] int32, N [n_v,3], charges [n_c,4]: all numpy arrays
    (host mode) or all CUDA torch tensors (device mode). scheme "hobi" (the paper's method) or
    "lobi" (its low-order comparison scheme: unknowns at the n_f face centroids). fast_degree > 0
    replaces the FP32 far field by a treecode of that interpolation degree with admissibility
    parameter fast_theta (hobi_options.fast_degree / fast_theta). gmres_scaling (default True) runs
    GMRES on the unknowns scaled by the inverse diagonal coefficients of the two row blocks;
    False runs it on A u = b as it stands (hobi_options.gmres_scaling).
    """

    def __init__(self, V, F, N, charges, eps1: float, eps2: float, kappa: float, precision: str = "fp32",
                 restart: int = 50, use_graph: bool = True, device: int | None = None, stream=None,
                 scheme: str = "hobi", autotune: bool = True, ff_shape: int = -1, fast_degree: int = 0,
                 fast_theta: float = 0.7, gmres_scaling: bool = True):
        lib = load_library()
        self._lib = lib
        self.device_mode = _is_cuda_tensor(V)
        opt = Options()
        lib.hobi_default_options(C.byref(opt))
        opt.precision = _precision(precision)
        opt.restart = int(restart)
        opt.use_graph = 1 if use_graph else 0
        opt.scheme = _scheme(scheme)
        opt.autotune = 1 if autotune else 0
        opt.ff_shape = int(ff_shape)
        opt.fast_degree = int(fast_degree)
        opt.fast_theta = float(fast_theta)
        opt.gmres_scaling = 1 if gmres_scaling else 0
        if self.device_mode:
            import torch

            dev = V.device.index if device is None else device
            opt.device = int(dev if dev is not None else torch.cuda.current_device())
            opt.mem_device = 1
            s = stream if stream is not None else torch.cuda.current_stream(opt.device)
            opt.stream = C.c_void_p(s.cuda_stream)
            self._keep = [t.contiguous() for t in (V, F, N, charges)]
            Vt, Ft, Nt, Qt = self._keep
            if not (Vt.dtype == Nt.dtype == Qt.dtype == torch.float64 and Ft.dtype == torch.int32):
                raise TypeError("device inputs must be float64 (V, N, charges) and int32 (F) CUDA tensors")
            if not all(_is_cuda_tensor(t) and t.device == Vt.device for t in (Ft, Nt, Qt) if t.numel()):
                raise ValueError("device inputs must all be CUDA tensors on one device")
            _check_mesh(Vt, Ft, Nt, Qt.reshape(-1, 4))
            ptrs = [Vt.data_ptr(), Ft.data_ptr(), Nt.data_ptr(), Qt.data_ptr() if Qt.numel() else None]
            nv, nf, nc = Vt.shape[0], Ft.shape[0], Qt.reshape(-1, 4).shape[0]
        else:
            opt.device = -1 if device is None else int(device)
            opt.mem_device = 0
            if _is_torch(V):  # host torch tensors (e.g. pinned buffers): pass their host pointers
                import torch

                self._keep = [t.contiguous() for t in (V, F, N, charges)]
                Vt, Ft, Nt, Qt = self._keep
                if not (Vt.dtype == Nt.dtype == Qt.dtype == torch.float64 and Ft.dtype == torch.int32):
                    raise TypeError("host tensor inputs must be float64 (V, N, charges) and int32 (F)")
                _check_mesh(Vt, Ft, Nt, Qt.reshape(-1, 4))
                ptrs = [t.data_ptr() if t.numel() else None for t in self._keep]
                nv, nf, nc = self._keep[0].shape[0], self._keep[1].shape[0], self._keep[3].reshape(-1, 4).shape[0]
            else:
                self._keep = [np.ascontiguousarray(V, dtype=np.float64), np.ascontiguousarray(F, dtype=np.int32),
                              np.ascontiguousarray(N, dtype=np.float64),
                              np.ascontiguousarray(charges, dtype=np.float64).reshape(-1, 4)]
                Va, Fa, Na, Qa = self._keep
                _check_mesh(Va, Fa, Na, Qa)
                ptrs = [Va.ctypes.data, Fa.ctypes.data, Na.ctypes.data, Qa.ctypes.data if Qa.size else None]
                nv, nf, nc = Va.shape[0], Fa.shape[0], Qa.shape[0]
        h = C.c_void_p()
        _check(lib.hobi_setup(ptrs[0], nv, ptrs[1], nf, ptrs[2], ptrs[3], nc, float(eps1), float(eps2),
                              float(kappa), C.byref(opt), C.byref(h)))
        self._h = h
        self.nv, self.nf, self.nc = int(nv), int(nf), int(nc)
        n_nodes, npts = C.c_int64(), C.c_int64()
        _check(lib.hobi_sizes(h, None, None, None, C.byref(n_nodes), C.byref(npts)))
        self.n_nodes, self.npts = int(n_nodes.value), int(npts.value)  # npts: collocation points
        self.scheme = scheme
        self.eps1, self.eps2, self.kappa = float(eps1), float(eps2), float(kappa)

    # ------------------------------------------------------------ helpers
    def _out(self, n, like=None):
        if self.device_mode:
            import torch

            return torch.empty(n, dtype=torch.float64, device=self._keep[0].device)
        return np.empty(n, dtype=np.float64)

    def _ptr(self, a):
        if self.device_mode:
            return a.data_ptr()
        return a.ctypes.data

    def _in(self, a, n):
        if self.device_mode:
            import torch

            t = a if _is_torch(a) else torch.as_tensor(np.asarray(a))
            t = t.to(device=self._keep[0].device, dtype=torch.float64).contiguous().reshape(-1)
            if t.numel() != n:
                raise ValueError(f"expected {n} values, got {t.numel()}")
            return t
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        if a.size != n:
            raise ValueError(f"expected {n} values, got {a.size}")
        return a

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hobi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ API
    def set_precision(self, precision: str):
        _check(self._lib.hobi_set_precision(self._h, _precision(precision)))

    def matvec(self, u):
        u = self._in(u, 2 * self.npts)
        out = self._out(2 * self.npts)
        _check(self._lib.hobi_matvec(self._h, self._ptr(u), self._ptr(out)))
        return out

    def rhs(self):
        out = self._out(2 * self.npts)
        _check(self._lib.hobi_rhs(self._h, self._ptr(out)))
        return out

    def solve(self, tol: float = 1e-6, max_it: int = 200, history: int = 0, raise_on_fail: bool = True,
              u0=None, resume: bool = False):
        """Returns (phi, dphi, info dict). info['status'] holds the return code. With u0 (an initial
        guess [phi; dphi]) or resume=True (start from the handle's current solution) GMRES is warm
        started (hobi_solve_from)."""
        phi = self._out(self.npts)
        dphi = self._out(self.npts)
        info = SolveInfo()
        hist = None
        if history > 0:
            hist = (C.c_double * history)()
            info.resid_history = C.cast(hist, C.POINTER(C.c_double))
            info.resid_capacity = history
        if u0 is not None or resume:
            u0p = None
            if u0 is not None:
                self._u0_keep = self._in(u0, 2 * self.npts)  # alive until the call returns
                u0p = self._ptr(self._u0_keep)
            code = self._lib.hobi_solve_from(self._h, u0p, float(tol), int(max_it), self._ptr(phi), self._ptr(dphi),
                                             C.byref(info))
        else:
            code = self._lib.hobi_solve(self._h, float(tol), int(max_it), self._ptr(phi), self._ptr(dphi),
                                        C.byref(info))
        if raise_on_fail and code not in (HOBI_OK,):
            _check(code)
        d = {"status": code, "iterations": info.iterations, "converged": bool(info.converged),
             "rel_residual": info.rel_residual, "solve_ms": info.solve_ms, "farfield_pairs": info.farfield_pairs}
        if hist is not None:
            d["history"] = np.array(hist[: min(history, info.iterations + 1)])
        return phi, dphi, d

    def solve_refined(self, tol: float = 1e-10, max_refine: int = 8, max_it: int = 200, history: int = 0,
                      raise_on_fail: bool = True):
        """Mixed-precision solve (hobi_solve_refined): FP32-bulk GMRES corrections, FP64 residuals,
        until ||b - A u|| / ||b|| <= tol on the FP64 operator. Returns (phi, dphi, info)."""
        phi = self._out(self.npts)
        dphi = self._out(self.npts)
        info = SolveInfo()
        hist = None
        if history > 0:
            hist = (C.c_double * history)()
            info.resid_history = C.cast(hist, C.POINTER(C.c_double))
            info.resid_capacity = history
        code = self._lib.hobi_solve_refined(self._h, float(tol), int(max_refine), int(max_it), self._ptr(phi),
                                            self._ptr(dphi), C.byref(info))
        if raise_on_fail and code != HOBI_OK:
            _check(code)
        d = {"status": code, "iterations": info.iterations, "converged": bool(info.converged),
             "rel_residual": info.rel_residual, "solve_ms": info.solve_ms, "farfield_pairs": info.farfield_pairs}
        if hist is not None:
            d["history"] = np.array(hist[: min(history, max_refine + 1)])
        return phi, dphi, d

    def set_solution(self, u):
        u = self._in(u, 2 * self.npts)
        _check(self._lib.hobi_set_solution(self._h, self._ptr(u)))

    def solution(self):
        out = self._out(2 * self.npts)
        _check(self._lib.hobi_get_solution(self._h, self._ptr(out)))
        return out

    def reaction_potential(self, points):
        n = int(np.prod(points.shape)) // 3
        p = self._in(points, 3 * n)
        out = self._out(n)
        _check(self._lib.hobi_reaction_potential(self._h, self._ptr(p), n, self._ptr(out)))
        return out

    def reaction_field(self, points):
        """-grad phi_reac at the points, [n, 3] (host array or CUDA tensor, like the inputs)."""
        n = int(np.prod(points.shape)) // 3
        p = self._in(points, 3 * n)
        out = self._out(3 * n)
        _check(self._lib.hobi_reaction_field(self._h, self._ptr(p), n, self._ptr(out)))
        return out.reshape(n, 3)

    def reaction_forces(self):
        """Reaction-field force on every charge, kcal/(mol A), [n_c, 3]."""
        out = self._out(3 * self.nc)
        _check(self._lib.hobi_reaction_forces(self._h, self._ptr(out)))
        return out.reshape(self.nc, 3)

    def energy(self) -> float:
        e = C.c_double()
        _check(self._lib.hobi_energy(self._h, C.byref(e)))
        return float(e.value)

    def nodes(self):
        """(y, nu, W): [n_f, 4, 3] each for HOBI; [n_f, 3] for LOBI (centroid, normal, (area, 0, 0))."""
        outs = [self._out(3 * self.n_nodes) for _ in range(3)]
        _check(self._lib.hobi_get_nodes(self._h, *[self._ptr(o) for o in outs]))
        shape = (self.nf, 4, 3) if self.scheme != "lobi" else (self.nf, 3)
        return tuple(o.reshape(shape) for o in outs)

    def correction(self):
        """(vertex[e], face[e], coeff[e,3,4]) for every (vertex, incident face) entry."""
        n = C.c_int64()
        _check(self._lib.hobi_get_correction(self._h, C.byref(n), None, None, None))
        ne = n.value
        v = np.empty(ne, dtype=np.int32)
        f = np.empty(ne, dtype=np.int32)
        c = np.empty((ne, 3, 4), dtype=np.float64)
        _check(self._lib.hobi_get_correction(self._h, C.byref(n), v.ctypes.data, f.ctypes.data, c.ctypes.data))
        return v, f, c

    def kernel_launches(self) -> int:
        n = C.c_int64()
        _check(self._lib.hobi_kernel_launches(self._h, C.byref(n)))
        return int(n.value)

    def plan_info(self):
        """FP32 far-field plan: {'shape', 'chunks', 'tuned'}."""
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        _check(self._lib.hobi_plan_info(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return {"shape": a.value, "chunks": b.value, "tuned": bool(c.value)}

    def fast_info(self):
        """Treecode statistics per matvec (all zero when fast summation is off)."""
        d, a = C.c_int64(), C.c_int64()
        b, p, t = C.c_int32(), C.c_int32(), C.c_int32()
        _check(self._lib.hobi_fast_info(self._h, C.byref(d), C.byref(a), C.byref(b), C.byref(p), C.byref(t)))
        return {"direct_pairs": d.value, "approx_pairs": a.value, "batches": b.value, "proxy_clusters": p.value,
                "tasks": t.value}

    def check_tile_wait_timeout(self):
        """Run the far-field tile pipeline's bounded wait on a barrier nothing completes: returns
        (status code, message, kernel milliseconds); the expected status is HOBI_ERR_CUDA."""
        ms = C.c_double()
        code = self._lib.hobi_check_tile_wait_timeout(self._h, C.byref(ms))
        return code, self._lib.hobi_last_error().decode() if code != HOBI_OK else "", ms.value

    def profile_enable(self, on: bool = True):
        _check(self._lib.hobi_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        ms, pairs = C.c_double(), C.c_double()
        n = C.c_int64()
        _check(self._lib.hobi_profile_read(self._h, C.byref(ms), C.byref(n), C.byref(pairs)))
        return {"farfield_ms": ms.value, "launches": n.value, "pairs": pairs.value}


class BatchSolver:
    """Many molecules with the same eps1, eps2, kappa, solved together (wraps hobi_batch_t).

    molecules: list of (V, F, N, charges) numpy arrays (host mode). With device=True the
    concatenated inputs are first placed in CUDA torch tensors (device-pointer mode).
    fast_degree > 0: molecules with at least 4096 collocation points whose treecode plan pays off
    use fast summation for the FP32 far field (hobi_options.fast_degree / fast_theta).
    gmres_scaling as for Solver.
    """

    def __init__(self, molecules, eps1: float, eps2: float, kappa: float, precision: str = "fp32",
                 restart: int = 50, use_graph: bool = True, device_mode: bool = False, stream=None,
                 device_arrays=None, fast_degree: int = 0, fast_theta: float = 0.7, gmres_scaling: bool = True):
        lib = load_library()
        self._lib = lib
        if len(molecules) == 0:
            raise ValueError("a batch needs at least one molecule")
        for m in molecules:
            _check_mesh(np.asarray(m[0]), np.asarray(m[1]), np.asarray(m[2]), np.asarray(m[3]).reshape(-1, 4))
        V = np.ascontiguousarray(np.concatenate([m[0] for m in molecules]), dtype=np.float64)
        F = np.ascontiguousarray(np.concatenate([m[1] for m in molecules]), dtype=np.int32)
        N = np.ascontiguousarray(np.concatenate([m[2] for m in molecules]), dtype=np.float64)
        Q = np.ascontiguousarray(np.concatenate([np.asarray(m[3]).reshape(-1, 4) for m in molecules]),
                                 dtype=np.float64)
        self.vert_off = np.concatenate([[0], np.cumsum([m[0].shape[0] for m in molecules])]).astype(np.int64)
        self.face_off = np.concatenate([[0], np.cumsum([m[1].shape[0] for m in molecules])]).astype(np.int64)
        self.charge_off = np.concatenate([[0], np.cumsum([np.asarray(m[3]).reshape(-1, 4).shape[0]
                                                          for m in molecules])]).astype(np.int64)
        self.n_mol = len(molecules)
        self.nv_total = int(self.vert_off[-1])
        self.device_mode = device_mode or device_arrays is not None
        opt = Options()
        lib.hobi_default_options(C.byref(opt))
        opt.precision = _precision(precision)
        opt.restart = int(restart)
        opt.use_graph = 1 if use_graph else 0
        opt.fast_degree = int(fast_degree)
        opt.fast_theta = float(fast_theta)
        opt.gmres_scaling = 1 if gmres_scaling else 0
        if self.device_mode:
            import torch

            dev = torch.device("cuda", torch.cuda.current_device())
            opt.device = dev.index
            opt.mem_device = 1
            s = stream if stream is not None else torch.cuda.current_stream(dev)
            opt.stream = C.c_void_p(s.cuda_stream)
            if device_arrays is not None:  # the concatenated inputs, already resident on the GPU
                self._keep = [t.contiguous() for t in device_arrays]
                for t, a in zip(self._keep, (V, F, N, Q)):
                    if tuple(t.shape) != a.shape or t.element_size() != a.itemsize:
                        raise ValueError("device_arrays must be the concatenated V, F, N, charges of the batch")
            else:
                self._keep = [torch.as_tensor(a, device=dev) for a in (V, F, N, Q)]
            ptrs = [t.data_ptr() for t in self._keep]
        else:
            opt.device = -1
            self._keep = [V, F, N, Q]
            ptrs = [a.ctypes.data for a in self._keep]
        h = C.c_void_p()
        _check(lib.hobi_setup_batch(self.n_mol, ptrs[0], self.vert_off.ctypes.data, ptrs[1], self.face_off.ctypes.data,
                                    ptrs[2], ptrs[3] if Q.size else None, self.charge_off.ctypes.data, float(eps1),
                                    float(eps2), float(kappa), C.byref(opt), C.byref(h)))
        self._h = h

    def _out(self, n):
        if self.device_mode:
            import torch

            return torch.empty(n, dtype=torch.float64, device=self._keep[0].device)
        return np.empty(n, dtype=np.float64)

    def _ptr(self, a):
        return a.data_ptr() if self.device_mode else a.ctypes.data

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hobi_destroy_batch(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision: str):
        _check(self._lib.hobi_batch_set_precision(self._h, _precision(precision)))

    def split(self, a):
        """Split a concatenated per-vertex array into per-molecule arrays."""
        return [a[self.vert_off[i]:self.vert_off[i + 1]] for i in range(self.n_mol)]

    def matvec(self, u):
        """u: concatenation of the molecules' [phi; dphi] blocks (host mode: numpy)."""
        n = 2 * self.nv_total
        if self.device_mode:
            import torch

            u = torch.as_tensor(u, device=self._keep[0].device, dtype=torch.float64).contiguous()
        else:
            u = np.ascontiguousarray(u, dtype=np.float64)
        out = self._out(n)
        _check(self._lib.hobi_matvec_batch(self._h, self._ptr(u), self._ptr(out)))
        return out

    def solve(self, tol: float = 1e-6, max_it: int = 200, raise_on_fail: bool = True):
        """Returns (phi per molecule, dphi per molecule, info); info has per-molecule iterations/status."""
        phi = self._out(self.nv_total)
        dphi = self._out(self.nv_total)
        its = np.zeros(self.n_mol, dtype=np.int32)
        st = np.zeros(self.n_mol, dtype=np.int32)
        info = SolveInfo()
        code = self._lib.hobi_solve_batch(self._h, float(tol), int(max_it), self._ptr(phi), self._ptr(dphi),
                                          its.ctypes.data, st.ctypes.data, C.byref(info))
        if raise_on_fail and code != HOBI_OK:
            _check(code)
        d = {"status": code, "steps": info.iterations, "converged": bool(info.converged),
             "rel_residual": info.rel_residual, "solve_ms": info.solve_ms, "farfield_pairs": info.farfield_pairs,
             "iterations": its, "mol_status": st}
        return self.split(phi), self.split(dphi), d

    def energy(self) -> np.ndarray:
        e = np.zeros(self.n_mol, dtype=np.float64)
        _check(self._lib.hobi_energy_batch(self._h, e.ctypes.data))
        return e

    def reaction_forces(self):
        """Reaction-field forces on the charges, one [n_c, 3] array per molecule (kcal/(mol A))."""
        f = np.zeros((int(self.charge_off[-1]), 3), dtype=np.float64)
        _check(self._lib.hobi_reaction_forces_batch(self._h, f.ctypes.data))
        return [f[self.charge_off[m]:self.charge_off[m + 1]] for m in range(self.n_mol)]

    def kernel_launches(self) -> int:
        n = C.c_int64()
        _check(self._lib.hobi_batch_kernel_launches(self._h, C.byref(n)))
        return int(n.value)

    def profile_enable(self, on: bool = True):
        _check(self._lib.hobi_batch_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        ms, pairs = C.c_double(), C.c_double()
        n = C.c_int64()
        _check(self._lib.hobi_batch_profile_read(self._h, C.byref(ms), C.byref(n), C.byref(pairs)))
        return {"farfield_ms": ms.value, "launches": n.value, "pairs": pairs.value}
