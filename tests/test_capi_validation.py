"""Argument and option validation of the C ABI, on the host (no GPU): every invalid input is
refused with HOBI_ERR_ARG and a message before any device work starts."""
import ctypes as C
import math

import numpy as np
import pytest

from paper_1301_5914_gb300 import hobi, synth


@pytest.fixture(scope="module")
def lib():
    return hobi.load_library()


@pytest.fixture(scope="module")
def mesh():
    V, F, N = synth.icosphere(1, 2.0)
    Q = synth.ball_charges(2, 1.0, 1)
    return (np.ascontiguousarray(V), np.ascontiguousarray(F, dtype=np.int32), np.ascontiguousarray(N),
            np.ascontiguousarray(Q))


def _setup(lib, mesh, nv=None, nf=None, nc=None, eps1=1.0, eps2=80.0, kappa=0.1, charges=True, **opts):
    V, F, N, Q = mesh
    o = hobi.Options()
    lib.hobi_default_options(C.byref(o))
    for k, v in opts.items():
        setattr(o, k, v)
    h = C.c_void_p()
    rc = lib.hobi_setup(V.ctypes.data, V.shape[0] if nv is None else nv, F.ctypes.data,
                        F.shape[0] if nf is None else nf, N.ctypes.data, Q.ctypes.data if charges else None,
                        Q.shape[0] if nc is None else nc, eps1, eps2, kappa, C.byref(o), C.byref(h))
    return rc, lib.hobi_last_error().decode(), h.value


@pytest.mark.parametrize("kw,msg", [
    (dict(nv=3), "at least 4 vertices"),
    (dict(nf=2), "at least 4 vertices and 4 faces"),
    (dict(nc=-1), "n_c < 0"),
    (dict(charges=False), "charges is NULL"),
    (dict(nf=(1 << 28) + 1), "problem too large"),
    (dict(eps1=0.0), "eps1 and eps2"),
    (dict(eps2=-80.0), "eps1 and eps2"),
    (dict(eps2=math.nan), "eps1 and eps2"),
    (dict(eps1=math.inf), "eps1 and eps2"),
    (dict(kappa=-0.1), "kappa"),
    (dict(kappa=math.nan), "kappa"),
    (dict(kappa=math.inf), "kappa"),
    (dict(precision=7), "unknown precision"),
    (dict(scheme=5), "unknown scheme"),
    (dict(ff_shape=4), "ff_shape"),
    (dict(ff_shape=-2), "ff_shape"),
    (dict(fast_degree=1), "fast_degree"),
    (dict(fast_degree=11), "fast_degree"),
    (dict(fast_degree=4, fast_theta=0.0), "fast_theta"),
    (dict(fast_degree=4, fast_theta=1.5), "fast_theta"),
    (dict(fast_degree=4, fast_theta=math.nan), "fast_theta"),
    (dict(fast_degree=4, scheme=hobi.HOBI_SCHEME_LOBI), "HOBI scheme only"),
    (dict(restart=201), "restart"),
    (dict(gmres_scaling=2), "gmres_scaling"),
    (dict(gmres_scaling=-1), "gmres_scaling"),
])
def test_setup_rejects_invalid_input(lib, mesh, kw, msg):
    rc, err, h = _setup(lib, mesh, **kw)
    assert rc == hobi.HOBI_ERR_ARG and h is None
    assert msg in err, err


def test_calls_on_a_null_handle(lib):
    for rc in (lib.hobi_set_precision(None, hobi.HOBI_FP64), lib.hobi_rhs(None, None),
               lib.hobi_solve(None, 1e-6, 10, None, None, None),
               lib.hobi_sizes(None, None, None, None, None, None)):
        assert rc == hobi.HOBI_ERR_ARG
    lib.hobi_destroy(None)  # a no-op


def test_fast_plan_stats_validation_and_counts():
    V, F, N = synth.icosphere(3, 5.0)
    y = np.random.default_rng(0).normal(size=(3000, 3)) * 5.0
    for deg, theta in ((1, 0.7), (11, 0.7), (4, 0.0), (4, 1.01)):
        with pytest.raises(hobi.HobiError):
            hobi.fast_plan_stats(y, V, deg, theta)
    with pytest.raises(hobi.HobiError):
        hobi.fast_plan_stats(np.zeros((0, 3)), V, 4, 0.7)
    st = hobi.fast_plan_stats(y, V, 4, 0.7)
    # every (target, node) pair is either summed directly or through a proxy cluster's points
    assert st["batches"] == -(-V.shape[0] // 256)
    assert st["direct_pairs"] + st["approx_pairs"] > 0
    assert st["direct_pairs"] <= V.shape[0] * y.shape[0]
    # theta -> 0: no cluster is admissible and the plan is the direct sum
    st0 = hobi.fast_plan_stats(y, V, 4, 1e-3)
    assert st0["approx_pairs"] == 0 and st0["direct_pairs"] == V.shape[0] * y.shape[0]


def _setup_batch(lib, mesh, n_mol=2, voff=None, foff=None, qoff=None, charges=True, eps1=1.0, eps2=80.0,
                 kappa=0.1, **opts):
    V, F, N, Q = mesh
    Vb, Fb, Nb, Qb = (np.ascontiguousarray(np.concatenate([a, a])) for a in (V, F, N, Q))
    voff = np.array([0, V.shape[0], 2 * V.shape[0]] if voff is None else voff, dtype=np.int64)
    foff = np.array([0, F.shape[0], 2 * F.shape[0]] if foff is None else foff, dtype=np.int64)
    qoff = np.array([0, Q.shape[0], 2 * Q.shape[0]] if qoff is None else qoff, dtype=np.int64)
    o = hobi.Options()
    lib.hobi_default_options(C.byref(o))
    for k, v in opts.items():
        setattr(o, k, v)
    h = C.c_void_p()
    rc = lib.hobi_setup_batch(n_mol, Vb.ctypes.data, voff.ctypes.data, Fb.ctypes.data, foff.ctypes.data,
                              Nb.ctypes.data, Qb.ctypes.data if charges else None, qoff.ctypes.data, eps1, eps2, kappa,
                              C.byref(o), C.byref(h))
    return rc, lib.hobi_last_error().decode(), h.value


@pytest.mark.parametrize("kw,msg", [
    (dict(n_mol=0), "n_mol"),
    (dict(voff=[0, 50, 42]), "non-decreasing"),
    (dict(foff=[1, 80, 160]), "start at 0"),
    (dict(charges=False), "charges is NULL"),
    (dict(eps1=-1.0), "eps1, eps2 > 0"),
    (dict(kappa=math.nan), "kappa >= 0"),
    (dict(precision=3), "unknown precision"),
    (dict(scheme=hobi.HOBI_SCHEME_LOBI), "HOBI scheme only"),
    (dict(fast_degree=12), "fast_degree"),
    (dict(fast_degree=5, fast_theta=2.0), "fast_theta"),
    (dict(restart=500), "restart"),
    (dict(gmres_scaling=3), "gmres_scaling"),
])
def test_setup_batch_rejects_invalid_input(lib, mesh, kw, msg):
    rc, err, h = _setup_batch(lib, mesh, **kw)
    assert rc == hobi.HOBI_ERR_ARG and h is None
    assert msg in err, err
