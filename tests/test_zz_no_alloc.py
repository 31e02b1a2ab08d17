"""hobi_reaction_potential_noalloc: the reaction potential for callers that cannot allocate
device memory at call time (e.g. while a stream is being captured into a CUDA graph).

It must return what hobi_reaction_potential returns for the same handle and points (up to
summation order), on consecutive calls that reuse the shared scratch array. This file is
collected last so that a run stopping at its first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1301_5914_gb300 import hobi, synth

pytestmark = pytest.mark.gpu


def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _noalloc(solver, pts):
    """Call the entry point through the C ABI (host-pointer handle)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    out = np.empty(pts.shape[0], dtype=np.float64)
    rc = hobi._lib.hobi_reaction_potential_noalloc(solver._h, pts.ctypes.data, pts.shape[0], out.ctypes.data)
    return rc, out


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_noalloc_matches_reaction_potential_twice(prec, tol):
    _gpu()
    V, F, N = synth.icosphere(4, 10.0)
    Q = synth.ball_charges(10, 8.0, 2)
    s = hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.1257, precision=prec)
    s.solve(1e-6)
    for seed, n in ((21, 1000), (22, 37)):  # two calls in a row, the second smaller
        pts = synth.ball_charges(n, 7.5, seed)[:, :3]
        ref = s.reaction_potential(pts)
        rc, got = _noalloc(s, pts)
        assert rc == hobi.HOBI_OK, hobi._lib.hobi_last_error()
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    s.close()


def test_noalloc_rejects_oversized_request():
    _gpu()
    V, F, N = synth.icosphere(2, 2.0)
    s = hobi.Solver(V, F, N, synth.point_charge(0, 0, 0, 1.0), 1.0, 80.0, 0.0, precision="fp64")
    s.solve(1e-6)
    pts = np.zeros((4097, 3))
    rc, _ = _noalloc(s, pts)
    assert rc == hobi.HOBI_ERR_ARG
    assert b"4096" in hobi._lib.hobi_last_error()
    s.close()
