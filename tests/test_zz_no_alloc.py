"""hobi_reaction_potential_noalloc: the reaction potential for callers that must not allocate
device memory once they are running (a host whose device memory belongs to another allocator, a
service with a fixed memory footprint, a latency-bound loop that cannot pay for cudaMalloc).

It must return what hobi_reaction_potential returns for the same handle and points (up to
summation order), and what the oracle computes from the handle's solution, on consecutive calls
that reuse the shared scratch array, with host pointers and with device pointers. This file is
collected last so that a run stopping at its first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1301_5914_gb300 import hobi, synth

pytestmark = pytest.mark.gpu

A, EPS1, EPS2, KAPPA = 10.0, 1.0, 80.0, 0.1257


def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _noalloc(solver, pts, device_mode):
    """Call the entry point through the C ABI with host pointers (numpy) or device pointers
    (CUDA torch tensors, the handle in device-pointer mode)."""
    if device_mode:
        import torch

        p = torch.as_tensor(np.ascontiguousarray(pts, dtype=np.float64), device="cuda").reshape(-1, 3).contiguous()
        out = torch.full((p.shape[0],), np.nan, dtype=torch.float64, device="cuda")
        rc = hobi._lib.hobi_reaction_potential_noalloc(solver._h, p.data_ptr(), p.shape[0], out.data_ptr())
        torch.cuda.synchronize()
        return rc, out.cpu().numpy()
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.full(pts.shape[0], np.nan)
    rc = hobi._lib.hobi_reaction_potential_noalloc(solver._h, pts.ctypes.data, pts.shape[0], out.ctypes.data)
    return rc, out


def _np(a):
    return a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)


@pytest.mark.parametrize("device_mode", [False, True], ids=["host_pointers", "device_pointers"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_noalloc_matches_reaction_potential_and_oracle_twice(prec, tol, device_mode):
    _gpu()
    import torch

    V, F, N = synth.icosphere(4, A)
    Q = synth.ball_charges(10, 8.0, 2)
    args = (V, F, N, Q)
    if device_mode:
        args = tuple(torch.as_tensor(a, device="cuda") for a in (V, F.astype(np.int32), N, Q))
    s = hobi.Solver(*args, EPS1, EPS2, KAPPA, precision=prec)
    assert s.device_mode == device_mode
    s.solve(1e-6)
    u = _np(s.solution())
    orc = oracle.Problem(V, F, N, Q, EPS1, EPS2, KAPPA)
    for seed, n in ((21, 1000), (22, 37)):  # two calls in a row, the second smaller
        pts = synth.ball_charges(n, 7.5, seed)[:, :3].copy()
        ref = _np(s.reaction_potential(torch.as_tensor(pts, device="cuda") if device_mode else pts))
        rc, got = _noalloc(s, pts, device_mode)
        assert rc == hobi.HOBI_OK, hobi._lib.hobi_last_error()
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
        want = orc.reaction_potential(u, pts)
        assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    rc, got = _noalloc(s, np.zeros((0, 3)), device_mode)
    assert rc == hobi.HOBI_OK and got.size == 0
    s.close()


def test_noalloc_rejects_oversized_request():
    _gpu()
    V, F, N = synth.icosphere(2, 2.0)
    s = hobi.Solver(V, F, N, synth.point_charge(0, 0, 0, 1.0), 1.0, 80.0, 0.0, precision="fp64")
    s.solve(1e-6)
    rc, _ = _noalloc(s, np.zeros((4097, 3)), False)
    assert rc == hobi.HOBI_ERR_ARG
    assert b"4096" in hobi._lib.hobi_last_error()
    s.close()


def test_noalloc_launch_is_profiled():
    _gpu()
    V, F, N = synth.icosphere(3, A)
    s = hobi.Solver(V, F, N, synth.ball_charges(4, 8.0, 3), EPS1, EPS2, KAPPA, precision="fp32")
    s.solve(1e-6)
    s.profile_enable(True)
    s.profile_read()
    rc, _ = _noalloc(s, synth.ball_charges(100, 7.5, 5)[:, :3], False)
    assert rc == hobi.HOBI_OK
    prof = s.profile_read()
    assert prof["launches"] == 1 and prof["pairs"] == 100 * s.n_nodes and prof["farfield_ms"] > 0.0
    s.close()
