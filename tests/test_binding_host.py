"""The Python binding's argument checks, on the host (no GPU): shapes, dtypes and option strings
are validated before any pointer reaches the C ABI; valid inputs reach the library (which, without
a GPU, reports its CUDA error rather than falling back to anything)."""
import numpy as np
import pytest
import torch

from paper_1301_5914_gb300 import hobi, synth


@pytest.fixture(scope="module")
def mesh():
    V, F, N = synth.icosphere(1, 2.0)
    return V, F, N, synth.ball_charges(2, 1.0, 1)


def _reaches_library(fn):
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the call would succeed")
    with pytest.raises(hobi.HobiError) as ei:
        fn()
    assert ei.value.code in (hobi.HOBI_ERR_CUDA, hobi.HOBI_ERR_NOMEM)


def test_valid_inputs_reach_the_library(mesh):
    V, F, N, Q = mesh
    _reaches_library(lambda: hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.1))
    _reaches_library(lambda: hobi.Solver(*(torch.as_tensor(a) for a in (V, F.astype(np.int32), N, Q)), 1.0, 80.0, 0.1))
    _reaches_library(lambda: hobi.Solver(V, F, N, np.zeros((0, 4)), 1.0, 80.0, 0.1, precision="fp64",
                                         scheme="lobi"))
    _reaches_library(lambda: hobi.BatchSolver([(V, F, N, Q), (V, F, N, Q)], 1.0, 80.0, 0.1))


@pytest.mark.parametrize("bad", ["V flat", "N short", "F flat", "Q three columns"])
def test_shapes_checked_before_the_call(mesh, bad):
    V, F, N, Q = mesh
    args = {"V flat": (V.ravel(), F, N, Q), "N short": (V, F, N[:-1], Q), "F flat": (V, F.ravel(), N, Q),
            "Q three columns": (V, F, N, Q[:, :3])}[bad]
    with pytest.raises(ValueError):
        hobi.Solver(*args, 1.0, 80.0, 0.1)
    with pytest.raises(ValueError):
        hobi.BatchSolver([(V, F, N, Q), args], 1.0, 80.0, 0.1)


def test_option_strings_and_dtypes(mesh):
    V, F, N, Q = mesh
    with pytest.raises(ValueError, match="precision"):
        hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.1, precision="fp16")
    with pytest.raises(ValueError, match="scheme"):
        hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.1, scheme="flat")
    with pytest.raises(ValueError, match="precision"):
        hobi.BatchSolver([(V, F, N, Q)], 1.0, 80.0, 0.1, precision="double")
    with pytest.raises(ValueError):
        hobi.BatchSolver([], 1.0, 80.0, 0.1)
    with pytest.raises(TypeError):  # host tensors are passed by pointer: their dtypes must match the ABI
        hobi.Solver(*(torch.as_tensor(a) for a in (V, F.astype(np.int64), N, Q)), 1.0, 80.0, 0.1)
    with pytest.raises(TypeError):
        hobi.Solver(*(torch.as_tensor(a, dtype=torch.float32) if a.dtype.kind == "f" else torch.as_tensor(a)
                      for a in (V, F.astype(np.int32), N, Q)), 1.0, 80.0, 0.1)


class _FakeStream:
    cuda_stream = 0


def test_device_mode_branches_run_up_to_the_library(mesh, monkeypatch):
    """The device-pointer branches of Solver and BatchSolver, exercised on the host by treating
    CPU tensors as device tensors: every check runs, wrong inputs are refused, and valid ones
    reach the library (which, without a GPU, reports a CUDA error)."""
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the real device path is covered by the GPU tests")
    V, F, N, Q = mesh
    monkeypatch.setattr(hobi, "_is_cuda_tensor", lambda x: hobi._is_torch(x))
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    t = [torch.as_tensor(a) for a in (V, F.astype(np.int32), N, Q)]
    _reaches_library(lambda: hobi.Solver(*t, 1.0, 80.0, 0.1, device=0, stream=_FakeStream()))
    with pytest.raises(TypeError):
        hobi.Solver(t[0], t[1].long(), t[2], t[3], 1.0, 80.0, 0.1, device=0, stream=_FakeStream())
    with pytest.raises(ValueError):
        hobi.Solver(t[0], t[1], t[2][:-1], t[3], 1.0, 80.0, 0.1, device=0, stream=_FakeStream())
    mols = [(V, F, N, Q), (V, F, N, Q)]
    cat = [torch.as_tensor(np.concatenate([m[k] for m in mols])) for k in range(4)]
    cat[1] = cat[1].to(torch.int32)
    _reaches_library(lambda: hobi.BatchSolver(mols, 1.0, 80.0, 0.1, device_arrays=cat, stream=_FakeStream()))
    with pytest.raises(ValueError):
        hobi.BatchSolver(mols, 1.0, 80.0, 0.1, device_arrays=[cat[0][:-1], *cat[1:]], stream=_FakeStream())
