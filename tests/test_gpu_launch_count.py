"""The library's own count of the kernels it launched (hobi_kernel_launches,
hobi_batch_kernel_launches; the bench line's `gpu_launches` comes from it) against an
independent count: the CUDA kernel activity that torch's profiler (CUPTI) records in the same
process, kernels of captured graphs included."""
import numpy as np
import pytest

from paper_1301_5914_gb300 import hobi, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    # the first profiler session of a process may come back without device activity
    try:
        from torch.profiler import ProfilerActivity, profile

        with profile(activities=[ProfilerActivity.CUDA]):
            (torch.ones(16, device="cuda") + 1).sum().item()
    except Exception:
        pass


def _library_kernels(fn):
    """Kernels of this library recorded by the profiler while fn runs."""
    import torch
    from torch.profiler import ProfilerActivity, profile

    try:
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            fn()
            torch.cuda.synchronize()
    except Exception as e:  # no CUPTI on this install
        pytest.skip(f"torch profiler unavailable: {e}")
    names = [e.name for e in prof.events() if str(e.device_type).endswith("CUDA")]
    if not names:
        pytest.skip("the profiler recorded no CUDA kernels")
    return sum(1 for n in names if "hobi::" in n)


@pytest.mark.parametrize("prec,graph", [("fp32", True), ("fp64", False)])
def test_single_step_launch_count(prec, graph):
    V, F, N = synth.icosphere(3, 4.0)
    Q = synth.ball_charges(5, 3.0, 4)
    box = {}

    def step():
        s = hobi.Solver(V, F, N, Q, 2.0, 80.0, 0.1257, precision=prec, use_graph=graph, autotune=False)
        s.solve(1e-6, 100)
        s.energy()
        box["n"] = s.kernel_launches()
        s.close()

    step()  # first set-up of this size outside the count
    seen = _library_kernels(step)
    assert box["n"] == seen, (box["n"], seen)


def test_batch_step_launch_count():
    mols = []
    for lvl, R, seed in ((1, 1.5, 11), (2, 3.0, 12), (3, 5.0, 13)):
        V, F, N = synth.icosphere(lvl, R)
        mols.append((V, F, N, synth.ball_charges(4, 0.6 * R, seed)))
    box = {}

    def step():
        b = hobi.BatchSolver(mols, 2.0, 80.0, 0.1257, precision="fp32")
        b.solve(1e-6, 100)
        b.energy()
        box["n"] = b.kernel_launches()
        b.close()

    step()
    seen = _library_kernels(step)
    assert box["n"] == seen, (box["n"], seen)
