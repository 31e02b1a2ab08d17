"""The handles' device memory comes from a library-owned stream-ordered pool per device that
keeps freed memory for later handles. Reused memory must not change results: a solve repeated
after handles of other sizes, schemes and precisions have been created and destroyed gives
bit-identical output; and repeated set-up / destroy of one size must not grow the device memory
in use (the pool hands the same memory back)."""
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


def _solve(level, prec="fp32", scheme="hobi"):
    V, F, N = synth.icosphere(level, 10.0)
    Q = synth.ball_charges(10, 8.0, 2)
    s = hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.1257, precision=prec, scheme=scheme)
    phi, dphi, info = s.solve(1e-6, 200)
    E = s.energy()
    s.close()
    return np.concatenate([phi, dphi]), E


def test_results_bit_identical_after_memory_reuse():
    u1, E1 = _solve(4)
    # other handles in between: larger, smaller, FP64, LOBI, a batch
    _solve(5)
    _solve(2, "fp64")
    _solve(3, "fp32", "lobi")
    mols = [synth.icosphere(l, r) + (synth.ball_charges(3, 0.6 * r, 60 + l),) for l, r in ((2, 3.0), (3, 5.0))]
    b = hobi.BatchSolver(mols, 1.0, 80.0, 0.1257, precision="fp32")
    b.solve(1e-6, 200)
    b.close()
    u2, E2 = _solve(4)
    assert np.array_equal(u1, u2) and E1 == E2


def test_repeated_setup_does_not_grow_device_memory():
    import torch

    _solve(5)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(10):
        _solve(5)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # one level-5 handle holds a few tens of MB; ten more set-ups must reuse it
    assert free0 - free1 < 64 * 1024 * 1024, (free0 - free1) / 2**20


def test_growing_point_counts_keep_device_memory_bounded():
    """Reaction potentials at slowly growing point counts: the point buffers grow geometrically,
    so 300 calls from 2,000 to 2,299 points re-allocate a few times, not 300 times."""
    import torch

    V, F, N = synth.icosphere(4, 10.0)
    Q = synth.ball_charges(10, 8.0, 2)
    s = hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.1257, precision="fp32")
    s.solve(1e-6, 200)
    pts = synth.ball_charges(2400, 7.0, 5)[:, :3]
    ref = s.reaction_potential(pts[:2000])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for n in range(2000, 2300):
        out = s.reaction_potential(pts[:n])
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    # the plan's source chunks depend on the point count: equal up to FP32 sum order
    assert np.max(np.abs(out[:2000] - ref)) <= 1e-5 * np.max(np.abs(ref))
    assert free0 - free1 < 32 * 1024 * 1024, (free0 - free1) / 2**20
    s.close()
