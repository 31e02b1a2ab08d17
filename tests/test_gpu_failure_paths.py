"""Failure detection without a GPU fault: the far-field kernels' bounded barrier waits.

Every wait of a far-field tile pipeline on a bulk-copied source tile is bounded; when it gives up,
the kernel sets the handle's error flag and returns, and the calling entry point reports
HOBI_ERR_CUDA. hobi_check_tile_wait_timeout drives that path with a barrier phase that nothing
completes (no copy, no fault): the status and message must be the pipeline-timeout report, the
wait must end after about a second, and the handle must keep working afterwards (same results as
before, the flag cleared).
"""
import numpy as np
import pytest

from paper_1301_5914_gb300 import hobi, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_tile_wait_timeout_is_reported_and_the_handle_stays_usable(prec):
    V, F, N = synth.icosphere(3, 5.0)
    Q = synth.ball_charges(4, 4.0, 8)
    s = hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.1257, precision=prec)
    u = np.random.default_rng(1).normal(size=2 * s.nv)
    before = s.matvec(u)
    code, msg, ms = s.check_tile_wait_timeout()
    assert code == hobi.HOBI_ERR_CUDA, (code, msg)
    assert "timed out" in msg
    # 2^18 polls of mbarrier.try_wait at about 4 us each (measured): about one second
    assert 200.0 <= ms <= 5000.0, ms
    after = s.matvec(u)  # would raise if the flag were still set
    assert np.array_equal(before, after)
    phi, dphi, info = s.solve(1e-6, 100)
    assert info["converged"] and np.isfinite(s.energy())
    # a second check behaves the same (the flag was cleared by the first report)
    code2, _, _ = s.check_tile_wait_timeout()
    assert code2 == hobi.HOBI_ERR_CUDA
    s.close()


def test_tile_wait_check_rejects_null_handle():
    lib = hobi.load_library()
    assert lib.hobi_check_tile_wait_timeout(None, None) == hobi.HOBI_ERR_ARG
