"""Handles used from several host threads at once (include/hobi.h: one thread per handle, any
number of handles): four threads each set up, solve and destroy handles of different sizes and
precisions while the others run; every result equals the same work done sequentially."""
import threading

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


JOBS = [(3, 4.0, "fp32", 41), (4, 8.0, "fp32", 42), (3, 5.0, "fp64", 43), (2, 2.0, "fp32", 44)]


def _job(level, radius, prec, seed):
    V, F, N = synth.icosphere(level, radius)
    Q = synth.ball_charges(4, 0.6 * radius, seed)
    out = []
    for _ in range(3):
        s = hobi.Solver(V, F, N, Q, 2.0, 80.0, 0.1257, precision=prec)
        phi, dphi, info = s.solve(1e-8, 200)
        out.append((np.concatenate([phi, dphi]), s.energy(), info["iterations"]))
        s.close()
    return out


def test_handles_on_concurrent_threads_match_sequential_results():
    seq = [_job(*j) for j in JOBS]
    res = [None] * len(JOBS)
    errs = []

    def run(i):
        try:
            res[i] = _job(*JOBS[i])
        except Exception as e:  # reported below
            errs.append(e)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(len(JOBS))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errs, errs
    for a, b in zip(seq, res):
        for (ua, ea, ia), (ub, eb, ib) in zip(a, b):
            assert ia == ib and ea == eb and np.array_equal(ua, ub)
