"""The library's treecode plan (host C++, no GPU) against the oracle treecode's plan: built from
the same FP64 node and target coordinates under the same rules, the two give identical
statistics (pair evaluations with nodes and with proxies, batches, proxy clusters)."""
import numpy as np
import pytest

import oracle
from oracle import treecode as tc
from paper_1301_5914_gb300 import hobi, synth


def _oracle_stats(y, x, degree, theta):
    src, _ = tc.build_tree(y, 256)
    batches, _ = tc.kd_batches(x, 256)
    lists = tc.interaction_lists(batches, src, theta, degree)
    n3 = (degree + 1) ** 3
    direct = sum((b["end"] - b["begin"]) * sum(src[c]["end"] - src[c]["begin"] for c in d)
                 for b, (d, a) in zip(batches, lists))
    approx = sum((b["end"] - b["begin"]) * len(a) * n3 for b, (d, a) in zip(batches, lists))
    pcs = {c for _, a in lists for c in a}
    return {"direct_pairs": direct, "approx_pairs": approx, "batches": len(batches), "proxy_clusters": len(pcs)}


@pytest.mark.parametrize("degree,theta", [(4, 0.8), (5, 0.7), (6, 0.5)])
def test_plan_matches_oracle_on_a_sphere(degree, theta):
    V, F, N = synth.icosphere(4, 10.0)
    orc = oracle.Problem(V, F, N, synth.ball_charges(3, 8.0, 2), 1.0, 80.0, 0.1257)
    y = orc.nodes()[0].reshape(-1, 3)
    assert hobi.fast_plan_stats(y, V, degree, theta) == _oracle_stats(y, V, degree, theta)


def test_plan_matches_oracle_on_a_molecule():
    V, F, N, Q = synth.synthetic_molecule(200, 11)
    orc = oracle.Problem(V, F, N, Q, 2.0, 80.0, 0.1257)
    y = orc.nodes()[0].reshape(-1, 3)
    got = hobi.fast_plan_stats(y, V, 5, 0.8)
    assert got == _oracle_stats(y, V, 5, 0.8)
    assert got["approx_pairs"] > 0 and got["direct_pairs"] + got["approx_pairs"] < len(V) * len(y)


def test_plan_argument_errors():
    y = np.zeros((10, 3))
    with pytest.raises(hobi.HobiError):
        hobi.fast_plan_stats(y, y, 1, 0.7)
    with pytest.raises(hobi.HobiError):
        hobi.fast_plan_stats(y, y, 4, 0.0)
