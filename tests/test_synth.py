"""Seeded input generators: sizes, closedness, orientation, determinism."""
import numpy as np

from paper_1301_5914_gb300 import synth


def test_icosphere_counts_and_orientation():
    for L in range(5):
        V, F, N = synth.icosphere(L, 2.0)
        assert V.shape == (10 * 4**L + 2, 3) and F.shape == (20 * 4**L, 3)
        st = synth.mesh_stats(V, F)
        assert st["closed_oriented"] and st["euler"] == 2
        assert np.allclose(np.linalg.norm(V, axis=1), 2.0, atol=1e-14)
        assert np.allclose(N * 2.0, V, atol=1e-14)
        a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
        assert np.all(np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c) > 0)


def test_ball_charges_seeded():
    q1 = synth.ball_charges(10, 8.0, 2)
    q2 = synth.ball_charges(10, 8.0, 2)
    assert np.array_equal(q1, q2)
    assert np.all(np.linalg.norm(q1[:, :3], axis=1) <= 8.0)
    assert np.all(np.abs(q1[:, 3]) <= 1.0)
