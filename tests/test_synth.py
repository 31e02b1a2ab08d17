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


def _quality(V, F, N):
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    cr = np.cross(b - a, c - a)
    fn = cr / np.linalg.norm(cr, axis=1, keepdims=True)
    agree = np.einsum("ij,ij->i", fn, (N[F[:, 0]] + N[F[:, 1]] + N[F[:, 2]]) / 3)
    return agree


def test_synthetic_molecule_surface():
    """Gaussian-density molecule: closed, consistently oriented, outward, genus 0 here, normals
    unit and agreeing with the faces, integer net charge, seeded and reproducible, charges inside."""
    V, F, N, Q = synth.synthetic_molecule(60, 7)
    st = synth.mesh_stats(V, F)
    assert st["closed_oriented"] and st["euler"] == 2
    assert abs(F.shape[0] - 40 * 60) < 0.15 * 40 * 60
    assert np.allclose(np.linalg.norm(N, axis=1), 1.0)
    assert np.all(_quality(V, F, N) > 0.3)  # no face tilted more than ~72 deg from its normals
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    assert np.einsum("ij,ij->i", a, np.cross(b, c)).sum() > 0  # positive enclosed volume
    assert abs(Q[:, 3].sum() - round(Q[:, 3].sum())) < 1e-12
    V2, F2, N2, Q2 = synth.synthetic_molecule(60, 7)
    assert np.array_equal(V, V2) and np.array_equal(F, F2) and np.array_equal(Q, Q2)
    # every charge (atom centre) is inside: nearest surface vertex is farther than 0.5 A
    d = np.min(np.linalg.norm(V[None, :, :] - Q[:, None, :3], axis=2), axis=1)
    assert np.all(d > 0.5)


def test_two_globule_complex_is_one_closed_surface():
    """The C5 recipe at a small size: two seeded globules in contact give one closed, oriented
    surface (Euler characteristic 2), both globules' charges inside it, reproducible."""
    V, F, N, Q = synth.two_globule_complex(60, 51, 52, n_faces=6000)
    st = synth.mesh_stats(V, F)
    assert st["closed_oriented"] and st["euler"] == 2
    assert Q.shape[0] == 120 and abs(F.shape[0] - 6000) < 0.15 * 6000
    assert np.allclose(np.linalg.norm(N, axis=1), 1.0)
    # the two halves: atoms of each globule on either side of the contact plane
    rg = 20.0 * (60 / 1000.0) ** (1.0 / 3.0)
    assert np.median(Q[:60, 0]) < rg - 1.0 < np.median(Q[60:, 0])
    d = np.min(np.linalg.norm(V[None, :, :] - Q[:, None, :3], axis=2), axis=1)
    assert np.all(d > 0.5)
    V2, F2, N2, Q2 = synth.two_globule_complex(60, 51, 52, n_faces=6000)
    assert np.array_equal(V, V2) and np.array_equal(F, F2)


def test_point_charge_and_icosphere_radius():
    q = synth.point_charge(0.5, -0.25, 0.0, 2.0)
    assert q.shape == (1, 4) and np.array_equal(q[0], [0.5, -0.25, 0.0, 2.0])
    V, F, N = synth.icosphere(3, 2.5, center=(1.0, 0.0, -1.0))
    r = np.linalg.norm(V - [1.0, 0.0, -1.0], axis=1)
    assert np.allclose(r, 2.5) and np.allclose(N, (V - [1.0, 0.0, -1.0]) / 2.5)
