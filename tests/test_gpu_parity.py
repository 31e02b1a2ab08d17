"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: the plain FP64 GPU path agrees with the oracle to <= 1e-10 relative;
the FP32-bulk path to <= 1e-4 relative L2 for surface potentials and <= 1e-5
relative for the solvation energy. Integer/index tables are compared exactly.
"""
import numpy as np
import pytest

import oracle
from oracle import kirkwood as kw
from paper_1301_5914_gb300 import hobi, synth

pytestmark = pytest.mark.gpu

EPS1, EPS2, KAPPA = 1.0, 80.0, 0.1257


def _require_gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    _require_gpu()


def _case(level, radius, charges, eps1=EPS1, eps2=EPS2, kappa=KAPPA):
    V, F, N = synth.icosphere(level, radius)
    return V, F, N, charges, eps1, eps2, kappa


CASES = {
    # C1: radius 2, one charge at (0.5,0,0): 642 vertices, 5120 nodes (20 source tiles)
    "c1_l3": lambda: _case(3, 2.0, synth.point_charge(0.5, 0, 0, 1.0)),
    # radius 10, 10 charges (seed 2): 2562 vertices (3 ragged target blocks), 20480 nodes
    "c2_l4": lambda: _case(4, 10.0, synth.ball_charges(10, 8.0, 2)),
    # tiny: 42 vertices, 320 nodes (a ragged source tail inside one tile)
    "tiny_l1": lambda: _case(1, 1.0, synth.ball_charges(3, 0.6, 5), eps1=2.0, kappa=1.0),
}


@pytest.fixture(scope="module")
def problems():
    out = {}
    for k, f in CASES.items():
        V, F, N, Q, e1, e2, ka = f()
        out[k] = (V, F, N, Q, e1, e2, ka, oracle.Problem(V, F, N, Q, e1, e2, ka))
    return out


def _solver(p, prec="fp64", **kw):
    V, F, N, Q, e1, e2, ka, _ = p
    return hobi.Solver(V, F, N, Q, e1, e2, ka, precision=prec, **kw)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


@pytest.mark.parametrize("name", list(CASES))
def test_node_table_matches_oracle(problems, name):
    p = problems[name]
    s = _solver(p)
    y, nu, W = s.nodes()
    oy, onu, oW = p[-1].nodes()
    assert np.max(np.abs(y - oy)) <= 1e-12 * np.max(np.abs(oy))
    assert np.max(np.abs(nu - onu)) <= 1e-12
    assert np.max(np.abs(W - oW)) <= 1e-12 * np.max(np.abs(oW))


@pytest.mark.parametrize("name", ["c1_l3", "tiny_l1"])
def test_correction_table_matches_oracle(problems, name):
    """Each entry = (16-point singular rule) - (4-point regular rule) for that face."""
    p = problems[name]
    V, F, N, Q, e1, e2, ka, orc = p
    s = _solver(p)
    vert, face, coeff = s.correction()
    # adjacency: every (vertex, incident face) pair exactly once, sorted
    pairs = sorted((int(i), int(j)) for j in range(len(F)) for i in F[j])
    assert list(zip(vert.tolist(), face.tolist())) == pairs
    oy, onu, oW = orc.nodes()
    eps = e2 / e1
    sel = range(0, len(vert), max(1, len(vert) // 300))
    for e in sel:
        i, j = int(vert[e]), int(face[e])
        gl = orc.singular_coeffs(i, j)
        gr = np.zeros((3, 4))
        for m in range(4):
            K = oracle.kernels(V[i], N[i] / np.linalg.norm(N[i]), oy[j, m], onu[j, m], eps, ka)
            gr += np.outer(oW[j, m], K)
        ref = gl - gr
        assert np.max(np.abs(coeff[e] - ref)) <= 1e-10 * np.max(np.abs(gl)), e


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_matches_oracle(problems, name):
    p = problems[name]
    s = _solver(p)
    assert _rel(s.rhs(), p[-1].rhs()) <= 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_matvec_fp64_matches_oracle(problems, name):
    p = problems[name]
    s = _solver(p, "fp64")
    rng = np.random.default_rng(11)
    for _ in range(2):
        u = rng.normal(size=2 * s.nv)
        ref = p[-1].matvec(u)
        got = s.matvec(u)
        assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("name", list(CASES))
def test_matvec_fp32_bulk_accuracy(problems, name):
    """FP32 pair sums with compensated FP64 accumulation: relative L2 error <= 2e-6 on a smooth
    density (the solution), <= 1e-5 on a random vector."""
    p = problems[name]
    orc = p[-1]
    s = _solver(p, "fp32")
    u_sol, _, _, _ = orc.gmres(1e-8)
    assert _rel(s.matvec(u_sol), orc.matvec(u_sol)) <= 2e-6
    u = np.random.default_rng(3).normal(size=2 * s.nv)
    assert _rel(s.matvec(u), orc.matvec(u)) <= 1e-5


def test_matvec_deterministic_and_graph_free_equal(problems):
    p = problems["c2_l4"]
    for prec in ("fp32", "fp64"):
        s = _solver(p, prec)
        u = np.random.default_rng(5).normal(size=2 * s.nv)
        a, b = s.matvec(u), s.matvec(u)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("scaled", [True, False], ids=["scaled", "unscaled"])
@pytest.mark.parametrize("name", ["c1_l3", "c2_l4"])
def test_solve_fp64_matches_oracle(problems, name, scaled):
    """Same Krylov iterations as the oracle (x0 = 0), on the diagonally scaled unknowns and on
    the plain system: solutions agree to 1e-10, residual histories to 1e-8."""
    p = problems[name]
    orc = p[-1]
    u_ref, it_ref, conv, hist_ref = orc.gmres(1e-6, scaled=scaled)
    assert conv
    s = _solver(p, "fp64", gmres_scaling=scaled)
    phi, dphi, info = s.solve(1e-6, 200, history=64)
    assert info["converged"] and info["iterations"] == it_ref
    u = np.concatenate([phi, dphi])
    assert _rel(u, u_ref) <= 1e-10
    assert np.allclose(info["history"], hist_ref, rtol=1e-8, atol=0)
    assert abs(s.energy() - orc.energy(u_ref)) <= 1e-10 * abs(orc.energy(u_ref))


@pytest.mark.parametrize("name", ["c1_l3", "c2_l4", "tiny_l1"])
def test_solve_fp32_bulk_matches_oracle(problems, name):
    p = problems[name]
    orc = p[-1]
    u_ref, it_ref, conv, _ = orc.gmres(1e-6)
    s = _solver(p, "fp32")
    phi, dphi, info = s.solve(1e-6, 200)
    assert info["converged"] and abs(info["iterations"] - it_ref) <= 1
    nv = s.nv
    assert _rel(phi, u_ref[:nv]) <= 1e-4
    assert _rel(dphi, u_ref[nv:]) <= 1e-4
    e_ref = orc.energy(u_ref)
    assert abs(s.energy() - e_ref) <= 1e-5 * abs(e_ref)


def test_energy_and_reaction_potential_given_solution(problems):
    p = problems["c2_l4"]
    orc = p[-1]
    u_ref, _, _, _ = orc.gmres(1e-6)
    s = _solver(p, "fp64")
    s.set_solution(u_ref)
    assert np.array_equal(s.solution(), u_ref)
    assert abs(s.energy() - orc.energy(u_ref)) <= 1e-11 * abs(orc.energy(u_ref))
    pts = synth.ball_charges(37, 7.0, 9)[:, :3]
    ref = orc.reaction_potential(u_ref, pts)
    assert np.max(np.abs(s.reaction_potential(pts) - ref)) <= 1e-11 * np.max(np.abs(ref))
    s.set_precision("fp32")
    assert np.max(np.abs(s.reaction_potential(pts) - ref)) <= 1e-5 * np.max(np.abs(ref))
    assert abs(s.energy() - orc.energy(u_ref)) <= 1e-5 * abs(orc.energy(u_ref))


def test_born_sphere_on_gpu():
    """Table 2 on the GPU: E_sol = -81.98 for the radius-2 sphere, both precisions."""
    V, F, N = synth.icosphere(3, 2.0)
    for prec in ("fp64", "fp32"):
        s = hobi.Solver(V, F, N, synth.point_charge(0, 0, 0, 1.0), 1.0, 80.0, 0.0, precision=prec)
        s.solve(1e-8, 100)
        assert round(s.energy(), 2) == -81.98


def test_device_pointer_mode_matches_host_mode(problems):
    import torch

    V, F, N, Q, e1, e2, ka, orc = problems["c1_l3"]
    dev = torch.device("cuda:0")
    t = lambda a, dt=torch.float64: torch.as_tensor(a, dtype=dt, device=dev)
    for prec in ("fp64", "fp32"):
        sh = hobi.Solver(V, F, N, Q, e1, e2, ka, precision=prec)
        sd = hobi.Solver(t(V), t(F, torch.int32), t(N), t(Q), e1, e2, ka, precision=prec)
        u = np.random.default_rng(2).normal(size=2 * sh.nv)
        assert np.array_equal(sh.matvec(u), sd.matvec(t(u)).cpu().numpy())
        ph, dh, _ = sh.solve(1e-6)
        pd, dd, _ = sd.solve(1e-6)
        assert np.array_equal(ph, pd.cpu().numpy()) and np.array_equal(dh, dd.cpu().numpy())
        assert sh.energy() == sd.energy()


def test_graph_replay_equals_direct_launches(problems):
    p = problems["c2_l4"]
    a = _solver(p, "fp32", use_graph=True)
    b = _solver(p, "fp32", use_graph=False)
    pa, da, ia = a.solve(1e-6)
    pb, db, ib = b.solve(1e-6)
    assert ia["iterations"] == ib["iterations"]
    assert np.array_equal(pa, pb) and np.array_equal(da, db)


@pytest.mark.parametrize("scaled", [True, False], ids=["scaled", "unscaled"])
def test_restarted_gmres_matches_oracle(problems, scaled):
    p = problems["c1_l3"]
    orc = p[-1]
    u_ref, it_ref, conv, _ = orc.gmres(1e-9, max_it=200, restart=4, scaled=scaled)
    s = _solver(p, "fp64", restart=4, gmres_scaling=scaled)
    phi, dphi, info = s.solve(1e-9, 200)
    assert info["converged"] and info["iterations"] == it_ref
    assert _rel(np.concatenate([phi, dphi]), u_ref) <= 1e-9


def test_not_converged_status(problems):
    p = problems["c1_l3"]
    s = _solver(p, "fp64")
    phi, dphi, info = s.solve(1e-14, 3, raise_on_fail=False)
    assert info["status"] == hobi.HOBI_ERR_NOT_CONVERGED and info["iterations"] == 3
    assert np.all(np.isfinite(phi))


def test_mesh_errors_reported():
    V, F, N = synth.icosphere(2, 2.0)
    Q = synth.point_charge(0, 0, 0, 1.0)
    bad = [
        (V, F[:-1], N, "not closed"),
        (V, F[:, ::-1].copy(), N, "volume"),
        (V, np.where(F == 5, 10**6, F).astype(np.int32), N, "out of range"),
        (V, F, np.where(np.arange(len(N))[:, None] == 3, 0.0, N), "normal"),
    ]
    for Vb, Fb, Nb, msg in bad:
        with pytest.raises(hobi.HobiError) as ei:
            hobi.Solver(Vb, Fb, Nb, Q, 1.0, 80.0, 0.0)
        assert ei.value.code == hobi.HOBI_ERR_MESH and msg in str(ei.value)
    with pytest.raises(hobi.HobiError) as ei:
        hobi.Solver(V, F, N, Q, -1.0, 80.0, 0.0)
    assert ei.value.code == hobi.HOBI_ERR_ARG
    with pytest.raises(hobi.HobiError) as ei:
        hobi.Solver(V, F, N, np.array([[0, 0, np.nan, 1.0]]), 1.0, 80.0, 0.0)
    assert ei.value.code == hobi.HOBI_ERR_ARG


def test_energy_before_solve_is_state_error(problems):
    s = _solver(problems["tiny_l1"])
    with pytest.raises(hobi.HobiError) as ei:
        s.energy()
    assert ei.value.code == hobi.HOBI_ERR_STATE


def test_kirkwood_c2_level5_fp32_vs_fp64():
    """C2 at icosphere level 5 (20480 faces): both precisions solve in the same number of
    iterations, agree to the FP32 tolerances, and approach the Kirkwood solution."""
    V, F, N = synth.icosphere(5, 10.0)
    Q = synth.ball_charges(10, 8.0, 2)
    s = hobi.Solver(V, F, N, Q, 1.0, 80.0, 0.1257, precision="fp64")
    p64, d64, i64 = s.solve(1e-6)
    e64 = s.energy()
    s.set_precision("fp32")
    p32, d32, i32 = s.solve(1e-6)
    e32 = s.energy()
    assert abs(i64["iterations"] - i32["iterations"]) <= 1
    assert _rel(p32, p64) <= 1e-4 and abs(e32 - e64) <= 1e-5 * abs(e64)
    phi_ex, _ = kw.surface_potential(V, Q, 10.0, 1.0, 80.0, 0.1257)
    e_ex = kw.solvation_energy(Q, 10.0, 1.0, 80.0, 0.1257)
    assert np.max(np.abs(p64 - phi_ex)) / np.max(np.abs(phi_ex)) < 2e-3
    assert abs(e64 - e_ex) / abs(e_ex) < 2e-3


def test_profiling_counts_farfield_launches_with_graphs(problems):
    """Far-field timing via event nodes inside the captured graph: one launch per iteration
    (plus the energy launch), results identical to an unprofiled solve."""
    p = problems["c2_l4"]
    a = _solver(p, "fp32")
    b = _solver(p, "fp32")
    b.profile_enable(True)
    pa, da, ia = a.solve(1e-6)
    pb, db, ib = b.solve(1e-6)
    assert np.array_equal(pa, pb) and np.array_equal(da, db)
    b.energy()
    prof = b.profile_read()
    # every far-field launch timed (graph event nodes, or direct launches where those cannot be
    # timed -- the first replay is then lost to the switch)
    assert ib["iterations"] <= prof["launches"] <= ib["iterations"] + 1
    assert prof["farfield_ms"] > 0
    assert prof["pairs"] == (prof["launches"] - 1) * b.nv * b.n_nodes + b.nc * b.n_nodes
    assert b.kernel_launches() > 14 * ib["iterations"]


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
@pytest.mark.parametrize("scheme", ["hobi", "lobi"])
def test_every_block_shape_matches_oracle(problems, shape, scheme):
    """Each FP32 far-field block shape the autotuner may pick gives the same operator."""
    V, F, N, Q, e1, e2, ka, orc = problems["c2_l4"]
    s = hobi.Solver(V, F, N, Q, e1, e2, ka, precision="fp32", scheme=scheme, ff_shape=shape)
    assert s.plan_info()["shape"] == shape
    ref_p = orc if scheme == "hobi" else oracle.LobiProblem(V, F, N, Q, e1, e2, ka)
    u = np.random.default_rng(8).normal(size=2 * s.npts)
    assert _rel(s.matvec(u), ref_p.matvec(u)) <= 1e-5
    u_ref, it_ref, _, _ = ref_p.gmres(1e-6)
    phi, dphi, info = s.solve(1e-6)
    assert abs(info["iterations"] - it_ref) <= 1
    assert _rel(np.concatenate([phi, dphi]), u_ref) <= 1e-4


def test_autotuner_decides_once_per_size(problems):
    V, F, N, Q, e1, e2, ka, _ = problems["c1_l3"]
    a = hobi.Solver(V, F, N, Q, e1, e2, ka, precision="fp32")
    b = hobi.Solver(V, F, N, Q, e1, e2, ka, precision="fp32")
    ia, ib = a.plan_info(), b.plan_info()
    assert ia["tuned"] and ib["tuned"] and ia["shape"] == ib["shape"]
    c = hobi.Solver(V, F, N, Q, e1, e2, ka, precision="fp32", autotune=False)
    assert not c.plan_info()["tuned"]


def test_warm_start_resumes_and_checkpoint(problems):
    """Resume: a solve stopped at 1e-3 continued to 1e-6 reaches the oracle solution; a converged
    initial guess (a saved checkpoint of u) returns after 0 iterations."""
    p = problems["c2_l4"]
    orc = p[-1]
    u_ref, it_ref, _, _ = orc.gmres(1e-8)
    s = _solver(p, "fp64")
    _, _, i1 = s.solve(1e-3)
    phi, dphi, i2 = s.solve(1e-6, resume=True)
    assert i2["converged"] and i1["iterations"] + i2["iterations"] <= it_ref + 3
    assert _rel(np.concatenate([phi, dphi]), u_ref) <= 1e-5
    saved = s.solution()
    t = _solver(p, "fp64")
    phi3, dphi3, i3 = t.solve(1e-6, u0=saved)
    assert i3["iterations"] == 0 and i3["converged"]
    assert np.array_equal(np.concatenate([phi3, dphi3]), saved)
    fresh = _solver(p, "fp64")
    with pytest.raises(hobi.HobiError) as ei:
        fresh.solve(1e-6, resume=True)
    assert ei.value.code == hobi.HOBI_ERR_STATE


def test_correction_table_independent_of_precision_and_handle(problems):
    """The FP64 correction table of an FP32-bulk handle equals an FP64 handle's bit for bit, and
    fresh FP32 handles of one (tuned) size give bit-identical matvecs and solves."""
    p = problems["c2_l4"]
    orc = p[-1]
    _solver(p, "fp32").close()  # this size is tuned from here on
    ref = _solver(p, "fp64").correction()
    for a, b in zip(_solver(p, "fp32").correction(), ref):
        assert np.array_equal(a, b)
    u = np.random.default_rng(8).normal(size=2 * orc.nv)
    a, b = _solver(p, "fp32"), _solver(p, "fp32")
    assert np.array_equal(a.matvec(u), b.matvec(u))
    shape = a.plan_info()["shape"]
    assert np.array_equal(_solver(p, "fp32", ff_shape=shape).matvec(u), a.matvec(u))
    pa, da, ia = a.solve(1e-6, 200)
    pb, db, ib = b.solve(1e-6, 200)
    assert ia["iterations"] == ib["iterations"] and np.array_equal(pa, pb) and np.array_equal(da, db)
