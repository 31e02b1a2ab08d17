#!/usr/bin/env python3
"""Benchmark of the HOBI-PB hot path on GB300.

One step = the whole hot path on one synthetic molecule with its inputs resident
in HBM: hobi_setup (mesh validation, adjacency, curved-element nodes, singular
correction table, right-hand side), hobi_solve (GMRES to 1e-6 on the diagonally
scaled unknowns: per iteration the scaled Arnoldi vector, gather + far-field pair
sum + correction/diagonal + FP64 Arnoldi/Givens) and hobi_energy. Workload: Kirkwood sphere of radius 10 A, icosphere level 6
(81,920 curved triangles, 40,962 vertices, 327,680 quadrature nodes), 10 seeded
charges uniform in a radius-8 ball, eps1 = 1, eps2 = 80, kappa = 0.1257 1/A;
FP32-bulk far field.

value = far-field pair evaluations per second over the whole step (all ranks).
With --gpus N > 1 (torchrun) every rank solves its own replica (no collective on
the data path): weak scaling.

--workload selects other configurations for explicit runs (the default is the
one above): c3 (1000-atom synthetic molecule, ~40k triangles, eps1 = 2), c5 (two
3000-atom globules in contact, ~120k triangles) and c4 (64 synthetic molecules of
50-2000 atoms, log-uniform, solved as one batch).

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (matvec rows), same metric and unit.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "matvec pair-evals/s & %FP32 peak; GMRES time to 1e-6 (FP32-bulk vs FP64 plain)"
UNIT = "pair-evals/s"
WORKLOAD_C2 = {
    "workload": "kirkwood_sphere_r10_ico6_10charges",
    "mesh": "icosphere level 6, radius 10 A, exact radial normals",
    "n_faces": 81920,
    "n_vertices": 40962,
    "n_nodes": 327680,
    "n_charges": 10,
    "charges": "uniform in r<=8 A ball, q~U[-1,1] e, seed 2",
    "eps1": 1.0,
    "eps2": 80.0,
    "kappa": 0.1257,
    "gmres_tol": 1e-6,
    "precision": "fp32-bulk far field (FP32 pair sums, compensated tile sums, FP64 GMRES/correction/energy)",
}
WORKLOAD = WORKLOAD_C2
MOLECULE = {"eps1": 2.0, "eps2": 80.0, "kappa": 0.1257, "gmres_tol": 1e-6,
            "precision": WORKLOAD_C2["precision"],
            "surface": "Gaussian-density isosurface (marching tetrahedra, smoothed), density-gradient normals"}
# FP32 FMA-pipe operations per pair in the both-rows far-field kernel as written (kappa > 0:
# 6 for d and r^2, 3 for d.m, 3 for 1/r^2, 1/r^3 and v, 2 for 1 + kappa r and the exp2 argument,
# 1 for P - 1, 4 for row 1, 3 for S, 2 for the 1/r^3 factors, 6 for the vector accumulation)
OPS_PER_PAIR = 30
OPS_PER_PAIR_ROW1 = 18  # row 1 only (reaction potential, energy): d, r^2, d.m, 1/r^2, v, 1 + kappa r,
#                        the exp2 argument, P - 1 and the 4 operations of row 1
MUFU_PER_PAIR = 2  # rsqrt.approx + ex2.approx
OPS_PER_PAIR_FIELD = 28  # reaction field: d, r^2, d.m, 1/r^2, v, 1 + kappa r, exponent, P - 1, P - 1/eps,
#                          1/r^3, beta (4), its and (P - 1/eps)/r^3 factors (2), 3-vector accumulation (6)
# MUFU (XU) lanes per SM per clock: an rsqrt.approx.f32 throughput microbenchmark (independent
# chains, CUDA events) measured 15.9 lane-operations per SM per clock on GB300 at 2070 MHz.
MUFU_LANES_PER_SM = 16
# FP64 far field (kappa > 0, both rows): FP64-pipe operations per pair as written: 3 for d, 3 for
# r^2, 5 for the Newton step of 1/r, 1 for r, 1 for the exp argument, 3 for its reduction, 4 for its
# polynomial, 1 for the table product, 2 for P - 1, 3 for d.m, 2 for 1/r^2 and v, 4 for row 1 and
# 12 for row 2 (S, 1/r^3, the two factors, the vector accumulation).
FP64_OPS_PER_PAIR = 44
# FP64-pipe lanes per SM per clock: the nominal 1.25 TFLOP/s FP64 rate of GB300 is 0.625e12 FMA per
# second = 2 lanes per SM per clock at 152 SMs x 2070 MHz. (ncu on the FP64 far field: 1.70 FP64
# thread instructions per SM per cycle with sm__pipe_fp64_cycles_active at 88.9 % of peak, i.e. a
# pipe peak of about 1.9.)
FP64_LANES_PER_SM = 2.0
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "farfield32_c2_ico6_traffic.txt")
FARFIELD_SRC = [os.path.join(ROOT, "paper_1301_5914_gb300", "csrc", f) for f in ("k_farfield.cu", "ff_body.cuh")]


def _inputs():
    from paper_1301_5914_gb300 import synth

    V, F, N = synth.icosphere(6, 10.0)
    Q = synth.ball_charges(10, 8.0, 2)
    return V, F, N, Q


def _c4_member(m):
    import numpy as np

    from paper_1301_5914_gb300 import synth

    n_atoms = int(round(np.exp(np.random.default_rng(1000 + m).uniform(np.log(50), np.log(2000)))))
    return synth.synthetic_molecule(n_atoms, 1000 + m)


def make_workload(name):
    """(config dict, list of (V, F, N, Q) molecules); one molecule unless batched."""
    from paper_1301_5914_gb300 import synth

    if name == "c2l6":
        return dict(WORKLOAD_C2), [_inputs()]
    if name == "c3":
        mol = synth.synthetic_molecule(1000, 3)
        cfg = dict(MOLECULE, workload="synthetic_molecule_1000_atoms_seed3", n_atoms=1000)
    elif name == "c5":
        mol = synth.two_globule_complex(3000, 51, 52, n_faces=120000)
        cfg = dict(MOLECULE, workload="two_globule_complex_2x3000_atoms_seeds51_52", n_atoms=6000)
    elif name == "c4":
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
            mols = pool.map(_c4_member, range(64))
        cfg = dict(MOLECULE, workload="batch_64_synthetic_molecules_50_2000_atoms_seeds1000_1063",
                   n_molecules=64, n_atoms=int(sum(m[3].shape[0] for m in mols)))
        cfg.update(n_faces=int(sum(m[1].shape[0] for m in mols)), n_vertices=int(sum(m[0].shape[0] for m in mols)),
                   n_nodes=int(sum(4 * m[1].shape[0] for m in mols)), n_charges=cfg["n_atoms"],
                   faces_min_max=[int(min(m[1].shape[0] for m in mols)), int(max(m[1].shape[0] for m in mols))])
        return cfg, mols
    else:
        raise ValueError(name)
    V, F, N, Q = mol
    cfg.update(n_faces=int(F.shape[0]), n_vertices=int(V.shape[0]), n_nodes=int(4 * F.shape[0]),
               n_charges=int(Q.shape[0]))
    return cfg, [mol]


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def gather_rank_times(total_ms: float, world_size: int, device=None) -> list[float]:
    """Every rank's timed-region total (ms), via all_gather on the default process group."""
    if world_size <= 1:
        return [total_ms]
    import torch
    import torch.distributed as dist

    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    gathered = [torch.zeros_like(t) for _ in range(world_size)]
    dist.all_gather(gathered, t)
    return [float(g.item()) for g in gathered]


def aggregate(per_rank_total_ms: list[float], pairs_per_step: float, steps: int) -> tuple[float, float]:
    """Whole-job throughput: all ranks' pairs over the slowest rank's time."""
    t = max(per_rank_total_ms)
    return len(per_rank_total_ms) * pairs_per_step * steps / (t / 1e3), t / steps


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _cpu_model(path: str = "/proc/cpuinfo") -> str:
    """The host CPU's model name from /proc/cpuinfo (on Arm: implementer and part codes)."""
    fields = {}
    try:
        with open(path) as f:
            for line in f:
                k, _, v = line.partition(":")
                fields.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    if fields.get("model name"):
        return fields["model name"]
    import platform

    parts = [platform.machine() or "unknown"]
    if "CPU implementer" in fields and "CPU part" in fields:
        parts.append(f"(CPU implementer {fields['CPU implementer']}, part {fields['CPU part']})")
    return " ".join(parts)


def _traffic_per_launch():
    """DRAM bytes per far-field launch from the committed ncu summary, if the kernel source is unchanged."""
    try:
        rec = {}
        for line in open(TRAFFIC_FILE):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                rec[k.strip()] = v.strip()
        h = hashlib.sha256(b"".join(open(f, "rb").read() for f in FARFIELD_SRC)).hexdigest()
        if rec.get("kernel_source_sha256") == h:
            return int(rec["dram_bytes_per_launch_full_size"])
    except (OSError, ValueError, KeyError):
        pass
    return None


def cpu_oracle_sample(V, F, N, Q, rows: int, params=None, seed: int = 0, threads: int = 0):
    """Time the FP64 oracle's matvec on `rows` sampled rows of the workload (bounded CPU work),
    on all host cores or on `threads` threads."""
    import numpy as np

    import oracle

    p = params or WORKLOAD
    prob = oracle.Problem(V, F, N, Q, p["eps1"], p["eps2"], p["kappa"])
    rng = np.random.default_rng(seed)
    u = rng.normal(size=2 * prob.nv)
    rows = min(rows, prob.nv)
    sel = np.sort(rng.choice(prob.nv, size=rows, replace=False))
    all_threads = oracle.num_threads()
    if threads:
        oracle.set_num_threads(threads)
    try:
        used = oracle.num_threads()
        t0 = time.perf_counter()
        prob.matvec_rows(u, sel)
        dt = time.perf_counter() - t0
    finally:
        if threads:
            oracle.set_num_threads(all_threads)
    pairs = rows * 4.0 * prob.nf
    return pairs / dt, dt, pairs, used


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    V, F, N, Q = _inputs()
    rows = args.ref_rows
    for _ in range(args.warmup):
        cpu_oracle_sample(V, F, N, Q, max(8, rows // 8), seed=99)
    t_total, pairs_total, cores = 0.0, 0.0, 1
    for k in range(args.steps):
        _, dt, pairs, cores = cpu_oracle_sample(V, F, N, Q, rows, seed=k)
        t_total += dt
        pairs_total += pairs
    value = pairs_total / t_total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(WORKLOAD, precision="FP64 CPU oracle (plain C, OpenMP over rows)",
                       sample=f"{rows} sampled matvec rows per step"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": _cpu_model(),
                         "sample": f"{rows} of {V.shape[0]} matvec rows x {4 * F.shape[0]} nodes per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def step_phases(make, batched, tol, stream):
    """Setup, one matvec, the GMRES solve and the energy of one FP32 step, timed separately."""
    import torch

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    s = make("fp32")
    ev[1].record(stream)
    u = torch.ones(2 * s.nv, dtype=torch.float64, device=stream.device)
    for _ in range(3):
        s.matvec(u)
    ev[2].record(stream)
    for _ in range(10):
        s.matvec(u)
    ev[3].record(stream)
    phi, dphi, info = s.solve(tol, 400)
    ev[4].record(stream)
    s.energy()
    ev[5].record(stream)
    torch.cuda.synchronize()
    s.close()
    return {"setup_ms": ev[0].elapsed_time(ev[1]), "matvec_ms": ev[2].elapsed_time(ev[3]) / 10,
            "solve_ms": ev[3].elapsed_time(ev[4]), "energy_ms": ev[4].elapsed_time(ev[5]),
            "iterations": info["iterations"],
            "note": "setup includes the autotuner only on a problem size's first setup in a process"}


def fast_summation(hobi, arrays, e1, e2, ka, tol, stream, degree, theta):
    """Treecode far field (degree, theta) against the direct FP32 far field on the same problem."""
    import numpy as np
    import torch

    out = {"degree": degree, "theta": theta}
    u = torch.as_tensor(np.random.default_rng(0).normal(size=2 * arrays[0].shape[0]), device=arrays[0].device)
    res = {}
    for name, kw in (("direct", {}), ("fast", {"fast_degree": degree, "fast_theta": theta})):
        s = hobi.Solver(*arrays, e1, e2, ka, precision="fp32", stream=stream, **kw)
        s.profile_enable(True)
        for _ in range(3):
            s.matvec(u)
        s.profile_read()
        for _ in range(10):
            Au = s.matvec(u)
        p = s.profile_read()
        phi, dphi, info = s.solve(tol, 400)
        res[name] = dict(ms=p["farfield_ms"] / p["launches"], Au=Au, phi=torch.cat([phi, dphi]), E=s.energy(),
                         solve_ms=info["solve_ms"], it=info["iterations"], fi=s.fast_info(), nv=s.nv, nn=s.n_nodes)
        s.close()
    d, f = res["direct"], res["fast"]
    rel = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
    out.update(farfield_ms_direct=d["ms"], farfield_ms_fast=f["ms"], farfield_speedup=d["ms"] / f["ms"],
               pairs_fraction=(f["fi"]["direct_pairs"] + f["fi"]["approx_pairs"]) / (d["nv"] * d["nn"]),
               batches=f["fi"]["batches"], proxy_clusters=f["fi"]["proxy_clusters"],
               solve_ms_direct=d["solve_ms"], solve_ms_fast=f["solve_ms"], iterations_direct=d["it"],
               iterations_fast=f["it"], matvec_rel_l2_vs_direct=rel(f["Au"], d["Au"]),
               u_rel_l2_vs_direct=rel(f["phi"], d["phi"]), E_rel_vs_direct=abs(f["E"] - d["E"]) / abs(d["E"]))
    return out


def fast_summation_batch(hobi, mols, arrays, e1, e2, ka, tol, stream, degree, theta):
    """Batched solve with fast summation for the molecules it pays off on, against the direct batch."""
    import numpy as np

    res = {}
    for name, kw in (("direct", {}), ("fast", {"fast_degree": degree, "fast_theta": theta})):
        b = hobi.BatchSolver(mols, e1, e2, ka, precision="fp32", device_arrays=arrays, stream=stream, **kw)
        b.profile_enable(True)
        phis, dphis, info = b.solve(tol, 400)
        p = b.profile_read()
        res[name] = dict(ms=p["farfield_ms"], launches=p["launches"], pairs=p["pairs"], E=np.asarray(b.energy()),
                         solve_ms=info["solve_ms"], it=info["iterations"].tolist())
        b.close()
    d, f = res["direct"], res["fast"]
    return {"degree": degree, "theta": theta, "farfield_ms_direct": d["ms"], "farfield_ms_fast": f["ms"],
            "farfield_speedup": d["ms"] / f["ms"], "pairs_fraction": f["pairs"] / d["pairs"],
            "solve_ms_direct": d["solve_ms"], "solve_ms_fast": f["solve_ms"],
            "solve_speedup": d["solve_ms"] / f["solve_ms"],
            "E_rel_vs_direct_max": float(np.max(np.abs(f["E"] - d["E"]) / np.abs(d["E"]))),
            "iterations_fast_minus_direct_max": int(np.max(np.abs(np.asarray(f["it"]) - np.asarray(d["it"]))))}


def ff_launch_rate(prof):
    """Average duration (s) and pair evaluations of the profiled far-field launches."""
    n = max(int(prof["launches"]), 1)
    return prof["farfield_ms"] / n / 1e3, prof["pairs"] / n


def alu_fraction(launch_s, pairs_per_launch, ops_per_pair, lanes_per_sm, sms, f_mhz):
    """Achieved lane operations per second of one kernel and its fraction of SMs x lanes x clock."""
    achieved = pairs_per_launch * ops_per_pair / launch_s
    peak = sms * lanes_per_sm * f_mhz * 1e6
    return achieved, peak, achieved / peak


def _dev(arrays, dev):
    import torch

    return tuple(torch.as_tensor(a, device=dev) for a in arrays)


def extra_workload(hobi, name, dev, stream, sms, fmax, fp64_sample=4):
    """One more benchmark workload, measured outside the timed region: its FP32 far-field rate
    and lane-peak fraction in a GMRES solve to 1e-6, the solve time, and the FP32-bulk solution
    against the FP64 operator's (mixed-precision refinement to 1e-10 on the FP64 far field; for a
    batch, on `fp64_sample` sampled molecules). Plain FP64 GMRES on these sizes runs for minutes
    and is not repeated here."""
    import numpy as np
    import torch

    t0 = time.perf_counter()
    cfg, mols = make_workload(name)
    gen_s = time.perf_counter() - t0
    e1, e2, ka, tol = cfg["eps1"], cfg["eps2"], cfg["kappa"], cfg["gmres_tol"]
    rec = {k: cfg[k] for k in ("workload", "n_faces", "n_vertices", "n_nodes", "n_charges") if k in cfg}
    rec["generate_s"] = gen_s
    rel = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
    relmax = lambda a, b: float(torch.max(torch.abs(a - b)) / torch.max(torch.abs(b)))
    if len(mols) == 1:
        s = hobi.Solver(*_dev(mols[0], dev), e1, e2, ka, precision="fp32", stream=stream)
        s.profile_enable(True)
        phi, dphi, info = s.solve(tol, 400)
        prof = s.profile_read()
        E32 = s.energy()
        _, _, ir = s.solve_refined(1e-10, 8, 400)
        u64 = s.solution()
        E64 = s.energy()
        s.close()
        nv = phi.numel()
        acc = {"phi_rel_l2": rel(phi, u64[:nv]), "phi_rel_max": relmax(phi, u64[:nv]),
               "dphi_rel_l2": rel(dphi, u64[nv:]), "E_sol_fp32": E32, "E_sol_fp64_operator": E64,
               "E_rel": abs(E32 - E64) / abs(E64), "reference": "FP64-operator solution (refinement to 1e-10)",
               "reference_s": ir["solve_ms"] / 1e3, "reference_fp64_residual": ir["rel_residual"]}
        gm = {"fp32_bulk_s": info["solve_ms"] / 1e3, "iterations": info["iterations"]}
    else:
        arrays = _dev([np.concatenate([np.asarray(m[k]).reshape(-1, 4 if k == 3 else 3) for m in mols]).astype(
            np.int32 if k == 1 else np.float64) for k in range(4)], dev)
        b = hobi.BatchSolver(mols, e1, e2, ka, precision="fp32", device_arrays=arrays, stream=stream)
        b.profile_enable(True)
        phis, dphis, info = b.solve(tol, 400)
        prof = b.profile_read()
        E32 = np.asarray(b.energy())
        b.close()
        order = np.argsort([m[1].shape[0] for m in mols])
        sample = [int(order[i]) for i in np.linspace(0, len(mols) - 1, fp64_sample).round().astype(int)]
        worst = {"phi_rel_l2": 0.0, "phi_rel_max": 0.0, "dphi_rel_l2": 0.0, "E_rel": 0.0}
        for m in sample:
            s = hobi.Solver(*_dev(mols[m], dev), e1, e2, ka, precision="fp32", stream=stream)
            s.solve_refined(1e-10, 8, 400)
            u64 = s.solution()
            E64 = s.energy()
            s.close()
            nv = mols[m][0].shape[0]
            p32, d32 = torch.as_tensor(phis[m], device=dev), torch.as_tensor(dphis[m], device=dev)
            for k, v in (("phi_rel_l2", rel(p32, u64[:nv])), ("phi_rel_max", relmax(p32, u64[:nv])),
                         ("dphi_rel_l2", rel(d32, u64[nv:])), ("E_rel", abs(E32[m] - E64) / abs(E64))):
                worst[k] = max(worst[k], v)
        acc = dict(worst, reference=f"FP64-operator solutions (refinement to 1e-10) of molecules {sample}, "
                                    "worst of them")
        its = info["iterations"].tolist()
        gm = {"fp32_bulk_s": info["solve_ms"] / 1e3, "iterations_min_max": [int(min(its)), int(max(its))],
              "n_molecules": len(mols)}
    launch_s, pairs = ff_launch_rate(prof)
    ach, peak, frac = alu_fraction(launch_s, pairs, OPS_PER_PAIR, 128, sms, fmax)
    rec.update(farfield={"kernel": "k_farfield_batch32" if len(mols) > 1 else "k_farfield32<ROW2=true>",
                         "pairs_per_s": pairs / launch_s, "avg_launch_ms": launch_s * 1e3, "launches": prof["launches"],
                         "frac_fp32_lane_peak": frac, "mufu_frac": pairs * MUFU_PER_PAIR / launch_s / (sms * MUFU_LANES_PER_SM * fmax * 1e6)},
               gmres_fp32_bulk=gm, accuracy_fp32_vs_fp64_operator=acc,
               fp64_plain="not run: plain FP64 GMRES on this size takes minutes")
    return rec


def lobi_object(hobi, arrays, e1, e2, ka, tol, stream, sms, fmax):
    """LOBI-PB (the paper's low-order scheme) on the same surface: its self-skipping FP32 far field
    (N_f targets x N_f sources per matvec) and its GMRES to 1e-6."""
    import numpy as np
    import torch

    s = hobi.Solver(*arrays, e1, e2, ka, precision="fp32", scheme="lobi", stream=stream)
    u = torch.as_tensor(np.random.default_rng(0).normal(size=2 * s.npts), device=arrays[0].device)
    s.profile_enable(True)
    for _ in range(3):
        s.matvec(u)
    s.profile_read()
    for _ in range(10):
        s.matvec(u)
    launch_s, pairs = ff_launch_rate(s.profile_read())
    _, _, frac = alu_fraction(launch_s, pairs, OPS_PER_PAIR, 128, sms, fmax)
    phi, dphi, info = s.solve(tol, 400)
    E = s.energy()
    s.close()
    return {"scheme": "LOBI-PB (flat faces, centroid collocation, self term dropped)", "n_unknowns": 2 * s.npts,
            "pairs_per_matvec": pairs, "farfield_ms": launch_s * 1e3, "pairs_per_s": pairs / launch_s,
            "frac_fp32_lane_peak": frac, "ops_per_pair": f"{OPS_PER_PAIR} FP32 FMA-pipe (+ a zero-distance select in the tiles holding the block's own targets)",
            "gmres_fp32_bulk_s": info["solve_ms"] / 1e3, "iterations": info["iterations"], "E_sol": E}


def reaction_object(hobi, arrays, e1, e2, ka, tol, stream, sms, fmax, n_points=16384, radius=8.0):
    """Off-surface output: the reaction potential and the reaction field at n_points interior points
    from a solved handle, FP32-bulk and FP64 (N_points x N_nodes pairs per call)."""
    import numpy as np
    import torch

    from paper_1301_5914_gb300 import synth

    pts = torch.as_tensor(synth.ball_charges(n_points, radius, 77)[:, :3].copy(), device=arrays[0].device)
    s = hobi.Solver(*arrays, e1, e2, ka, precision="fp32", stream=stream)
    s.solve(tol, 400)
    out = {"n_points": n_points, "points": f"uniform in the r <= {radius} A ball, seed 77"}
    for prec, ops, lanes in (("fp32", OPS_PER_PAIR_ROW1, 128), ("fp64", None, FP64_LANES_PER_SM)):
        s.set_precision(prec)
        s.profile_enable(True)
        for _ in range(2):
            s.reaction_potential(pts)
        s.profile_read()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        reps = 5 if prec == "fp32" else 2
        ev[0].record(stream)
        for _ in range(reps):
            phi = s.reaction_potential(pts)
        ev[1].record(stream)
        torch.cuda.synchronize()
        launch_s, pairs = ff_launch_rate(s.profile_read())
        rec = {"call_ms": ev[0].elapsed_time(ev[1]) / reps, "farfield_ms": launch_s * 1e3, "pairs_per_s": pairs / launch_s}
        if ops:
            rec["frac_fp32_lane_peak"] = alu_fraction(launch_s, pairs, ops, lanes, sms, fmax)[2]
        # the reaction field at the same points (whole call: points, gather, field kernel, reduction)
        s.reaction_field(pts)
        ev[0].record(stream)
        for _ in range(reps):
            fld = s.reaction_field(pts)
        ev[1].record(stream)
        torch.cuda.synchronize()
        call_s = ev[0].elapsed_time(ev[1]) / reps / 1e3
        field_pairs = float(n_points) * s.n_nodes
        rec["field_call_ms"] = call_s * 1e3
        rec["field_pairs_per_s"] = field_pairs / call_s
        if ops:
            rec["field_frac_fp32_lane_peak"] = alu_fraction(call_s, field_pairs, OPS_PER_PAIR_FIELD, lanes, sms, fmax)[2]
        out[prec] = rec
        if prec == "fp32":
            phi32, fld32 = phi.clone(), fld.clone()
    out["fp32_vs_fp64_rel_l2"] = float(torch.linalg.norm(phi32 - phi) / torch.linalg.norm(phi))
    out["field_fp32_vs_fp64_rel_l2"] = float(torch.linalg.norm(fld32 - fld) / torch.linalg.norm(fld))
    out["field_ops_per_pair"] = f"{OPS_PER_PAIR_FIELD} FP32 FMA-pipe + 2 MUFU"
    s.close()
    return out


def run_ours(args):
    cfg, mols = make_workload(args.workload)  # before any CUDA call (the c4 generator uses a spawn pool)
    import numpy as np
    import torch

    from paper_1301_5914_gb300 import hobi

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    e1, e2, ka, tol = cfg["eps1"], cfg["eps2"], cfg["kappa"], cfg["gmres_tol"]
    batched = len(mols) > 1
    cat = lambda k, dt=np.float64: np.ascontiguousarray(np.concatenate([np.asarray(m[k]).reshape(-1, 4 if k == 3 else 3)
                                                                         for m in mols]), dtype=dt)
    Vh, Fh, Nh, Qh = cat(0), cat(1, np.int32), cat(2), cat(3)
    Vd, Fd, Nd, Qd = (torch.as_tensor(a, device=dev) for a in (Vh, Fh, Nh, Qh))
    stream = torch.cuda.current_stream(dev)
    energy_pairs = float(sum(m[3].shape[0] * 4.0 * m[1].shape[0] for m in mols))

    def make(precision, host=False):
        if batched:
            if host:
                return hobi.BatchSolver(mols, e1, e2, ka, precision=precision)
            return hobi.BatchSolver(mols, e1, e2, ka, precision=precision, device_arrays=(Vd, Fd, Nd, Qd), stream=stream)
        if host:
            pin = [torch.as_tensor(a).pin_memory() for a in (Vh, Fh, Nh, Qh)]
            return hobi.Solver(*pin, e1, e2, ka, precision=precision)
        return hobi.Solver(Vd, Fd, Nd, Qd, e1, e2, ka, precision=precision, stream=stream)

    def step(profile: bool, precision="fp32", host=False):
        """setup + solve + energy; with profile, the far-field launches of the solve (the matvecs)
        and those of the energy are read separately."""
        s = make(precision, host)
        if profile:
            s.profile_enable(True)
        phi, dphi, info = s.solve(tol, 400)
        prof = s.profile_read() if profile else None
        E = s.energy()
        prof_e = s.profile_read() if profile else None
        n_launch = s.kernel_launches()
        s.close()
        return info, E, prof, prof_e, n_launch, phi, dphi

    for _ in range(args.warmup):
        step(False)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    times, ff_ms, ff_launch, ff_pairs, pairs_step, launches, iters = [], 0.0, 0, 0.0, [], 0, []
    E = None
    for k in range(args.steps):
        flush.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        info, E, prof, prof_e, nl, _, _ = step(True)
        ev1.record(stream)
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1))
        ff_ms += prof["farfield_ms"]
        ff_launch += prof["launches"]
        ff_pairs += prof["pairs"]
        # single molecule: the energy's far-field launch is profiled on its own; a batch computes
        # its energies per molecule (not profiled), so their pairs are counted from the sizes
        pairs_step.append(prof["pairs"] + (energy_pairs if batched else prof_e["pairs"]))
        launches += nl
        iters.append(info["iterations"].tolist() if batched else info["iterations"])
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = sum(times)
    per_rank = gather_rank_times(total_ms, ws, dev)
    pairs_per_step = statistics.mean(pairs_step)
    value, ms_per_step = aggregate(per_rank, pairs_per_step, args.steps)

    if rank == 0:
        # roofline of the dominant kernel: the far field of the GMRES matvecs (FP32 bulk, both rows),
        # live CUDA-event timing of those launches only (the energy launch is reported apart)
        props = torch.cuda.get_device_properties(dev)
        sms = props.multi_processor_count
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
            fmax = float(peaks.get("sm_max_mhz", 2070.0))
            peak_src = "MEASURED_PEAKS.json sm_max_mhz"
        except (OSError, ValueError):
            fmax, peak_src = 2070.0, "nominal maximum SM clock (MEASURED_PEAKS.json absent)"
        peak = sms * 128 * fmax * 1e6 / 1e9  # Ginst/s, FP32 FMA-pipe lanes
        avg_launch_s = ff_ms / ff_launch / 1e3
        pairs_per_launch = ff_pairs / ff_launch
        achieved = pairs_per_launch * OPS_PER_PAIR / avg_launch_s / 1e9
        traffic = _traffic_per_launch() if args.workload == "c2l6" else None
        fobs = clk.get("sm_mhz") or fmax
        roof = {
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Ginst/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": "k_farfield32<ROW2=true>" if not batched else "k_farfield_batch32",
            "algorithmic": f"{OPS_PER_PAIR} FP32 FMA-pipe instructions + {MUFU_PER_PAIR} MUFU per pair",
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x {fmax:.0f} MHz ({peak_src})",
            "pairs_per_s": pairs_per_launch / avg_launch_s,
            "avg_launch_ms": avg_launch_s * 1e3,
            "launches_per_step": ff_launch / args.steps,
            "frac_at_median_clock": achieved / (sms * 128 * fobs * 1e6 / 1e9),
            "mufu_frac": pairs_per_launch * MUFU_PER_PAIR / avg_launch_s / (sms * MUFU_LANES_PER_SM * fmax * 1e6),
            "mufu_basis": f"{sms} SMs x {MUFU_LANES_PER_SM} MUFU lanes (rsqrt.approx.f32 microbenchmark) x {fmax:.0f} MHz",
            "farfield_share_of_step": ff_ms / total_ms,
        }
        if not batched:
            roof["energy_launch_ms"] = prof_e["farfield_ms"] / max(prof_e["launches"], 1)
        # FP64 plain path on the same inputs (outside the timed region): GMRES time to 1e-6 and the
        # roofline of its far-field kernel
        gm = {"fp32_bulk_s": None, "fp64_plain_s": None}
        acc = {}
        fp64_roof = None
        if not args.no_fp64:
            i64, E64, p64prof, _, _, p64, d64 = step(True, "fp64")
            i32, E32, _, _, _, p32, d32 = step(False, "fp32")
            it32 = i32["iterations"].tolist() if batched else i32["iterations"]
            it64 = i64["iterations"].tolist() if batched else i64["iterations"]
            gm = {"fp32_bulk_s": i32["solve_ms"] / 1e3, "fp64_plain_s": i64["solve_ms"] / 1e3,
                  "iterations_fp32": it32, "iterations_fp64": it64, "speedup": i64["solve_ms"] / i32["solve_ms"]}
            l64, pr64 = ff_launch_rate(p64prof)
            a64, pk64, f64 = alu_fraction(l64, pr64, FP64_OPS_PER_PAIR, FP64_LANES_PER_SM, sms, fmax)
            fp64_roof = {"bound": "alu", "kernel": "k_farfield64<ROW2=true>" if not batched else "k_farfield_batch64",
                         "achieved": a64 / 1e9, "peak": pk64 / 1e9, "unit": "Ginst/s", "frac": f64,
                         "algorithmic": f"{FP64_OPS_PER_PAIR} FP64-pipe instructions + 1 MUFU (rsqrt seed) per pair",
                         "peak_basis": f"{sms} SMs x {FP64_LANES_PER_SM:g} FP64 lanes (nominal 1.25 TFLOP/s) x {fmax:.0f} MHz",
                         "pairs_per_s": pr64 / l64, "avg_launch_ms": l64 * 1e3}
            if not batched:  # mixed precision: FP32-bulk corrections, tolerance met on the FP64 operator
                for rtol in (tol, 1e-10):
                    sr = make("fp32")
                    _, _, ir = sr.solve_refined(rtol, 8, 400)
                    sr.close()
                    gm[f"refined_to_{rtol:g}_s"] = ir["solve_ms"] / 1e3
                    gm[f"refined_to_{rtol:g}_fp64_residual"] = ir["rel_residual"]
                gm["refined_speedup_vs_fp64_plain"] = gm["fp64_plain_s"] / gm[f"refined_to_{tol:g}_s"]
            if batched:
                p32, p64 = torch.cat(list(map(torch.as_tensor, p32))), torch.cat(list(map(torch.as_tensor, p64)))
                d32, d64 = torch.cat(list(map(torch.as_tensor, d32))), torch.cat(list(map(torch.as_tensor, d64)))
                E32, E64 = np.asarray(E32), np.asarray(E64)
            rel = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
            relmax = lambda a, b: float(torch.max(torch.abs(a - b)) / torch.max(torch.abs(b)))
            acc = {"phi_rel_l2_fp32_vs_fp64": rel(p32, p64), "dphi_rel_l2_fp32_vs_fp64": rel(d32, d64),
                   "phi_rel_max_fp32_vs_fp64": relmax(p32, p64), "dphi_rel_max_fp32_vs_fp64": relmax(d32, d64)}
            if batched:
                acc["E_rel_fp32_vs_fp64_max"] = float(np.max(np.abs(E32 - E64) / np.abs(E64)))
            else:
                acc.update(E_sol_fp32=E32, E_sol_fp64=E64, E_rel_fp32_vs_fp64=abs(E32 - E64) / abs(E64))
        # phases of one step, outside the timed region (CUDA events on the library's stream order)
        phases = step_phases(make, batched, tol, stream) if not batched else None
        # fast summation (treecode, beyond the paper) on the same inputs, outside the timed region:
        # far-field time per matvec and solve time against the direct FP32 path, and its deviation
        fast = None
        if not args.no_fast:
            if batched:
                fast = fast_summation_batch(hobi, mols, (Vd, Fd, Nd, Qd), e1, e2, ka, tol, stream, args.fast_degree,
                                            args.fast_theta)
            else:
                fast = fast_summation(hobi, (Vd, Fd, Nd, Qd), e1, e2, ka, tol, stream, args.fast_degree,
                                      args.fast_theta)
        # the paper's low-order scheme and the off-surface output on the same surface
        lobi = reaction = None
        if not batched and not args.no_extra:
            lobi = lobi_object(hobi, (Vd, Fd, Nd, Qd), e1, e2, ka, tol, stream, sms, fmax)
            reaction = reaction_object(hobi, (Vd, Fd, Nd, Qd), e1, e2, ka, tol, stream, sms, fmax)
        # end to end through the public API with host buffers, copies inside the timed region
        e2e_t, e2e_pairs = [], []
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            inf, _, prof, prof_e, _, _, _ = step(True, "fp32", host=True)
            e2e_t.append(time.perf_counter() - t0)
            e2e_pairs.append(prof["pairs"] + (energy_pairs if batched else prof_e["pairs"]))
        h2d = Vh.nbytes + Fh.nbytes + Nh.nbytes + Qh.nbytes
        d2h = 2 * Vh.shape[0] * 8 + 8 * len(mols)
        e2e = {"value": sum(e2e_pairs) / sum(e2e_t), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * sum(e2e_t) / len(e2e_t)}
        # CPU baseline: the oracle on a bounded sample of the same workload (rank 0, N = 1 only)
        cpu = None
        if ws == 1 and not args.no_cpu:
            big = max(range(len(mols)), key=lambda i: mols[i][1].shape[0])
            V, F, N, Q = mols[big]
            val, dt, pairs, cores = cpu_oracle_sample(V, F, N, Q, args.cpu_rows, cfg)
            val1, dt1, pairs1, _ = cpu_oracle_sample(V, F, N, Q, max(8, args.cpu_rows // 16), cfg, seed=1, threads=1)
            cpu = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": _cpu_model(),
                   "sample": f"{min(args.cpu_rows, V.shape[0])} of {V.shape[0]} matvec rows x {4 * F.shape[0]} "
                             f"nodes ({pairs:.3g} pairs, {dt:.1f} s)" + (f", molecule {big}" if batched else ""),
                   "value_1_thread": val1,
                   "sample_1_thread": f"{max(8, args.cpu_rows // 16)} rows ({pairs1:.3g} pairs, {dt1:.1f} s)",
                   # the oracle's time for the whole timed step at its measured rate (pairs / rate)
                   "step_s_extrapolated": pairs_per_step / val}
        # the larger benchmark workloads (outside the timed region)
        extra = None
        if args.workload == "c2l6" and not args.no_extra and ws == 1:
            extra = {}
            for name in args.extra.split(","):
                if name:
                    extra[name] = extra_workload(hobi, name, dev, stream, sms, fmax)
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(cfg, parallelism=f"replicas x{ws}" if ws > 1 else "single GPU",
                           l2="flushed between timed steps (256 MB write)",
                           pairs_per_step=pairs_per_step, gmres_iterations=iters[-1],
                           E_sol=(E.tolist() if batched else E)),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "gmres": gm, "fp64_roofline": fp64_roof, "accuracy": acc, "phases": phases, "fast_summation": fast,
            "lobi": lobi, "reaction_potential": reaction, "workloads": extra,
        }
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["c2l6", "c3", "c5", "c4"], default="c2l6")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-plain GMRES comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-fast", action="store_true", help="skip the fast-summation (treecode) comparison")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the LOBI-PB, off-surface potential and larger-workload objects")
    ap.add_argument("--extra", default="c5,c4", help="larger workloads measured after the default one")
    ap.add_argument("--fast-degree", type=int, default=5)
    ap.add_argument("--fast-theta", type=float, default=0.7)
    ap.add_argument("--cpu-rows", type=int, default=1024)
    ap.add_argument("--ref-rows", type=int, default=1024)
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
