#!/usr/bin/env python3
"""Benchmark of the HOBI-PB hot path on GB300.

One step = the whole hot path on one synthetic molecule with its inputs resident
in HBM: hobi_setup (mesh validation, adjacency, curved-element nodes, singular
correction table, right-hand side), hobi_solve (GMRES to 1e-6: per iteration
gather + far-field pair sum + correction/diagonal + FP64 Arnoldi/Givens) and
hobi_energy. Workload: Kirkwood sphere of radius 10 A, icosphere level 6
(81,920 curved triangles, 40,962 vertices, 327,680 quadrature nodes), 10 seeded
charges uniform in a radius-8 ball, eps1 = 1, eps2 = 80, kappa = 0.1257 1/A;
FP32-bulk far field.

value = far-field pair evaluations per second over the whole step (all ranks).
With --gpus N > 1 (torchrun) every rank solves its own replica (no collective on
the data path): weak scaling.

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
WORKLOAD = {
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
OPS_PER_PAIR = 36  # FP32 FMA-pipe instructions per pair in the both-rows far-field kernel
MUFU_PER_PAIR = 2  # rsqrt.approx + ex2.approx
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "farfield32_c2_ico6_traffic.txt")
FARFIELD_SRC = [os.path.join(ROOT, "paper_1301_5914_gb300", "csrc", f) for f in ("k_farfield.cu", "ff_body.cuh")]


def _inputs():
    from paper_1301_5914_gb300 import synth

    V, F, N = synth.icosphere(6, 10.0)
    Q = synth.ball_charges(10, 8.0, 2)
    return V, F, N, Q


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


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


def cpu_oracle_sample(V, F, N, Q, rows: int, seed: int = 0):
    """Time the FP64 oracle's matvec on `rows` sampled rows of the workload (bounded CPU work)."""
    import numpy as np

    import oracle

    prob = oracle.Problem(V, F, N, Q, WORKLOAD["eps1"], WORKLOAD["eps2"], WORKLOAD["kappa"])
    rng = np.random.default_rng(seed)
    u = rng.normal(size=2 * prob.nv)
    sel = np.sort(rng.choice(prob.nv, size=rows, replace=False))
    t0 = time.perf_counter()
    prob.matvec_rows(u, sel)
    dt = time.perf_counter() - t0
    pairs = rows * 4.0 * prob.nf
    return pairs / dt, dt, pairs, oracle.num_threads()


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
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{rows} of {V.shape[0]} matvec rows x {4 * F.shape[0]} nodes per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    from paper_1301_5914_gb300 import hobi

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    V, F, N, Q = _inputs()
    e1, e2, ka, tol = WORKLOAD["eps1"], WORKLOAD["eps2"], WORKLOAD["kappa"], WORKLOAD["gmres_tol"]
    Vd = torch.as_tensor(V, device=dev)
    Fd = torch.as_tensor(F, dtype=torch.int32, device=dev)
    Nd = torch.as_tensor(N, device=dev)
    Qd = torch.as_tensor(Q, device=dev)
    nv, nn, nc = V.shape[0], 4 * F.shape[0], Q.shape[0]
    stream = torch.cuda.current_stream(dev)

    def step(profile: bool):
        s = hobi.Solver(Vd, Fd, Nd, Qd, e1, e2, ka, precision="fp32", stream=stream)
        if profile:
            s.profile_enable(True)
        phi, dphi, info = s.solve(tol, 200)
        E = s.energy()
        prof = s.profile_read() if profile else None
        n_launch = s.kernel_launches()
        s.close()
        return info, E, prof, n_launch, phi, dphi

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
        info, E, prof, nl, phi32, dphi32 = step(True)
        ev1.record(stream)
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1))
        ff_ms += prof["farfield_ms"]
        ff_launch += prof["launches"]
        ff_pairs += prof["pairs"]
        pairs_step.append(prof["pairs"])
        launches += nl
        iters.append(info["iterations"])
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    total_ms = sum(times)
    per_rank = [total_ms]
    if ws > 1:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        gathered = [torch.zeros_like(t) for _ in range(ws)]
        torch.distributed.all_gather(gathered, t)
        per_rank = [float(g.item()) for g in gathered]
    pairs_per_step = statistics.mean(pairs_step)
    value, ms_per_step = aggregate(per_rank, pairs_per_step, args.steps)

    out = None
    if rank == 0:
        # roofline of the dominant kernel (far field, FP32 bulk, both rows), live CUDA-event timing
        props = torch.cuda.get_device_properties(dev)
        sms = props.multi_processor_count
        try:
            peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
            fmax = float(peaks.get("sm_max_mhz", 2070.0))
            peak_src = "MEASURED_PEAKS.json sm_max_mhz"
        except (OSError, ValueError):
            fmax, peak_src = 2070.0, "nominal max SM clock"
        peak = sms * 128 * fmax * 1e6 / 1e9  # Ginst/s, FP32 FMA-pipe lanes
        avg_launch_s = ff_ms / ff_launch / 1e3
        pairs_per_launch = ff_pairs / ff_launch
        achieved = pairs_per_launch * OPS_PER_PAIR / avg_launch_s / 1e9
        traffic = _traffic_per_launch()
        fobs = clk.get("sm_mhz") or fmax
        roof = {
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Ginst/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": "k_farfield32<ROW2=true>",
            "algorithmic": f"{OPS_PER_PAIR} FP32 FMA-pipe instructions + {MUFU_PER_PAIR} MUFU per pair",
            "peak_basis": f"{sms} SMs x 128 FP32 lanes x {fmax:.0f} MHz ({peak_src})",
            "pairs_per_s": pairs_per_launch / avg_launch_s,
            "avg_launch_ms": avg_launch_s * 1e3,
            "frac_at_median_clock": achieved / (sms * 128 * fobs * 1e6 / 1e9),
            "mufu_frac": pairs_per_launch * MUFU_PER_PAIR / avg_launch_s / (sms * 16 * fmax * 1e6),
            "farfield_share_of_step": ff_ms / total_ms,
        }
        # FP64 plain path on the same inputs (outside the timed region): GMRES time to 1e-6
        gm = {"fp32_bulk_s": None, "fp64_plain_s": None}
        acc = {}
        if not args.no_fp64:
            s64 = hobi.Solver(Vd, Fd, Nd, Qd, e1, e2, ka, precision="fp64", stream=stream)
            p64, d64, i64 = s64.solve(tol, 200)
            E64 = s64.energy()
            s64.close()
            s32 = hobi.Solver(Vd, Fd, Nd, Qd, e1, e2, ka, precision="fp32", stream=stream)
            p32, d32, i32 = s32.solve(tol, 200)
            E32 = s32.energy()
            s32.close()
            gm = {"fp32_bulk_s": i32["solve_ms"] / 1e3, "fp64_plain_s": i64["solve_ms"] / 1e3,
                  "iterations_fp32": i32["iterations"], "iterations_fp64": i64["iterations"],
                  "speedup": i64["solve_ms"] / i32["solve_ms"]}
            rel = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
            acc = {"phi_rel_l2_fp32_vs_fp64": rel(p32, p64), "dphi_rel_l2_fp32_vs_fp64": rel(d32, d64),
                   "E_sol_fp32": E32, "E_sol_fp64": E64, "E_rel_fp32_vs_fp64": abs(E32 - E64) / abs(E64)}
            try:
                from oracle import kirkwood as kw

                e_ex = kw.solvation_energy(Q, 10.0, e1, e2, ka)
                acc["E_sol_kirkwood"] = e_ex
                acc["E_rel_fp64_vs_kirkwood"] = abs(E64 - e_ex) / abs(e_ex)
            except ImportError:
                pass
        # end to end through the public API with host buffers (pinned), copies inside the timed region
        Vh = torch.as_tensor(V).pin_memory()
        Fh = torch.as_tensor(F, dtype=torch.int32).pin_memory()
        Nh = torch.as_tensor(N).pin_memory()
        Qh = torch.as_tensor(Q).pin_memory()
        e2e_t, e2e_pairs = [], []
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s = hobi.Solver(Vh, Fh, Nh, Qh, e1, e2, ka, precision="fp32")
            _, _, inf = s.solve(tol, 200)
            s.energy()
            s.close()
            e2e_t.append(time.perf_counter() - t0)
            e2e_pairs.append(inf["iterations"] * nv * nn + nc * nn)
        h2d = V.nbytes + F.astype("int32").nbytes + N.nbytes + Q.nbytes
        d2h = 2 * nv * 8 + 8
        e2e = {"value": sum(e2e_pairs) / sum(e2e_t), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * sum(e2e_t) / len(e2e_t)}
        # CPU baseline: the oracle on a bounded sample of the same workload (rank 0, N = 1 only)
        cpu = None
        if ws == 1 and not args.no_cpu:
            val, dt, pairs, cores = cpu_oracle_sample(V, F, N, Q, args.cpu_rows)
            cpu = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{args.cpu_rows} of {nv} matvec rows x {nn} nodes ({pairs:.3g} pairs, {dt:.1f} s)"}
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(WORKLOAD, parallelism=f"replicas x{ws}" if ws > 1 else "single GPU",
                           l2="flushed between timed steps (256 MB write)",
                           pairs_per_step=pairs_per_step, gmres_iterations=iters[-1], E_sol=E),
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "gmres": gm, "accuracy": acc,
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
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-plain GMRES comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-rows", type=int, default=1024)
    ap.add_argument("--ref-rows", type=int, default=1024)
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
