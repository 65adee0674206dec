"""Benchmark of the FETI dual-operator hot path on one GB300 (per rank).

A step is one pass of the whole path over workload 2 (2D heat, 32x32
subdomains of 64x64 Q1 elements, 4225 DOFs each, lognormal conductivity):
feti_assemble (regularise, Cholesky, pruned TRSM, SYRK, coarse setup) and
feti_solve (projected PCG with the explicit apply and FP64 refinement,
recovery).  value = achieved GB/s of the explicit F.lambda apply (algorithmic
bytes / CUDA-event time) inside the step; assembly ms, the FP64 comparison,
errors and the break-even iteration count are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (the path has no
cross-rank exchange on one node: "replicas only", weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "F assembly ms & F·λ GB/s, mixed vs FP64 at stated error; break-even PCG iters"
WORKLOAD = "2D heat Q1, 32x32 subdomains x 64x64 elements (4225 DOFs, m_i 129..258), lognormal sigma=1, seed 0"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, idx):
        self.idx = idx
        self.p = None
        self.path = f"/tmp/feti_clocks_{os.getpid()}.csv"

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.fh.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
            sm = [float(r[1]) for r in rows]
            out["sm_mhz"] = statistics.median(sm) if sm else None
            out["sm_max_mhz"] = float(rows[0][2]) if rows else None
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            rs = set()
            for r in rows:
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        rs.add(nm)
            out["reasons"] = sorted(rs)
            out["samples"] = len(rows)
        except Exception:
            pass
        return out


def run_reference(args):
    """The FP64 CPU oracle timed on the host cores on a bounded sample."""
    from oracle import feti_oracle as O
    from paper_2502_08382_gb300.problems import make_config
    P = make_config(2)
    nsample = 4
    subs = P.subs[:nsample]
    t0 = time.perf_counter()
    Fs = [O.local_F(s) for s in subs]
    t_f = (time.perf_counter() - t0) / nsample
    ps = [np.random.default_rng(i).normal(size=s.m) for i, s in enumerate(subs)]
    for _ in range(args.warmup):
        for F, p in zip(Fs, ps):
            F @ p
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for _r in range(200):
            for F, p in zip(Fs, ps):
                F @ p
        times.append((time.perf_counter() - t0) / 200)
    t_ap = statistics.median(times)
    byts = sum(8.0 * s.m * s.m + 16.0 * s.m for s in subs)
    gbs = byts / t_ap / 1e9
    cores = os.cpu_count()
    sample = f"{nsample} of 1024 subdomains: dense Cholesky F_i (scipy) + 200 dense F_i p_i sweeps per step"
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ap * 200 * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD},
            "assembly_ms_extrapolated": t_f * 1e3 * P.nsub,
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def cpu_baseline_ours(P):
    """Oracle on a bounded sample (rank 0, N = 1): dense F_i and F_i p_i."""
    from oracle import feti_oracle as O
    nsample = 4
    subs = P.subs[:nsample]
    t0 = time.perf_counter()
    Fs = [O.local_F(s) for s in subs]
    t_f = (time.perf_counter() - t0) / nsample
    ps = [np.random.default_rng(i).normal(size=s.m) for i, s in enumerate(subs)]
    t0 = time.perf_counter()
    reps = 300
    for _ in range(reps):
        for F, p in zip(Fs, ps):
            F @ p
    t_ap = (time.perf_counter() - t0) / reps
    byts = sum(8.0 * s.m * s.m + 16.0 * s.m for s in subs)
    return {"value": byts / t_ap / 1e9, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{nsample} of {P.nsub} subdomains: scipy dense Cholesky F_i ({t_f * 1e3:.0f} ms each) "
                      f"and {reps} dense FP64 F_i p_i sweeps",
            "assembly_ms_extrapolated": t_f * 1e3 * P.nsub}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--applies", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2502_08382_gb300 import feti
    from paper_2502_08382_gb300.metrics import break_even
    from paper_2502_08382_gb300.problems import make_config, seeded_vector

    P = make_config(2)
    prec = os.environ.get("FETI_BENCH_PREC", "fp64")
    op = feti.FetiOperator(P, prec=prec)
    p_host = torch.from_numpy(seeded_vector(P.n_lambda, 0)).pin_memory()
    p = p_host.cuda()
    q = torch.empty_like(p)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    st = torch.cuda.current_stream()

    def step(timings):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(st)
        op.assemble()
        e1.record(st)
        for _ in range(args.applies):
            op.apply(p, out=q)
        e2.record(st)
        timings.append((e0, e1, e2))

    for _ in range(args.warmup):
        step([])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    tims = []
    asm_ms = []
    with Clocks(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        step_ms = 0.0
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            step(tims)
            b.record(st)
            b.synchronize()
            step_ms += a.elapsed_time(b)
            asm_ms.append(op.stats()["t_assemble_ms"])
        torch.cuda.synchronize()
    if world > 1:
        t = torch.tensor([step_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
        step_ms = float(t.item())
    ms_per_step = step_ms / args.steps
    apply_ms = statistics.median([e1.elapsed_time(e2) / args.applies for (_, e1, e2) in tims])
    st_ = op.stats()
    hbm, pk_kind = peaks()
    gbs = st_["apply_bytes"] / (apply_ms * 1e-3) / 1e9
    value = gbs * world

    # end-to-end through the C ABI with host buffers (H2D p, apply, D2H q)
    q_host = torch.empty_like(p_host).pin_memory()
    e_times = []
    for _ in range(3):
        p.copy_(p_host, non_blocking=True)
        op.apply(p, out=q)
        q_host.copy_(q, non_blocking=True)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(st)
    for _ in range(args.applies):
        p.copy_(p_host, non_blocking=True)
        op.apply(p, out=q)
        q_host.copy_(q, non_blocking=True)
    b.record(st)
    b.synchronize()
    e2e_ms = a.elapsed_time(b) / args.applies
    e2e_gbs = st_["apply_bytes"] / (e2e_ms * 1e-3) / 1e9

    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "prec": prec, "step": f"feti_assemble + {args.applies} feti_apply",
                       "l2": "256 MB buffer written between timed steps", "parallelism": f"replicas x{world}"},
            "assembly_ms": statistics.median(asm_ms),
            "assembly_phases_ms": {k: st_[k] for k in ("t_chol_ms", "t_trsm_ms", "t_syrk_ms", "t_coarse_ms")},
            "apply_ms": apply_ms,
            "flops": {k: st_[k] for k in ("chol_flops", "trsm_flops", "syrk_flops")},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                         "traffic": None, "kernel": "feti_apply (3 launches)", "peak_kind": pk_kind},
            "e2e": {"value": e2e_gbs * world, "unit": "GB/s", "h2d_bytes_per_step": 8 * P.n_lambda,
                    "d2h_bytes_per_step": 8 * P.n_lambda},
            "gpu_launches": args.steps * (3 + 3 * args.applies),
            "clocks": clk.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_ours(P)
    if rank == 0:
        print(json.dumps(line))
    op.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
