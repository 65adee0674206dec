"""Benchmark of the FETI dual-operator hot path on one GB300 (per rank).

Default workload (3): 3D linear elasticity, Hex8, the unit cube cut into
8 x 8 x 8 = 512 subdomains of 12^3 elements (6591 DOFs each, m_i 1407..2814,
n_lambda = 664 800), E = 1, nu = 0.3, clamped at x = 0, body force (0, 0, -1):
the largest of the forward configurations (6.7 GB of FP32 F tiles).
`--workload 2|4|5` runs the other configurations (2: 2D lognormal heat, 1024
subdomains of 4225 DOFs; 4: uneven 3D heat; 5: the sensitivity
configuration, 8.0 GB of F tiles, with its adjoint timed).  Seeded synthetic
inputs; the paper's data are not used.

A step is one pass of the whole path, on the mixed-precision configuration
(FP64 Cholesky; FP32 pruned TRSM with split-bf16 tensor-core panel updates;
split-bf16 tensor-core SYRK into FP32 F_i tiles; FP64 coarse problem and PCPG
vectors; the FP64 residual recomputed with the implicit operator each time the
projected residual has dropped by 1e4, and to confirm convergence):
feti_assemble (regularise, Cholesky, TRSM, SYRK) followed by feti_solve
(projected PCG with the explicit apply, refinement, alpha, u).
`value` is the achieved GB/s of the explicit F.lambda apply inside the timed
steps: algorithmic bytes per apply / mean CUDA-event time of the F-streaming
kernel, recorded by the library on its stream.  The FP64 assembly and apply,
the F and solution differences between the two paths, the implicit-apply time
and the break-even iteration count are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload 2|3|4|5]
Under torchrun each rank runs an independent replica of the workload (the
single-GPU path has no exchange step: "replicas only", weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "F assembly ms & F·λ GB/s, mixed vs FP64 at stated error; break-even PCG iters"
WORKLOADS = {
    2: "2D heat Q1, 32x32 subdomains of 64x64 elements (4225 DOFs, m_i 129..258, n_lambda 130048), "
       "lognormal sigma=1, seed 0",
    3: "3D elasticity Hex8, 8x8x8 subdomains of 12^3 elements (6591 DOFs, n_lambda 664800), E=1, nu=0.3",
    4: "3D heat Hex8, 120^3 box cut into 10x10x10 uneven subdomains (8..24 elements per axis, seed 0), "
       "lognormal sigma=0.5",
    5: "3D elasticity Hex8, 6x6x6 subdomains of 16^3 elements (14739 DOFs, n_lambda 473832), rho~U[0.1,1], E=rho^3",
}
DEFAULT_WORKLOAD = 3
PREC = "split_bf16"
REFINE_DROP = 1e-4   # FP64 residual recomputed whenever ||P r|| has dropped by this factor
REFINE_RESTART = True  # the search direction restarts after each FP64 residual (refinement with inner CG)
TOL = 1e-10


def arm_config(workload, world):
    """The workload and settings both arms name (the same dict on the reference line)."""
    return {"workload": WORKLOADS[workload],
            "prec": f"{PREC} SYRK and TRSM panel updates, FP32 TRSM/F tiles, FP64 Cholesky/PCPG",
            "step": f"feti_assemble + feti_solve (tol {TOL}, FP64 residual after each {1 / REFINE_DROP:.0e} "
                    f"drop, CG direction restarted after it)",
            "value": "explicit F.lambda apply GB/s (algorithmic bytes / F-streaming kernel time)",
            "l2": "256 MB buffer written before each timed step; the F tiles of one apply exceed L2 (129 MB)",
            "parallelism": f"replicas x{world}"}


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


# GB300's nominal HBM3e bandwidth, reported beside the measured copy peak
HBM_NOMINAL_GBS = 7900.0

# Peaks of the SIMT pipes, derived from GB300's unit counts at the 2070 MHz maximum SM clock:
# FP64 1.25 TFLOP/s nominal (an FMA probe on this GPU measured 1.20), FP32 152 SMs x 128 FMA x 2 x 2.07 GHz.
FP64_PEAK_TFLOPS = 1.25
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def other_rooflines(st, impl_ms, hbm):
    """Rooflines of the assembly kernels and of the FP64 implicit operator (last assembly).  The flop counts
    are the symbolic phase's algorithmic counters (feti_stats): Cholesky sum_s (w^3/3 + w^2 r + w r^2),
    pruned TRSM sum_s J_s (w_s^2 + 2 w_s r_s) (triangular solve and panel update of the J_s columns that
    reach supernode s), SYRK sum_s w_s J_s (J_s + 1) (the lower triangle of each supernode block's Gram
    matrix; the split-bf16 tensor-core rate counts its 3 products)."""
    bf16, bf16_kind = bf16_peak()
    out = {}
    if st["t_chol_ms"] > 0:
        a = st["chol_flops"] / (st["t_chol_ms"] * 1e-3) / 1e12
        out["chol_kernel"] = {"bound": "alu", "achieved": a, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                              "frac": a / FP64_PEAK_TFLOPS, "peak_kind": "derived FP64",
                              "algorithmic_flops": st["chol_flops"], "ms": st["t_chol_ms"],
                              "tc_kernel_ms": st.get("t_chol_tc_ms", 0.0),
                              "note": "FP64 flops of the factorisation over both Cholesky kernels; the rank-32 and "
                                      "rank-128 updates of the fronts at least 384 wide run on the tensor cores "
                                      "(exact bf16 slicing, chol_tc_kernel), so frac is against the FP64 pipe only"}
    if st["t_trsm_ms"] > 0:
        a = st["trsm_flops"] / (st["t_trsm_ms"] * 1e-3) / 1e12
        out["trsm_kernel<float>"] = {"bound": "alu", "achieved": a, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                                     "frac": a / FP32_PEAK_TFLOPS, "peak_kind": "derived FP32",
                                     "algorithmic_flops": st["trsm_flops"], "ms": st["t_trsm_ms"]}
    if st["t_syrk_ms"] > 0:
        a = 3 * st["syrk_flops"] / (st["t_syrk_ms"] * 1e-3) / 1e12  # split-bf16: 3 tensor products per FMA
        out["syrk_tc_kernel"] = {"bound": "tensor", "achieved": a, "peak": bf16, "unit": "TFLOP/s",
                                 "frac": a / bf16, "peak_kind": f"{bf16_kind} bf16",
                                 "algorithmic_flops": st["syrk_flops"], "tensor_flops": 3 * st["syrk_flops"],
                                 "ms": st["t_syrk_ms"]}
    if impl_ms > 0:
        # FP64-pipe bound (ncu: FP64 pipe ~2/3 active, DRAM ~12%): 2 FMAs per factor entry, forward and back
        a = st["implicit_bytes"] / 4 / (impl_ms * 1e-3) / 1e12
        g = st["implicit_bytes"] / (impl_ms * 1e-3) / 1e9
        out["implicit_kernel<0>"] = {"bound": "alu", "achieved": a, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                     "frac": a / FP64_PEAK_TFLOPS, "peak_kind": "derived FP64",
                                     "algorithmic_flops": st["implicit_bytes"] / 4, "ms": impl_ms,
                                     "factor_gbs": g, "factor_gbs_frac_of_hbm": g / hbm}
    return out


# Variant index of the apply autotuner -> kernel name.
APPLY_KERNELS = ["apply_tiles_kernel<{t}, 4>", "apply_tiles_kernel<{t}, 8>", "apply_tiles_kernel<{t}, 16>",
                 "apply_ring_kernel<{t}, 4, 3>", "apply_ring_kernel<{t}, 8, 3>", "apply_ring_kernel<{t}, 2, 6>"]

# dram__bytes_read.sum + dram__bytes_write.sum per launch of the FP32 apply tile kernels (all variants read the
# stored F bytes once), from an ncu capture of the kernel as it stands: workload 2 at full size, workload 3 on
# its 4 x 4 x 4-subdomain copy (0.84 GB of tiles) scaled to the full 512 subdomains by the tile bytes (the
# traffic is the tiles plus per-tile vector segments, both proportional).  The summaries are in profiles/.
APPLY_TRAFFIC = {2: (138.71e6, "ncu, profiles/apply_tiles_workload2.md"),
                 3: (684.77e6 * 6750564216.0 / 678647544.0,
                     "ncu on the 64-subdomain copy scaled by algorithmic bytes, profiles/apply_tiles_workload3.md")}


def max_over_ranks(values, device):
    """Element-wise maximum of a list of per-rank timings over all ranks (a barrier follows), so that the
    job's throughput is the work of all ranks over the slowest rank's time.  One rank: returned as given."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return [float(x) for x in t.tolist()]


def oracle_threads():
    """Threads the oracle's BLAS runs on (threadpoolctl where it is installed, else the host's core count)."""
    try:
        from threadpoolctl import threadpool_info
        n = max((int(i.get("num_threads", 0)) for i in threadpool_info() if i.get("user_api") == "blas"),
                default=0)
        if n > 0:
            return n
    except Exception:
        pass
    return os.cpu_count()


def oracle_sample(P, nsample, reps, keep_F=False):
    """The FP64 CPU oracle on a bounded sample: dense F_i for nsample
    subdomains and reps dense F_i p_i sweeps over them.  With keep_F the
    oracle's F_i are returned as well (the bench compares the GPU's F_i of the
    same subdomains with them)."""
    from oracle import feti_oracle as O
    subs = P.subs[:nsample]
    t0 = time.perf_counter()
    Fs = [O.local_F(s) for s in subs]
    t_f = (time.perf_counter() - t0) / nsample
    ps = [np.random.default_rng(i).normal(size=s.m) for i, s in enumerate(subs)]
    t0 = time.perf_counter()
    for _ in range(reps):
        for F, p in zip(Fs, ps):
            F @ p
    t_ap = (time.perf_counter() - t0) / reps
    byts = sum(8.0 * s.m * s.m + 16.0 * s.m for s in subs)
    if keep_F:
        return byts / t_ap / 1e9, t_f, t_ap, Fs
    return byts / t_ap / 1e9, t_f, t_ap


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on the host cores."""
    from paper_2502_08382_gb300.problems import make_config
    P = make_config(args.workload)
    nsample = 4 if args.workload == 2 else 1
    for _ in range(args.warmup):
        oracle_sample(P, 1, 5)
    vals, tf = [], []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        g, t_f, t_ap = oracle_sample(P, nsample, 50)
        vals.append(g)
        tf.append(t_f)
    ms = (time.perf_counter() - t_all) * 1e3 / max(args.steps, 1)
    gbs = statistics.median(vals)
    sample = (f"{nsample} of {P.nsub} subdomains per step: scipy dense Cholesky F_i and 50 dense FP64 F_i p_i "
              f"sweeps; value = GB/s of the F_i p_i sweeps")
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": arm_config(args.workload, args.gpus),
            "assembly_ms_extrapolated": statistics.median(tf) * 1e3 * P.nsub,
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": oracle_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", type=int, default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS),
                    help="3 (default: the largest assembly/apply configuration), 2, 4 or 5")
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

    P = make_config(args.workload)
    sens = args.workload == 5  # the sensitivity workload: the adjoint is timed too
    op = feti.FetiOperator(P, prec=PREC, tol=TOL, maxit=5000, refine_drop=REFINE_DROP, refine_restart=REFINE_RESTART,
                           with_elements=sens)
    st = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2 (129 MB)

    def step():
        op.assemble()
        return op.solve()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    op.set_profiling(True)
    step_ms, asm, info = [], [], None
    torch.cuda.nvtx.range_push("feti_timed")  # lets a profiler select the timed steps only
    with Clocks(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            lam, alpha, u, info = step()
            b.record(st)
            b.synchronize()
            step_ms.append(a.elapsed_time(b))
            asm.append(op.stats()["t_assemble_ms"])
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    st_ = op.stats()
    op.set_profiling(False)
    # replicas: every rank did the same work; the job's rate is N x the work over the slowest rank's time
    tot, tiles_ms, apply_ms = max_over_ranks(
        [sum(step_ms), st_["apply_tiles_ms"] / max(st_["apply_calls"], 1), st_["apply_ms"] / max(st_["apply_calls"], 1)],
        "cuda")
    ms_per_step = tot / args.steps
    impl_ms = st_["implicit_ms"] / max(st_["implicit_calls"], 1)
    hbm, pk_kind = peaks()
    tiles_gbs = st_["apply_bytes"] / (tiles_ms * 1e-3) / 1e9
    kname = (APPLY_KERNELS[st_["apply_variant"]].format(t="float") if 0 <= st_["apply_variant"] < len(APPLY_KERNELS)
             else "apply")
    traffic, traffic_src = APPLY_TRAFFIC.get(args.workload, (None, "not captured"))
    value = tiles_gbs * world

    # end to end through the C ABI with host buffers: H2D p, feti_apply, D2H q
    p_host = torch.from_numpy(seeded_vector(P.n_lambda, 0)).pin_memory()
    q_host = torch.empty_like(p_host).pin_memory()
    p = torch.empty(P.n_lambda, dtype=torch.float64, device="cuda")
    q = torch.empty_like(p)
    for _ in range(3):
        p.copy_(p_host, non_blocking=True)
        op.apply(p, out=q)
        q_host.copy_(q, non_blocking=True)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    nrep = 50
    a.record(st)
    for _ in range(nrep):
        p.copy_(p_host, non_blocking=True)
        op.apply(p, out=q)
        q_host.copy_(q, non_blocking=True)
    b.record(st)
    b.synchronize()
    e2e_gbs = st_["apply_bytes"] / (a.elapsed_time(b) / nrep * 1e-3) / 1e9

    adjoint = None
    if sens:
        # dL/drho_e for L = sum_i <W_i, F_i> with seeded symmetric N(0, 1) W_i drawn on the device (timing only;
        # the tests check the adjoint against the oracle): the batched FP64 adjoint with X_i recomputed
        gen = torch.Generator(device="cuda")
        gen.manual_seed(3)
        Wd = torch.empty(sum(s.m * s.m for s in P.subs), dtype=torch.float64, device="cuda")
        off = 0
        for s_ in P.subs:
            A = torch.randn(s_.m, s_.m, generator=gen, dtype=torch.float64, device="cuda")
            Wd[off:off + s_.m * s_.m] = ((A + A.T) * 0.5 ** 0.5).reshape(-1)
            off += s_.m * s_.m
        op.assemble()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        g = op.adjoint(Wd)
        b.record(st)
        b.synchronize()
        adjoint = {"ms": a.elapsed_time(b), "elements": int(g.numel()),
                   "what": "feti_adjoint over all 216 subdomains (FP64 X_u recomputed, Z and Y by backward solves, "
                           "element contraction), one call"}
        del Wd, g

    # plain FP64 GPU path on the same inputs (assembly time, F and solution differences)
    op64 = feti.FetiOperator(P, prec="fp64", tol=TOL, maxit=5000)
    op64.assemble()
    asm64 = []
    for _ in range(2):
        flush.zero_()
        op64.assemble()
        asm64.append(op64.stats()["t_assemble_ms"])
    st64 = op64.stats()
    lam64, alpha64, u64, info64 = op64.solve()
    # the plain FP64 explicit apply (FP64 F tiles: twice the F bytes)
    op64.set_profiling(True)
    for _ in range(10):
        flush.zero_()
        op64.apply(p, out=q)
    st64a = op64.stats()
    op64.set_profiling(False)
    t64_tiles = st64a["apply_tiles_ms"] / max(st64a["apply_calls"], 1)
    t64_call = st64a["apply_ms"] / max(st64a["apply_calls"], 1)
    apply64 = {"algorithmic_bytes": st64a["apply_bytes"], "tiles_ms": t64_tiles, "ms": t64_call,
               "gbs": st64a["apply_bytes"] / (t64_tiles * 1e-3) / 1e9,
               "gbs_whole_call": st64a["apply_bytes"] / (t64_call * 1e-3) / 1e9,
               "kernel": (APPLY_KERNELS[st64a["apply_variant"]].format(t="double")
                          if 0 <= st64a["apply_variant"] < len(APPLY_KERNELS) else "apply"),
               "frac_of_hbm": st64a["apply_bytes"] / (t64_tiles * 1e-3) / 1e9 / hbm}
    sample = sorted({0, P.nsub // 3, (2 * P.nsub) // 3, P.nsub - 1})
    ferr = max(np.linalg.norm(op.get_F(i) - op64.get_F(i)) / np.linalg.norm(op64.get_F(i)) for i in sample)
    uerr = (torch.linalg.norm(u - u64) / torch.linalg.norm(u64)).item()
    p.copy_(p_host)
    op64.set_profiling(True)
    for _ in range(10):
        op64.apply_implicit(p, out=q)
    st64i = op64.stats()
    op64.set_profiling(False)
    impl64_ms = st64i["implicit_ms"] / max(st64i["implicit_calls"], 1)
    cpu_leg = rank == 0 and world == 1 and not args.no_cpu_baseline
    ns_cpu = 4 if args.workload == 2 else 1
    F64_sample = None
    if cpu_leg:
        try:
            F64_sample = [op64.get_F(i) for i in range(ns_cpu)]
        except Exception:  # the comparison is reported, never allowed to stop the bench
            F64_sample = None
    op64.close()
    t_asm = statistics.median(asm)
    st_last = op.stats()
    n_star = break_even(t_asm, apply_ms, st_last["t_chol_ms"], impl64_ms)

    line = {"metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": arm_config(args.workload, world),
            "F_tile_mb": st_["F_elems"] * 4 / 1e6,
            "assembly_ms": {"mixed": t_asm, "fp64": statistics.median(asm64),
                            "speedup": statistics.median(asm64) / t_asm,
                            "mixed_phases": {k: st_last[k] for k in ("t_chol_ms", "t_trsm_ms", "t_syrk_ms")},
                            "fp64_phases": {k: st64[k] for k in ("t_chol_ms", "t_trsm_ms", "t_syrk_ms")},
                            "coarse_once_ms": st_last["t_coarse_ms"]},
            "errors": {"F_rel_frobenius_mixed_vs_fp64": ferr, "u_rel_mixed_vs_fp64": uerr,
                       "F_fp64_vs_oracle": None, "F_mixed_vs_oracle": None,
                       "pcg_rel_residual": info["rel_residual"]},
            "pcg": {"iterations": info["iterations"], "refinements": info["refinements"],
                    "fp64_iterations": info64["iterations"]},
            "apply": {"ms": apply_ms, "tiles_ms": tiles_ms, "algorithmic_bytes": st_["apply_bytes"],
                      "autotuned": {"variant": st_["apply_variant"], "grid": st_["apply_grid"]},
                      "gbs_whole_call": st_["apply_bytes"] / (apply_ms * 1e-3) / 1e9,
                      "frac_whole_call": st_["apply_bytes"] / (apply_ms * 1e-3) / 1e9 / hbm},
            "apply_fp64": apply64,
            "implicit_fp64_apply_ms": impl64_ms,
            "break_even_iters": n_star,
            "roofline": {"bound": "hbm", "achieved": tiles_gbs, "peak": hbm, "unit": "GB/s",
                         "frac": tiles_gbs / hbm, "traffic": traffic, "traffic_source": traffic_src,
                         "kernel": kname, "peak_kind": pk_kind,
                         "frac_of_nominal": tiles_gbs / HBM_NOMINAL_GBS, "nominal_gbs": HBM_NOMINAL_GBS},
            "roofline_other": other_rooflines(st_last, impl64_ms, hbm),
            "e2e": {"value": e2e_gbs * world, "unit": "GB/s", "h2d_bytes_per_step": 8 * P.n_lambda,
                    "d2h_bytes_per_step": 8 * P.n_lambda},
            "gpu_launches": int(st_["launches"]),
            "adjoint": adjoint,
            "clocks": clk.summary()}
    if cpu_leg:
        gbs, t_f, t_ap, Fo = oracle_sample(P, ns_cpu, 300 if args.workload == 2 else 20, keep_F=True)
        # the CPU leg's oracle F_i of the same subdomains: relative Frobenius errors of both GPU paths
        try:
            rel = lambda A, i: float(np.linalg.norm(A - Fo[i]) / np.linalg.norm(Fo[i]))
            if F64_sample is not None:
                line["errors"]["F_fp64_vs_oracle"] = max(rel(F64_sample[i], i) for i in range(ns_cpu))
            line["errors"]["F_mixed_vs_oracle"] = max(rel(op.get_F(i), i) for i in range(ns_cpu))
            line["errors"]["F_vs_oracle_sample"] = f"subdomains 0..{ns_cpu - 1} (the CPU baseline's oracle F_i)"
        except Exception as exc:
            line["errors"]["F_vs_oracle_sample"] = f"not computed: {type(exc).__name__}"
        line["cpu_baseline"] = {"value": gbs, "unit": "GB/s", "cores": oracle_threads(), "kind": "oracle",
                                "sample": f"{ns_cpu} of {P.nsub} subdomains: scipy dense Cholesky F_i "
                                          f"({t_f * 1e3:.0f} ms each) and {300 if args.workload == 2 else 20} "
                                          f"dense FP64 F_i p_i sweeps",
                                "assembly_ms_extrapolated": t_f * 1e3 * P.nsub}
    if rank == 0:
        print(json.dumps(line))
    op.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
