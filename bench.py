#!/usr/bin/env python
"""Benchmark of the persistent-kernel (PERKS) hot path on GB300.

Workload (one bench step): 3d7pt Jacobi, 384^3 interior cells, fp64, 1000 time
steps, centre 0.4 / neighbours 0.1, Dirichlet 0, field uniform[0,1) from a
seed -- one persistent cooperative launch per bench step.  The field (2 x 453
MB) is larger than L2 (129 MB), so no L2 flush is needed between timed steps.

Printed: ONE JSON line (rank 0) with the contract keys, plus
  roofline      dominant kernel's achieved algorithmic GB/s vs measured HBM peak;
  cpu_baseline  the CPU oracle timed on a bounded sample of the same workload;
  e2e           the same metric through the C ABI with host buffers (H2D + D2H
                inside the timed region);
  variants      other configurations of the stencil workload and the CG leg
                (n = 2^20 synthetic SPD CSR matrix, rtol 1e-10) for context.

``--impl reference`` times the CPU oracle instead (the slow reference arm).
Multi-GPU (torchrun): every rank runs an independent replica (the workload
does not shard; no collective on the data path), value = all ranks' cell
updates / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stencil GCell-updates/s vs HBM roofline; CG ms to 1e-8 resid (plain vs learned)"
UNIT = "GCell-updates/s"
L_3D = 384
STEPS_3D = 1000


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _loop(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([s.strip() for s in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._loop, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for i, n in enumerate(names):
                if len(s) > 5 + i and s[5 + i].strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(world, v):
    """The largest of the ranks' values (each rank times its own replica; the
    job takes as long as the slowest)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, units_per_rank, total_ms):
    """Whole-job throughput of `world` independent replicas: all ranks' units
    over the slowest rank's time (units per second)."""
    return world * units_per_rank / (total_ms * 1e-3)


def stencil_leg(api, torch, ctx, L, steps, dtype, variant, K, W, seed=1, tune=True, keep_result=False):
    """Times K runs of `steps` Jacobi steps (plan chosen by the autotuner for
    this variant first); returns dict with per-run ms (and the field after
    the last run, as float64 on the device, when keep_result)."""
    from paper_2204_02064_gb300 import inputs
    shape = (L, L, L)
    f = torch.from_numpy(inputs.stencil_field(shape, seed)).to(
        {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dtype]).cuda()
    st = api.Stencil(ctx, shape, inputs.shape_offsets("3d7pt"), inputs.workload_weights("3d7pt"),
                     dtype=dtype)
    tuned = None
    if tune:
        st.set_field(f)
        tuned = st.autotune(variant, probe_steps=10)
    desc = st.describe(steps, variant)
    stream = torch.cuda.current_stream()
    for _ in range(W):
        st.set_field(f)
        st.run(steps, variant)
    torch.cuda.synchronize()
    times = []
    for _ in range(K):
        st.set_field(f)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st.run(steps, variant)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    st.check()
    result = None
    if keep_result:
        out = torch.empty_like(f)
        st.get_field(out)
        result = out.double()
    st.close()
    return {"ms": times, "desc": desc, "cells": L ** 3, "plan": tuned, "result": result}


def field_error(torch, got, ref):
    """Error of a field against a reference field (both float64 on the
    device): max |g - r| / max |r|, and the normwise-per-element error of the
    parity tests, max |g - r| / max(|r|, 1e-3 max |r|)."""
    d = (got - ref).abs()
    m = ref.abs().max()
    floor = torch.clamp(ref.abs(), min=1e-3 * float(m))
    return {"max_rel_to_max": float(d.max() / m), "normwise": float((d / floor).max())}


def kernel_name(desc):
    return {1: "resident", 2: "streaming", 3: "per_step"}.get(desc.get("kernel"), "unknown")


def stencil2d_leg(api, torch, ctx, L, steps, variant, K, W):
    from paper_2204_02064_gb300 import inputs
    f = torch.from_numpy(inputs.stencil_field((L, L), inputs.SEED_2D)).cuda()
    st = api.Stencil(ctx, (L, L), inputs.shape_offsets("2d5pt"), inputs.workload_weights("2d5pt"))
    st.set_field(f)
    plan = st.autotune(variant, probe_steps=20)
    kernel = kernel_name(st.describe(steps, variant))
    stream = torch.cuda.current_stream()
    for _ in range(W):
        st.set_field(f)
        st.run(steps, variant)
    times = []
    for _ in range(K):
        st.set_field(f)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st.run(steps, variant)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    st.check()
    st.close()
    return {"ms": times, "plan": plan, "kernel": kernel}


def e2e_leg(api, torch, ctx, L, steps, K, W):
    """Host-buffer end-to-end: pinned H2D + persistent run + D2H, per step."""
    from paper_2204_02064_gb300 import inputs
    shape = (L, L, L)
    host_in = torch.from_numpy(inputs.stencil_field(shape, 1)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    st = api.Stencil(ctx, shape, inputs.shape_offsets("3d7pt"), inputs.workload_weights("3d7pt"))
    stream = torch.cuda.current_stream()
    st.set_field(host_in, stream)
    st.autotune(0, probe_steps=10)
    for _ in range(W):
        st.set_field(host_in, stream)
        st.run(steps, 0, stream)
        st.get_field(host_out, stream)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        st.set_field(host_in, stream)
        st.run(steps, 0, stream)
        st.get_field(host_out, stream)
    e1.record(stream)
    e1.synchronize()
    st.check()
    ms = e0.elapsed_time(e1) / K
    nbytes = host_in.numel() * 8
    st.close()
    return ms, nbytes, nbytes


def cg_leg(api, torch, ctx, K):
    from paper_2204_02064_gb300 import inputs
    n = 1 << 20
    rp, c, v = inputs.csr_spd_matrix(n, inputs.SEED_CG)
    b = torch.from_numpy(inputs.cg_rhs(n, inputs.SEED_CG)).cuda()
    op = api.CsrOperator(ctx, torch.from_numpy(rp).cuda(), torch.from_numpy(c).cuda(),
                         torch.from_numpy(v).cuda())
    out = {"n": n, "nnz": int(c.shape[0]), "rtol": 1e-10}
    stream = torch.cuda.current_stream()
    legs = [(api.CG_FP64, "fp64", api.SPMV_ROWVEC, 1e-10), (api.CG_FP32_IR, "fp32_ir", api.SPMV_ROWVEC, 1e-10),
            (api.CG_FP64_MULTI, "fp64_multi_launch", api.SPMV_ROWVEC, 1e-10),
            (api.CG_FP64, "fp64_seg", api.SPMV_SEG, 1e-10), (api.CG_FP32_IR, "fp32_ir_seg", api.SPMV_SEG, 1e-10),
            (api.CG_FP64, "fp64_rtol1e-8", api.SPMV_ROWVEC, 1e-8), (api.CG_FP32_IR, "fp32_ir_rtol1e-8", api.SPMV_ROWVEC, 1e-8)]
    for mode, name, kind, rtol in legs:
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        try:
            t0 = time.perf_counter()
            op.set_spmv(kind)
            setup_s = time.perf_counter() - t0
            op.solve(b, x, rtol=rtol, mode=mode)     # warm-up
            times, stats = [], None
            for _ in range(K if kind != api.SPMV_SEG else min(K, 3)):
                x.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                op.solve(b, x, rtol=rtol, mode=mode, stats=False)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
                stats = op.last_result()
            med = statistics.median(times)
            out[name] = {"ms_to_tol": med, "ms_min": min(times), "ms_max": max(times),
                         "ms_stdev": statistics.stdev(times) if len(times) > 1 else 0.0, "runs": len(times),
                         "rtol": rtol, "iters": stats["iterations"], "spmv": kind,
                         "set_spmv_s": setup_s,
                         "outer": stats["outer_iterations"],
                         "true_rel_residual": stats["true_rel_residual"],
                         "sustained_gbs": stats["bytes_per_iteration"] * stats["iterations"]
                         / (med * 1e-3) / 1e9}
        except Exception as e:  # report, do not hide
            out[name] = {"error": str(e)}
    # the SpMV alone, against the rate at which this GPU serves random 8-byte
    # gathers from an L2-resident vector (its ceiling for a matrix whose
    # columns are scattered uniformly) and against HBM for its bytes
    try:
        op.set_spmv(api.SPMV_ROWVEC)
        xv = torch.rand(n, dtype=torch.float64, device="cuda")
        yv = torch.empty_like(xv)
        op.spmv(xv, yv)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(20):
            op.spmv(xv, yv)
        e1.record(stream)
        e1.synchronize()
        spmv_ms = e0.elapsed_time(e1) / 20
        g = ctx.gather_benchmark(20, 2000)
        g4 = ctx.gather_benchmark(20, 2000, elem_bytes=4)
        nnz = int(c.shape[0])
        hbm_bytes = 12.0 * nnz + 4.0 * (n + 1) + 16.0 * n
        out["spmv_alone"] = {"ms": spmv_ms, "gathers_per_s": g, "gathers_per_s_4byte": g4,
                             "gather_bound_ms": nnz / g * 1e3,
                             "frac_of_gather_bound": nnz / g * 1e3 / spmv_ms,
                             "hbm_bound_ms": hbm_bytes / (_peaks()[0] * 1e9) * 1e3,
                             "frac_of_hbm_bound": hbm_bytes / (_peaks()[0] * 1e9) * 1e3 / spmv_ms}
    except Exception as e:
        out["spmv_alone"] = {"error": str(e)}
    op.close()
    return out


def batch_leg(api, torch, ctx, K):
    """The batched workload: 64 uneven 2-D domains (sides 128..2048, 3x3 box
    1/9 and 5x5 box seeded weights), fp32, 500 steps in one persistent launch
    after the autotuner picked the plan; the per-domain per-step baseline
    beside it."""
    from paper_2204_02064_gb300 import inputs
    doms = inputs.batch_domains()
    b = api.Batch(ctx, doms, dtype="f32")
    fields = [torch.from_numpy(inputs.stencil_field(d["shape"], d["seed"])).float().cuda() for d in doms]
    cells = float(sum(d["shape"][0] * d["shape"][1] for d in doms))
    t0 = time.perf_counter()
    tuned = b.autotune(5)
    tune_s = time.perf_counter() - t0
    out = {"domains": len(doms), "cells": cells, "steps": 500, "autotune_s": tune_s,
           "plan": {k: tuned.get(k) for k in ("granularity", "width_cap", "grid_blocks", "tiles")}}
    stream = torch.cuda.current_stream()
    for variant, name in ((api.PERSISTENT, "persistent"), (api.PER_STEP, "per_step")):
        times = []
        for i in range(K + 1):
            for j, f in enumerate(fields):
                b.set_field(j, f)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run(500, variant=variant)
            e1.record(stream)
            e1.synchronize()
            if i > 0:
                times.append(e0.elapsed_time(e1))
        ms = min(times)
        out[name] = {"ms": ms, "gcells": cells * 500 / (ms * 1e-3) / 1e9}
    b.close()
    # the honest alternative: the 64 domains back to back, each through the
    # single-domain persistent path with its own autotuned plan
    sts = []
    for j, d in enumerate(doms):
        st = api.Stencil(ctx, d["shape"], d["offsets"], d["weights"], dtype="f32")
        st.set_field(fields[j])
        st.autotune(api.PERSISTENT, probe_steps=10)
        sts.append(st)
    times = []
    for i in range(K + 1):
        for j, st in enumerate(sts):
            st.set_field(fields[j])
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for st in sts:
            st.run(500)
        e1.record(stream)
        e1.synchronize()
        if i > 0:
            times.append(e0.elapsed_time(e1))
    for st in sts:
        st.check()
        st.close()
    ms = min(times)
    out["sequential_persistent"] = {"ms": ms, "gcells": cells * 500 / (ms * 1e-3) / 1e9}
    return out


def warmstart_leg(api, torch, ctx, ntrain=10000, nprob=256, n=512, epochs=8, batch=16, lr=1e-3,
                  label_rtol=1e-6, max_iter=100000, pool=4, reps=2):
    """The variable-coefficient Poisson workload: 256 problems on 512^2
    grids, k = exp(GRF, length 32, sigma 1), f uniform[-1,1), Dirichlet 0;
    CG to 1e-8 from zero vs from the BF16 warm-start network (inference
    included), the network trained on `ntrain` pairs generated by the same
    batched CG (labels solved to label_rtol)."""
    from paper_2204_02064_gb300 import inputs
    stream = torch.cuda.current_stream()
    out = {"n": n, "problems": nprob, "rtol": 1e-8, "train_pairs": ntrain, "epochs": epochs, "batch": batch,
           "label_rtol": label_rtol, "pool": pool}
    # training pairs, generated and solved in chunks of nprob problems
    t0 = time.perf_counter()
    ks, fs, us = [], [], []
    chunk_iters = []
    for c0 in range(0, ntrain, nprob):
        m = min(nprob, ntrain - c0)
        k, f = inputs.poisson_problems_device(n, m, seed=inputs.substream(inputs.SEED_POISSON, 500 + c0))
        P = api.Poisson(ctx, k)
        u = torch.zeros_like(f)
        r = P.solve(f, u, rtol=label_rtol, max_iter=max_iter)
        chunk_iters.append(r["mean_iterations"])
        print(f"warmstart: pairs {c0 + m}/{ntrain} solved, mean iterations {r['mean_iterations']:.0f}, "
              f"{time.perf_counter() - t0:.0f} s", file=sys.stderr, flush=True)
        P.close()
        ks.append(k)
        fs.append(f)
        us.append(u)
    k_tr, f_tr, u_tr = torch.cat(ks), torch.cat(fs), torch.cat(us)
    del ks, fs, us
    torch.cuda.synchronize()
    out["generate_s"] = time.perf_counter() - t0
    out["generate_mean_iterations"] = float(np.mean(chunk_iters))
    net = api.WarmNet(ctx, storage=api.BF16, seed=7, pool=pool)
    t0 = time.perf_counter()
    losses = net.fit(k_tr, f_tr, u_tr, batch=batch, epochs=epochs, lr=lr)
    torch.cuda.synchronize()
    out["train_s"] = time.perf_counter() - t0
    out["epoch_loss"] = [float(v) for v in losses]
    out["scale"] = net.scale
    del k_tr, f_tr, u_tr
    torch.cuda.empty_cache()
    # held-out evaluation problems
    k, f = inputs.poisson_problems_device(n, nprob, seed=inputs.SEED_POISSON)
    P = api.Poisson(ctx, k)
    x = torch.zeros_like(f)
    u0 = torch.zeros_like(f)
    res = {"zero": {"ms_runs": []}, "warm": {"ms_runs": [], "inference_ms": []}}
    for rep in range(reps):  # alternate the two starts
        for name in ("zero", "warm") if rep % 2 == 0 else ("warm", "zero"):
            x.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            ei = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if name == "warm":
                net.predict(k, f, x)
            ei.record(stream)
            P.solve(f, x, rtol=1e-8, max_iter=max_iter, stats=False)
            e1.record(stream)
            e1.synchronize()
            res[name]["ms_runs"].append(e0.elapsed_time(e1))
            if name == "warm":
                res[name]["inference_ms"].append(e0.elapsed_time(ei))
    for name in ("zero", "warm"):
        # the same solve again for the per-problem statistics (untimed)
        x.zero_()
        if name == "warm":
            net.predict(k, f, x)
        stats = P.solve(f, x, rtol=1e-8, max_iter=max_iter)
        runs = res[name]["ms_runs"]
        res[name].update({"ms_to_tol": statistics.median(runs), "ms_min": min(runs), "ms_max": max(runs),
                          "mean_iterations": stats["mean_iterations"],
                          "max_iterations": stats["max_iterations"],
                          "max_true_rel_residual": stats["max_true_rel_residual"]})
    res["warm"]["inference_ms"] = min(res["warm"]["inference_ms"])
    out.update(res)
    out["speedup"] = res["zero"]["ms_to_tol"] / res["warm"]["ms_to_tol"]
    # the gain counts only if it exceeds the run-to-run spread of either start
    out["spread_ms"] = max(res["zero"]["ms_max"] - res["zero"]["ms_min"], res["warm"]["ms_max"] - res["warm"]["ms_min"])
    out["gain_ms"] = res["zero"]["ms_to_tol"] - res["warm"]["ms_to_tol"]
    P.close()
    net.close()
    return out


def cpu_baseline_sample(max_seconds=15.0):
    """The oracle on a bounded sample of the workload: the 384^3 3d7pt field
    for as many whole steps as fit in ~max_seconds (at least one), timed
    single-threaded and, from the OpenMP build of the same source (identical
    results), on every host core.  The all-cores figure is the line's
    value."""
    from oracle import oracle
    from paper_2204_02064_gb300 import inputs
    f = inputs.stencil_field((L_3D, L_3D, L_3D), 1)
    offs = inputs.shape_offsets("3d7pt")
    w = inputs.workload_weights("3d7pt")
    t0 = time.perf_counter()
    oracle.stencil_run(f, offs, w, 1)
    t1 = time.perf_counter() - t0
    steps = max(1, min(int(max_seconds / max(t1, 1e-3)), 20))
    t0 = time.perf_counter()
    oracle.stencil_run(f, offs, w, steps)
    dt = time.perf_counter() - t0
    single = f.size * steps / dt / 1e9
    oracle.stencil_run_all_cores(f, offs, w, 1)           # builds the OpenMP library, warms the threads
    t0 = time.perf_counter()
    _, threads = oracle.stencil_run_all_cores(f, offs, w, steps)
    dt = time.perf_counter() - t0
    return {"value": f.size * steps / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"3d7pt fp64 {L_3D}^3 for {steps} steps (of {STEPS_3D}); the oracle's C built with "
                      f"OpenMP, planes of a step on {threads} host threads",
            "single_thread": {"value": single, "cores": 1}}


def run_reference(args):
    world, rank, local = _dist()
    if rank != 0:
        return 0
    from oracle import oracle
    from paper_2204_02064_gb300 import inputs
    f = inputs.stencil_field((L_3D, L_3D, L_3D), 1)
    offs = inputs.shape_offsets("3d7pt")
    w = inputs.workload_weights("3d7pt")
    for _ in range(args.warmup):
        oracle.stencil_run(f, offs, w, 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.stencil_run(f, offs, w, 1)
        times.append(time.perf_counter() - t0)
    dt = sum(times)
    value = f.size * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"3d7pt Jacobi {L_3D}^3 fp64, Dirichlet 0; CPU oracle, "
                                   f"each step one Jacobi step of the {STEPS_3D}-step workload",
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"one Jacobi step of {L_3D}^3 per bench step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-variants", action="store_true", help="only the headline workload")
    ap.add_argument("--profile", default=None,
                    help="run one small case for ncu and exit: headline, stencil3d-f64, "
                         "stencil3d-f32, stencil3d-bf16, stencil3d-f64-perstep, "
                         "stencil3d-f32-perstep, stencil384-*, stencil192-* (default plan: the resident "
                         "tile for fp32 / bf16), cg-fp64, cg-fp32ir, warmnet-tc, "
                         "batch64, poisson")
    ap.add_argument("--leg", default=None, choices=["warmstart", "cg"],
                    help="run one workload alone and print its JSON (warmstart: the learned "
                         "warm start for the 512^2 x 256 Poisson problems; cg: the n = 2^20 CG legs "
                         "and the SpMV against its gather and HBM bounds)")
    ap.add_argument("--ws-train", type=int, default=10000, help="warm start: training pairs")
    ap.add_argument("--ws-epochs", type=int, default=8, help="warm start: training epochs")
    ap.add_argument("--ws-pool", type=int, default=8, help="warm start: network grid coarsening factor")
    ap.add_argument("--ws-label-rtol", type=float, default=1e-6, help="warm start: label solve tolerance (--leg)")
    ap.add_argument("--ws-reps", type=int, default=2, help="warm start: alternated timed solves per start (--leg)")
    ap.add_argument("--ws-train-default", type=int, default=2048,
                    help="warm start inside the default run: training pairs (bounded so the run ends in minutes)")
    ap.add_argument("--no-warmstart", action="store_true", help="skip the warm-start leg of the default run")
    args = ap.parse_args()
    if args.leg == "warmstart":
        import torch
        from paper_2204_02064_gb300 import api
        ctx = api.Context(0)
        print(json.dumps({"leg": "warmstart", **warmstart_leg(api, torch, ctx, ntrain=args.ws_train,
                                                                epochs=args.ws_epochs, pool=args.ws_pool,
                                                                label_rtol=args.ws_label_rtol,
                                                                reps=args.ws_reps)}),
              flush=True)
        return 0
    if args.leg == "cg":
        import torch
        from paper_2204_02064_gb300 import api
        ctx = api.Context(0)
        print(json.dumps({"leg": "cg", **cg_leg(api, torch, ctx, 10)}), flush=True)
        return 0
    if args.profile:
        return profile_case(args.profile)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    world, rank, local = _dist()
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2204_02064_gb300 import api
    ctx = api.Context(local)
    info = ctx.info()
    peak, peak_kind = _peaks()

    # ---- headline: persistent 3d7pt 384^3 fp64, 1000 steps per bench step
    from paper_2204_02064_gb300 import inputs
    shape = (L_3D, L_3D, L_3D)
    f = torch.from_numpy(inputs.stencil_field(shape, 1)).cuda()
    st = api.Stencil(ctx, shape, inputs.shape_offsets("3d7pt"), inputs.workload_weights("3d7pt"))
    st.set_field(f)
    tuned = st.autotune(api.PERSISTENT, probe_steps=10)
    desc = st.describe(STEPS_3D, api.PERSISTENT)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        st.set_field(f)
        st.run(STEPS_3D)
    torch.cuda.synchronize()
    st.set_field(f)
    per_run = []
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        _barrier(world)
        torch.cuda.synchronize()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            evs[i][0].record(stream)
            st.run(STEPS_3D)
            evs[i][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
        _barrier(world)
    st.check()
    total_ms = t_start.elapsed_time(t_end)
    per_run = [a.elapsed_time(b) for a, b in evs]
    total_ms = _max_over_ranks(world, total_ms)
    cells = float(L_3D ** 3) * STEPS_3D
    value = replica_throughput(world, cells * args.steps, total_ms) / 1e9
    mean_launch_ms = sum(per_run) / len(per_run)
    achieved = desc["algorithmic_bytes"] / (mean_launch_ms * 1e-3) / 1e9
    # fp64 3d7pt: 7 fused multiply-adds per cell update = 14 FLOP
    flop_per_cell = 2 * len(inputs.shape_offsets("3d7pt"))
    tflops = cells * flop_per_cell / (mean_launch_ms * 1e-3) / 1e12
    try:
        sm_mhz = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"])
    except Exception:
        sm_mhz = 2070.0
    fp64_derived = fp64_peak_tflops(info["sm_count"], sm_mhz)
    # measured FP64 pipe throughput (independent FMA chains on every SM), best of 3
    fp64_peak = max(ctx.fp64_fma_benchmark(40000) for _ in range(3))
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        try:
            tj = json.load(open(prof))
            if (tj.get("kernel_signature") == desc_signature(desc)
                    and tj.get("source_sha256") == _sources_sha(tj.get("source_files", []))):
                traffic = tj.get("dram_bytes_per_launch")
        except Exception:
            pass
    st.close()
    del f
    torch.cuda.empty_cache()

    variants = {}
    if not args.no_variants and rank == 0:
        try:
            ps = stencil_leg(api, torch, ctx, L_3D, STEPS_3D, "f64", api.PER_STEP, 2, 1)
            variants["3d7pt_384_f64_per_step_baseline"] = {
                "gcells": cells / (min(ps["ms"]) * 1e-3) / 1e9, "ms": min(ps["ms"]), "plan": ps["plan"]}
            # the 2-D workload (2d5pt fp64 256^2, 100 steps): barrier-dominated
            for var, vname in ((api.PERSISTENT, "persistent"), (api.PER_STEP, "per_step")):
                r = stencil2d_leg(api, torch, ctx, 256, 100, var, 5, 2)
                variants[f"2d5pt_256_f64_{vname}"] = {
                    "gcells": 256 * 256 * 100 / (min(r["ms"]) * 1e-3) / 1e9, "ms": min(r["ms"]),
                    "us_per_step": min(r["ms"]) * 1e3 / 100, "kernel": r["kernel"], "plan": r["plan"]}
            # 3d7pt at 192^3 (fits on chip in fp32 / bf16) and 384^3, every storage type; the
            # fp32 / bf16 results are compared with the fp64 persistent result of the same field
            # (itself within 1e-12 of the fp64 oracle in the parity tests)
            for L in (192, 384):
                ref = None
                for dt in ("f64", "f32", "bf16"):
                    if L == 384 and dt == "f64":
                        r = stencil_leg(api, torch, ctx, L, STEPS_3D, dt, api.PERSISTENT, 1, 0, keep_result=True)
                        ref = r["result"]
                        continue
                    for var, vname in ((api.PERSISTENT, "persistent"), (api.PER_STEP, "per_step")):
                        r = stencil_leg(api, torch, ctx, L, STEPS_3D, dt, var, 2, 1,
                                        keep_result=(var == api.PERSISTENT))
                        c = float(L ** 3) * STEPS_3D
                        d = r["desc"]
                        ms = min(r["ms"])
                        v = {"gcells": c / (ms * 1e-3) / 1e9, "ms": ms,
                             "algorithmic_gbs": d["algorithmic_bytes"] / (ms * 1e-3) / 1e9,
                             "cached_fraction": d["cached_cells"] / max(d["cells"], 1), "kernel": kernel_name(d),
                             "threads": d["threads_per_block"], "plan": r["plan"]}
                        if var == api.PERSISTENT:
                            if dt == "f64":
                                ref = r["result"]
                            elif ref is not None:
                                v["err_vs_fp64"] = field_error(torch, r["result"], ref)
                        variants[f"3d7pt_{L}_{dt}_{vname}"] = v
                        r["result"] = None
                del ref
                torch.cuda.empty_cache()
        except Exception as e:
            variants["stencil_error"] = str(e)
        try:
            variants["cg"] = cg_leg(api, torch, ctx, 10)
        except Exception as e:
            variants["cg"] = {"error": str(e)}
        try:
            variants["batch64"] = batch_leg(api, torch, ctx, 2)
        except Exception as e:
            variants["batch64"] = {"error": str(e)}
        if not args.no_warmstart:
            try:
                variants["warmstart"] = warmstart_leg(api, torch, ctx, ntrain=args.ws_train_default,
                                                      label_rtol=1e-5, pool=args.ws_pool, reps=4)
            except Exception as e:
                variants["warmstart"] = {"error": str(e)}
        try:
            variants["grid_barrier_us"] = {str(b): ctx.barrier_benchmark(b, 512, 2000)
                                           for b in (info["sm_count"] // 4, info["sm_count"], 2 * info["sm_count"])}
        except Exception as e:
            variants["grid_barrier_us"] = {"error": str(e)}

    e2e_ms, h2d, d2h = e2e_leg(api, torch, ctx, L_3D, STEPS_3D, max(1, min(args.steps, 3)), 1)
    e2e_ms = _max_over_ranks(world, e2e_ms)
    e2e_val = world * cells / (e2e_ms * 1e-3) / 1e9

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_sample()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"3d7pt Jacobi {L_3D}^3 fp64, {STEPS_3D} steps per bench "
                                   "step, centre 0.4 / neighbours 0.1, Dirichlet 0, "
                                   "uniform[0,1) seeded; one persistent cooperative launch",
                       "l2": "inputs larger than L2 (2 x 453 MB ping-pong)",
                       "parallelism": f"replicas x{world}",
                       "plan": {**{k: desc[k] for k in ("grid_blocks", "threads_per_block", "tiles_x",
                                                       "tiles_y", "tiles_z", "reg_cache_planes",
                                                       "smem_cache_planes", "cached_cells",
                                                       "halo_cells_per_step")},
                                "kernel": kernel_name(desc), "planes_per_sync": desc["planes_per_sync"],
                                "balanced": bool(tuned.get("balanced")), "autotuned": True}},
            "roofline": {"bound": "alu", "achieved": tflops, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": tflops / fp64_peak, "traffic": traffic,
                         "peak_kind": "measured: fp64 FMA throughput of this GPU (perks_fp64_fma_benchmark, "
                                      "8 independent chains per thread, 4 x 256 threads per SM, best of 3)",
                         "derived_peak": {"value": fp64_derived, "how": f"{info['sm_count']} SMs x 2 fp64 FMA/clk "
                                                                       f"x 2 FLOP x {sm_mhz:.0f} MHz"},
                         "kernel": kernel_signature(desc, tuned),
                         "flop_per_cell_update": flop_per_cell,
                         "algorithmic_bytes_per_launch": desc["algorithmic_bytes"],
                         "mean_launch_ms": mean_launch_ms,
                         "hbm_view": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                                      "frac": achieved / peak, "peak_kind": peak_kind}},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": args.steps,
            "clocks": clk.summary(),
            "device": info,
            "variants": variants,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def profile_case(name):
    """Small cases for ncu captures: inputs larger than L2 (129 MB) but a few GB
    on the device at most, one warm-up launch, then the captured launch."""
    import torch
    from paper_2204_02064_gb300 import api, inputs
    ctx = api.Context(0)
    if name.startswith("headline"):
        # the bench's own launch configuration (3d7pt fp64 384^3, same plan),
        # two short launches of 20 and 40 steps: per-launch DRAM traffic is
        # a + b * steps, so a 1000-step launch is extrapolated from the pair
        L = L_3D
        shape = (L, L, L)
        f = torch.from_numpy(inputs.stencil_field(shape, 1)).cuda()
        st = api.Stencil(ctx, shape, inputs.shape_offsets("3d7pt"), inputs.workload_weights("3d7pt"))
        st.set_field(f)
        tuned = st.autotune(api.PERSISTENT, probe_steps=10)   # the bench's own plan choice
        st.set_field(f)
        st.run(2, stats=True)                      # warm-up launch
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("capture")      # ncu --nvtx --nvtx-include capture/ selects these
        for steps in (20, 40):
            st.set_field(f)
            d = st.run(steps, stats=True)
            print(json.dumps({"case": name, "L": L, "steps": steps, "plan": d, "tuned": tuned}))
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    elif name.startswith("stencil3d") or name.startswith("stencil384") or name.startswith("stencil192"):
        dt = "f64" if "f64" in name else ("bf16" if "bf16" in name else "f32")
        variant = api.PER_STEP if name.endswith("perstep") else api.PERSISTENT
        L = 384 if name.startswith("stencil384") else (192 if name.startswith("stencil192") else 256)
        steps = 4 if variant == api.PER_STEP else (8 if L == 384 else (100 if L == 192 else 20))
        shape = (L, L, L)
        f = torch.from_numpy(inputs.stencil_field(shape, 1)).to(
            {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[dt]).cuda()
        st = api.Stencil(ctx, shape, inputs.shape_offsets("3d7pt"), inputs.workload_weights("3d7pt"),
                         dtype=dt)
        plan = os.environ.get("PERKS_PROFILE_PLAN")  # "tx,ty,tz,reg_cache,smem_planes,planes_per_barrier"
        if plan:
            tx, ty, tz, reg, zs, P = (int(v) for v in plan.split(","))
            st.set_plan(tiles=(tx, ty, tz), reg_cache=reg, smem_cache_planes=zs, planes_per_barrier=P)
        elif name.startswith("stencil192"):
            st.set_field(f)
            print(json.dumps({"tuned": st.autotune(variant, probe_steps=10)}))  # the bench's own plan
        st.set_field(f)
        st.run(steps, variant, stats=True)            # warm-up launch
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("capture")        # ncu --nvtx --nvtx-include capture/ selects this launch
        st.set_field(f)
        d = st.run(steps, variant, stats=True)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"case": name, "L": L, "steps": steps, "plan": d}))
    elif name.startswith("cg"):
        n = 1 << 20
        rp, c, v = inputs.csr_spd_matrix(n, inputs.SEED_CG)
        op = api.CsrOperator(ctx, torch.from_numpy(rp).cuda(), torch.from_numpy(c).cuda(),
                             torch.from_numpy(v).cuda())
        b = torch.from_numpy(inputs.cg_rhs(n, inputs.SEED_CG)).cuda()
        mode = api.CG_FP32_IR if name == "cg-fp32ir" else api.CG_FP64
        for _ in range(2):
            x = torch.zeros(n, dtype=torch.float64, device="cuda")
            r = op.solve(b, x, rtol=1e-10, mode=mode, max_iter=20, raise_on_error=False)
        print(json.dumps({"case": name, "n": n, "result": r}))
    elif name == "warmnet-tc":
        # the tensor-core inner layers: 32 images of 256^2, bf16 storage
        n, m = 256, 32
        k, f = inputs.poisson_problems_device(n, m, seed=inputs.SEED_POISSON, ell=16.0)
        net = api.WarmNet(ctx, storage=api.BF16, seed=7)
        u = torch.zeros_like(f)
        net.predict(k, f, u)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("capture")
        net.predict(k, f, u)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"case": name, "images": m, "n": n}))
    elif name == "batch64":
        doms = inputs.batch_domains()
        b = api.Batch(ctx, doms, dtype="f32")
        for j, d in enumerate(doms):
            b.set_field(j, torch.from_numpy(inputs.stencil_field(d["shape"], d["seed"])).float().cuda())
        b.autotune(5)
        b.run(20, stats=True)
        torch.cuda.nvtx.range_push("capture")
        st = b.run(20, stats=True)
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"case": name, "stats": st}))
    elif name == "poisson":
        k, f = inputs.poisson_problems_device(512, 256, seed=inputs.SEED_POISSON)
        P = api.Poisson(ctx, k)
        x = torch.zeros_like(f)
        P.solve(f, x, rtol=1e-8, max_iter=50, stats=False)
        x.zero_()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("capture")
        P.solve(f, x, rtol=1e-8, max_iter=50, stats=False)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"case": name, "problems": 256, "n": 512, "iterations": 50}))
    else:
        raise SystemExit(f"unknown profile case {name}")
    torch.cuda.synchronize()
    return 0


def _sources_sha(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def fp64_peak_tflops(sm_count, sm_mhz):
    """GB300's FP64 pipe: 2 fused multiply-adds per clock per SM (1.25 TFLOP/s
    nominal at 2.07 GHz on 152 SMs)."""
    return sm_count * 2 * 2 * sm_mhz * 1e6 / 1e12


def kernel_signature(desc, tuned):
    """The dominant kernel, named from the plan the run actually used."""
    if desc.get("kernel") == 1:
        return ("perks_stencil_tile_kernel<double, 3d7pt, NT=%d, V=2, M=%d> (resident tile), tiles %dx%dx%d"
                % (desc["threads_per_block"], desc["planes_per_sync"], desc["tiles_x"], desc["tiles_y"],
                   desc["tiles_z"]))
    body = ("cache-free body" if desc["reg_cache_planes"] == 0 and desc["smem_cache_planes"] == 0
            else "cached body (%d register + %d shared-memory planes)" % (desc["reg_cache_planes"],
                                                                          desc["smem_cache_planes"]))
    split = ("tile columns %dx%d in balanced shares over %d blocks" % (desc["tiles_x"], desc["tiles_y"],
                                                                       desc["grid_blocks"])
             if tuned and tuned.get("balanced") else
             "tiles %dx%dx%d" % (desc["tiles_x"], desc["tiles_y"], desc["tiles_z"]))
    return ("perks_stencil_vec_kernel<double, 3d7pt, NT=%d, V=2, ZR=%d, D=%d, P=%d> (plane streaming, %s), %s"
            % (desc["threads_per_block"], desc["reg_cache_planes"], desc["prefetch_planes"],
               desc["planes_per_sync"], body, split))


def desc_signature(desc):
    return "{grid_blocks}-{threads_per_block}-{tiles_x}x{tiles_y}x{tiles_z}-r{reg_cache_planes}-s{smem_cache_planes}".format(**desc)


if __name__ == "__main__":
    sys.exit(main())
