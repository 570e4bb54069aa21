#!/usr/bin/env python3
"""Benchmark of the SGD_Tucker hot path on one GB300.

Workload (default): the Netflix-shaped rating tensor 480,189 x 17,770 x 2,182
with 100M nonzeros (Zipf 1.1 users, Zipf 1.3 items, uniform time; values in
{1..5} from a planted J=10 Tucker model), 99/1 train/test split, ranks J=10,
R_core=5, minibatch 4096.  Synthetic data of that shape stands in for the
Netflix dataset.  One step = one SGD epoch over the training nonzeros (sampler,
tiler, core phase, core rebuild and factor phase of every minibatch) plus the
RMSE/MAE pass over the test entries.  The metric is sampled nonzeros per
second per epoch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

`--impl reference` times the FP64 CPU oracle (the only other implementation of
this path) on the host cores over a bounded sample of the same workload.
Under torchrun (N > 1) every rank runs an independent replica (the strict
minibatch sequence has no data-parallel split without a per-phase exchange, so
N GPUs run N replicas; scaling is weak).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sampled nonzeros/s per SGD epoch at oracle RMSE, BF16 vs FP32; serve p99 latency"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    p.add_argument("--scale", type=float, default=1.0, help="workload scale (1.0 = 100M nonzeros)")
    p.add_argument("--cpu-batches", type=int, default=200,
                   help="minibatches in the oracle's timed sample (cpu_baseline of the GPU leg)")
    p.add_argument("--ref-batches", type=int, default=48,
                   help="minibatches per step of --impl reference")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-bf16", action="store_true")
    p.add_argument("--no-kruskal", action="store_true")
    p.add_argument("--no-momentum", action="store_true")
    p.add_argument("--no-parity", action="store_true", help="skip the GPU-vs-oracle parameter comparison")
    p.add_argument("--no-snapshot", action="store_true", help="skip the K-snapshot form")
    p.add_argument("--snapshot-ks", type=int, nargs="*", default=[2, 4, 8])
    p.add_argument("--no-sub", action="store_true",
                   help="skip the 4-order, batched and serving sub-records of the default line")
    p.add_argument("--variant-steps", type=int, default=5,
                   help="timed epochs of the BF16, Kruskal and momentum forms in the default line")
    p.add_argument("--sub-serve-seconds", type=float, default=30.0)
    p.add_argument("--sub-order4-scale", type=float, default=0.25)
    p.add_argument("--sub-batched-scale", type=float, default=1.0)
    p.add_argument("--batched", action="store_true",
                   help="batched workload instead of the default line: 256 independent 3-order tensors "
                        "(lognormal sizes, J in {4, 8, 16}) in one persistent launch per epoch")
    p.add_argument("--order4", action="store_true",
                   help="the 4-order workload (50M nonzeros at --scale 1), FP32 and BF16 epochs")
    p.add_argument("--msweep", action="store_true",
                   help="throughput against the minibatch size on the rating tensor (--scale, default 0.25)")
    p.add_argument("--serve", action="store_true",
                   help="open-loop serving run (job arrivals + query batches) instead of the epoch bench")
    p.add_argument("--serve-seconds", type=float, default=60.0)
    p.add_argument("--serve-rate", type=float, default=50.0, help="job arrivals per second")
    p.add_argument("--serve-qrate", type=float, default=200.0, help="query batches per second")
    p.add_argument("--serve-epochs", type=int, default=3)
    p.add_argument("--serve-pool", type=int, default=48, help="distinct job tensors generated up front")
    p.add_argument("--serve-budget-gb", type=float, default=120.0)
    p.add_argument("--serve-batches", type=int, default=32, help="minibatches per job per tick")
    p.add_argument("--serve-ctas", type=int, default=-1,
                   help="CTAs per job; 0 = tuned at the first tick; -1 = from each job's own size "
                        "(4 below 400k nonzeros, 8 below 1.2M, else 16)")
    p.add_argument("--serve-seed", type=int, default=0)
    p.add_argument("--serve-fp32", action="store_true")
    p.add_argument("--sweep", action="store_true",
                   help="rank sweep of the paper's parameter study instead of the default line: one JSON "
                        "line per (ranks, R_core) point on a fixed rating tensor (--scale, default 0.05)")
    return p.parse_args()


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _workload(scale):
    from paper_2012_03550_gb300 import synth
    t0 = time.time()
    w = synth.config2(scale=scale)
    gen_s = time.time() - t0
    return w, gen_s


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per training
# nonzero of one k_epoch launch, from the last ncu capture of each form, keyed
# by the sha256 prefix of the kernel source the capture ran.  The figure is
# reported only while the source is unchanged.
PROFILED_TRAFFIC = {
    "fp32": {"sha256_prefix": "58c0d639846d1c82", "dram_bytes_per_nnz": 75.84,
             "capture": "ncu --set full, rating tensor at 2% scale, one launch over its epoch (1,980,000 nonzeros)"},
    "snapshot8": {"sha256_prefix": "58c0d639846d1c82", "dram_bytes_per_nnz": 78.56,
                  "capture": "ncu --set full, K = 8, rating tensor at 2% scale, one launch over its epoch"},
}


def _profiled_traffic_per_nnz(precision="fp32"):
    """(DRAM bytes per training nonzero of one k_epoch launch, capture note),
    or (None, reason) when no capture matches the current kernel source."""
    import hashlib
    rec = PROFILED_TRAFFIC.get(precision)
    src = os.path.join(ROOT, "paper_2012_03550_gb300", "csrc", "sgdt_epoch.cu")
    if rec is None or not os.path.exists(src):
        return None, "no ncu capture of this form"
    with open(src, "rb") as fh:
        if hashlib.sha256(fh.read()).hexdigest()[:16] != rec["sha256_prefix"]:
            return None, "kernel changed since the last ncu capture"
    return rec["dram_bytes_per_nnz"], rec["capture"] + ", scaled by nonzeros"


def _bytes_per_nnz(N, J, s_f=4):
    # (N+1) passes each read the COO entry ((N+1) words) and N factor rows;
    # the N factor modes each write and read back one FP32 gradient row.
    return (N + 1) * ((4 * N + 4) + N * J * s_f) + N * J * 8


def _oracle_worker(args):
    """One host core: the oracle's minibatch steps on its own minibatches
    from the shared initial state; returns the seconds they took."""
    shape, ranks, R, A0, B0, batches, lr, lam = args
    from oracle import oracle as O
    md = O.Model(shape, ranks, R, A0, B0)
    t0 = time.perf_counter()
    for bc, bv in batches:
        md.step(bc, bv, lr, lr, lam, lam)
    return time.perf_counter() - t0


def _oracle_all_cores(t, w, c, v, A0, B0, M, per_core=8):
    """The oracle (unchanged, one process per host core) on independent
    minibatches from one state: the host's aggregate oracle throughput.  The
    strict minibatch sequence has no parallel split, so this is a capacity
    figure (replicas), and the epoch time from it is an extrapolation."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    from oracle import oracle as O
    try:
        O.build()
        ids = O.perm_range(c.shape[0], 2, 0, 0, cores * per_core * M)
        jobs = []
        for q in range(cores):
            bl = []
            for b in range(per_core):
                sl = ids[(q * per_core + b) * M:(q * per_core + b + 1) * M]
                bl.append((c[sl], v[sl]))
            jobs.append((t.shape, w.ranks, w.r_core, A0, B0, bl, w.lr, w.lam))
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as pool:
            secs = pool.map(_oracle_worker, jobs)
    except Exception as e:                                      # reported, never fatal to the bench
        return {"error": f"{type(e).__name__}: {e}"}
    rate = cores * per_core * M / max(secs)
    return {"value": rate, "unit": "nnz/s", "cores": cores, "kind": "oracle",
            "sample": f"{per_core} minibatches of {M} per core, one process per core, all from the initial state "
                      f"(independent replicas; the slowest core's time)",
            "epoch_s_extrapolated": c.shape[0] / rate}


class ClockSampler:
    """nvidia-smi clock/throttle samples (200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names[1:], parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(a):
    """FP64 oracle on the host cores over bounded samples of the workload."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import numpy as np
    from oracle import oracle as O
    from paper_2012_03550_gb300 import synth
    w, _ = _workload(a.scale)
    c, v = w.tensor.split("train")
    A0, B0 = synth.init_params(w.tensor.shape, w.ranks, w.r_core, mode="rating", seed=1,
                               mean_value=float(np.mean(v)))
    md = O.Model(w.tensor.shape, w.ranks, w.r_core, A0, B0)
    M = w.minibatch
    nb = a.ref_batches
    times = []
    for step in range(a.warmup + a.steps):
        b0 = (step * nb) % max(1, (c.shape[0] // M) - nb)
        t0 = time.perf_counter()
        md.epoch(c, v, M, 2, 0, w.lr, w.lr, w.lam, w.lam, 0, b0, b0 + nb)
        dt = time.perf_counter() - t0
        if step >= a.warmup:
            times.append(dt)
    sample = nb * M
    ms = 1e3 * sum(times) / len(times)
    value = sample / (ms * 1e-3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "minibatch": M, "ranks": list(w.ranks), "r_core": w.r_core,
                   "step": f"{nb} minibatches of epoch 0 (bounded sample of one epoch)"},
        "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": 1, "kind": "oracle",
                         "sample": f"{nb} minibatches x {M} nonzeros per step, single thread"},
        "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(a):
    import numpy as np
    import torch

    from paper_2012_03550_gb300 import dist as D
    world, rank, local = D.world()
    if world > 1:
        D.init("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as ge
    ge.build()
    from paper_2012_03550_gb300 import binding as B
    from paper_2012_03550_gb300 import synth

    w, gen_s = _workload(a.scale)
    t = w.tensor
    c, v = t.split("train")
    tc, tv = t.split("test")
    N, J, R, M = t.order, w.ranks[0], w.r_core, w.minibatch
    A0, B0 = synth.init_params(t.shape, w.ranks, R, mode="rating", seed=1, mean_value=float(np.mean(v)))

    stream = torch.cuda.Stream(device=dev)
    # device-resident inputs: the COO and the test split live in HBM
    dc = torch.from_numpy(c).to(dev)
    dv = torch.from_numpy(v).to(dev)
    dtc = torch.from_numpy(tc).to(dev)
    dtv = torch.from_numpy(tv).to(dev)
    torch.cuda.synchronize()
    opt = B.std_default_options()
    opt.r_core = R
    opt.ptr_kind = 1
    opt.stream = stream.cuda_stream
    ctx = B.std_create(N, t.shape, w.ranks, c.shape[0], dc, dv, opt)
    B.std_set_params(ctx, [np.ascontiguousarray(x) for x in A0], [np.ascontiguousarray(x) for x in B0], 0)

    rm_at = {}    # test RMSE of the main run after e epochs

    def step():
        st = B.std_sgd_epoch(ctx, w.lr, w.lr, w.lam, w.lam, M)
        r = B.std_rmse(ctx, tc.shape[0], dtc, dtv)
        rm_at[st["epoch"] + 1] = r[0]
        return st, r

    vsteps = max(1, min(a.steps, a.variant_steps))
    vwarm = min(a.warmup, 3)
    for _ in range(a.warmup):
        step()
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    D.barrier()
    sampler.start()
    time.sleep(0.3)
    with torch.cuda.stream(stream):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        upd, sched, rm = [], [], None
        for _ in range(a.steps):
            st, rm = step()
            upd.append(st["update_seconds"])
            sched.append(st["sched_seconds"])
        e1.record(stream)
    torch.cuda.synchronize()
    D.barrier()
    clocks = sampler.stop()
    n_train = c.shape[0]
    # every rank runs its own replica: all ranks' nonzeros over the slowest rank's time
    value, elapsed = D.weak_scaling_rate(float(n_train * a.steps), e0.elapsed_time(e1) * 1e-3, device=dev)
    ms_per_step = 1e3 * elapsed / a.steps

    # the BF16 form on the same data and schedule (BF16 factor mirrors and core,
    # tensor-core contraction, FP32 masters): throughput and RMSE gap
    bf16 = None
    if not a.no_bf16:
        o16 = B.std_default_options()
        o16.r_core = R
        o16.ptr_kind = 1
        o16.precision = 1
        o16.stream = stream.cuda_stream
        cx16 = B.std_create(N, t.shape, w.ranks, c.shape[0], dc, dv, o16)
        B.std_set_params(cx16, [np.ascontiguousarray(x) for x in A0], [np.ascontiguousarray(x) for x in B0], 0)
        rm16 = None
        for _ in range(vwarm):
            B.std_sgd_epoch(cx16, w.lr, w.lr, w.lam, w.lam, M)
            B.std_rmse(cx16, tc.shape[0], dtc, dtv)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        upd16 = []
        for _ in range(vsteps):
            st16 = B.std_sgd_epoch(cx16, w.lr, w.lr, w.lam, w.lam, M)
            rm16 = B.std_rmse(cx16, tc.shape[0], dtc, dtv)
            upd16.append(st16["update_seconds"])
        f1.record(stream)
        torch.cuda.synchronize()
        v16, e16 = D.weak_scaling_rate(float(n_train * vsteps), f0.elapsed_time(f1) * 1e-3, device=dev)
        bf16 = {"value": v16, "unit": "nnz/s", "ms_per_step": 1e3 * e16 / vsteps,
                "kernel_ms": 1e3 * sum(upd16) / len(upd16),
                "speedup_vs_fp32": v16 / value,
                "test_rmse": rm16[0], "test_mae": rm16[1],
                "test_rmse_gap_vs_fp32": (abs(rm16[0] - rm_at[vwarm + vsteps])
                                          if (vwarm + vsteps) in rm_at else None),
                "bytes_per_nnz": _bytes_per_nnz(N, J, 2),
                "epochs": vwarm + vsteps,
                "note": ("same schedule and initial state as the FP32 run; test RMSE after its own epochs "
                         "(the gap compares it with the FP32 run after as many epochs)")}
        B.std_destroy(cx16)
    def variant(**fields):
        """Same workload, schedule and initial state under other options."""
        ov = B.std_default_options()
        ov.r_core = R
        ov.ptr_kind = 1
        ov.stream = stream.cuda_stream
        for k_, v_ in fields.items():
            setattr(ov, k_, v_)
        cxv = B.std_create(N, t.shape, w.ranks, c.shape[0], dc, dv, ov)
        B.std_set_params(cxv, [np.ascontiguousarray(x) for x in A0], [np.ascontiguousarray(x) for x in B0], 0)
        for _ in range(vwarm):
            B.std_sgd_epoch(cxv, w.lr, w.lr, w.lam, w.lam, M)
            B.std_rmse(cxv, tc.shape[0], dtc, dtv)
        torch.cuda.synchronize()
        v0 = torch.cuda.Event(enable_timing=True)
        v1 = torch.cuda.Event(enable_timing=True)
        v0.record(stream)
        updv, rmv = [], None
        for _ in range(vsteps):
            stv = B.std_sgd_epoch(cxv, w.lr, w.lr, w.lam, w.lam, M)
            rmv = B.std_rmse(cxv, tc.shape[0], dtc, dtv)
            updv.append(stv["update_seconds"])
        v1.record(stream)
        torch.cuda.synchronize()
        vv, ev = D.weak_scaling_rate(float(n_train * vsteps), v0.elapsed_time(v1) * 1e-3, device=dev)
        B.std_destroy(cxv)
        return {"value": vv, "unit": "nnz/s", "ms_per_step": 1e3 * ev / vsteps,
                "kernel_ms": 1e3 * sum(updv) / len(updv), "speedup_vs_main": vv / value,
                "epochs": vwarm + vsteps, "test_rmse": rmv[0], "test_rmse_main_same_epochs": rm_at.get(vwarm + vsteps)}

    # the Kruskal form of the factor-phase contraction (E_s = B(n) w_s, the
    # same product as the Kronecker rows against the unfolded core)
    kru = None
    if not a.no_kruskal:
        kru = variant(contraction=1)
        kru["note"] = "FP32; same schedule and initial state as the main line"
    # heavy-ball momentum (mu = 0.9) on the same workload
    mom = None
    if not a.no_momentum:
        mom = variant(momentum=0.9)
        mom["note"] = "FP32, mu = 0.9, same learning rate; RMSE after the same epochs"
    # the K-snapshot form (a labelled variant of the minibatch order: every
    # minibatch of a block of K steps from the block's starting model, the
    # changes added in minibatch order), K groups of CTAs at once
    snap = None
    if not a.no_snapshot:
        snap = {"note": ("labelled variant, not Algorithm 1's order: blocks of K minibatches step from one model "
                         "and their changes are added in minibatch order; FP32; roofline of its update kernel "
                         "against the same bytes per nonzero")}
        peak_s, _ = _peaks()
        for K in a.snapshot_ks:
            try:
                r = variant(snapshot=K)
            except B.StdError as e:
                snap[f"K{K}"] = {"unavailable": str(e)}
                continue
            ach = n_train * _bytes_per_nnz(N, J) / (r["kernel_ms"] * 1e-3) / 1e9
            r["roofline_frac"] = ach / peak_s
            r["achieved_gbs"] = ach
            tpk, _ = _profiled_traffic_per_nnz(f"snapshot{K}")
            r["traffic"] = tpk * n_train if tpk is not None else None
            snap[f"K{K}"] = r
    del dc, dv

    # roofline of the dominant kernel (the persistent update kernel)
    bpn = _bytes_per_nnz(N, J)
    upd_s = sum(upd) / len(upd)
    achieved = n_train * bpn / upd_s / 1e9
    peak, peak_kind = _peaks()
    tpn, tnote = _profiled_traffic_per_nnz()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (tpn * n_train if tpn is not None else None),
                "traffic_note": tnote,
                "kernel": "k_epoch", "peak_kind": peak_kind,
                "bytes_per_nnz": bpn, "kernel_ms": upd_s * 1e3, "sched_kernel_ms": 1e3 * sum(sched) / len(sched)}

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not a.no_e2e and a.e2e_steps > 0:
        pc = torch.from_numpy(c).pin_memory()
        pv = torch.from_numpy(v).pin_memory()
        ptc = torch.from_numpy(tc).pin_memory()
        ptv = torch.from_numpy(tv).pin_memory()
        hA = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in A0]
        hB = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in B0]
        nA = [x.numpy() for x in hA]
        nB = [x.numpy() for x in hB]
        o2 = B.std_default_options()
        o2.r_core = R
        o2.ptr_kind = 0
        o2.stream = stream.cuda_stream
        h2d = c.nbytes + v.nbytes + sum(x.nbytes for x in nA) + sum(x.nbytes for x in nB) + tc.nbytes + tv.nbytes
        d2h = 16
        times = []
        for i in range(a.e2e_steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cx = B.std_create(N, t.shape, w.ranks, c.shape[0], pc.numpy(), pv.numpy(), o2)
            B.std_set_params(cx, nA, nB, 0)
            B.std_sgd_epoch(cx, w.lr, w.lr, w.lam, w.lam, M)
            B.std_rmse(cx, tc.shape[0], ptc.numpy(), ptv.numpy())
            B.std_destroy(cx)
            torch.cuda.synchronize()
            if i > 0:
                times.append(time.perf_counter() - t0)
        e2e = {"value": n_train / (sum(times) / len(times)), "unit": "nnz/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": d2h, "steps": len(times),
               "path": "std_create(host COO) + std_set_params + std_sgd_epoch + std_rmse(host test) + std_destroy"}

    # CPU baseline: the oracle as it stands on a bounded sample (rank 0, N = 1)
    cpu = None
    parity = None
    if not a.no_cpu_baseline and world == 1 and rank == 0:
        from oracle import oracle as O
        md = O.Model(t.shape, w.ranks, R, A0, B0)
        nb = a.cpu_batches
        t0 = time.perf_counter()
        md.epoch(c, v, M, 2, 0, w.lr, w.lr, w.lam, w.lam, 0, 0, nb)
        dt = time.perf_counter() - t0
        cpu = {"value": nb * M / dt, "unit": "nnz/s", "cores": 1, "nproc": os.cpu_count(), "kind": "oracle",
               "sample": f"first {nb} minibatches ({nb * M} nonzeros) of epoch 0, FP64, single thread",
               "epoch_s_extrapolated": n_train / (nb * M / dt)}
        allc = _oracle_all_cores(t, w, c, v, A0, B0, M)
        if allc is not None:
            cpu["all_cores"] = allc
        # the same minibatches on the GPU from the same state, FP32 and BF16:
        # parameters and test RMSE against the oracle's after them
        if not a.no_parity:
            parity = {"minibatches": nb, "from": "the bench's initial state, epoch 0"}
            ro, mo = md.rmse_mae(tc, tv)
            for name, prec in (("fp32", 0), ("bf16", 1)):
                op = B.std_default_options()
                op.r_core = R
                op.ptr_kind = 1
                op.precision = prec
                op.stream = stream.cuda_stream
                dcp, dvp = torch.from_numpy(c).to(dev), torch.from_numpy(v).to(dev)
                cxp = B.std_create(N, t.shape, w.ranks, c.shape[0], dcp, dvp, op)
                B.std_set_params(cxp, [np.ascontiguousarray(x) for x in A0],
                                 [np.ascontiguousarray(x) for x in B0], 0)
                B.std_sgd_batches(cxp, w.lr, w.lr, w.lam, w.lam, M, 0, nb)
                Ag = [np.empty((t.shape[n], w.ranks[n]), np.float32) for n in range(N)]
                Bg = [np.empty((w.ranks[n], R), np.float32) for n in range(N)]
                B.std_get_params(cxp, Ag, Bg, None)
                rg, mg = B.std_rmse(cxp, tc.shape[0], dtc, dtv)
                B.std_destroy(cxp)
                del dcp, dvp
                parity[name] = {
                    "max_rel_err_A": max(float(np.abs(Ag[n] - md.A[n]).max() / np.abs(md.A[n]).max())
                                         for n in range(N)),
                    "max_rel_err_B": max(float(np.abs(Bg[n] - md.B[n]).max() / np.abs(md.B[n]).max())
                                         for n in range(N)),
                    "test_rmse": rg, "test_mae": mg, "test_rmse_oracle": ro, "test_mae_oracle": mo,
                    "test_rmse_abs_err": abs(rg - ro), "test_mae_abs_err": abs(mg - mo)}
            parity["note"] = ("max over modes of max|gpu - oracle| / max|oracle| per factor / Kruskal matrix; "
                              "RMSE/MAE over the test split (Eq. 19)")

    B.std_destroy(ctx)
    del dtc, dtv
    sub = {}
    if not a.no_sub and world == 1:
        torch.cuda.empty_cache()
        for key, fn in (("order4", lambda: order4_record(a, a.sub_order4_scale, 1, 3)),
                        ("batched", lambda: batched_record(a, a.sub_batched_scale, 1, 1)),
                        ("serve", lambda: serve_record(a, a.sub_serve_seconds))):
            t0 = time.time()
            sub[key] = fn()
            sub[key]["wall_s"] = round(time.time() - t0, 1)
            torch.cuda.empty_cache()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "nnz_train": int(n_train), "nnz_test": int(tc.shape[0]),
                       "minibatch": M, "ranks": list(w.ranks), "r_core": R, "precision": "fp32",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (COO and per-epoch schedule are GBs); no flush",
                       "step": "one epoch (sampler, tiler, core and factor phases) + test RMSE/MAE",
                       "datagen_s": round(gen_s, 1)},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "bf16": bf16,
            "kruskal_contraction": kru,
            "momentum": mom,
            "snapshot": snap,
            "oracle_parity": parity,
            "order4": sub.get("order4"),
            "batched": sub.get("batched"),
            "serve": sub.get("serve"),
            "gpu_launches": 4 * a.steps,
            "clocks": clocks,
            "test_rmse": rm[0] if rm else None,
            "test_mae": rm[1] if rm else None,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()
    return 0


def run_sweep(a):
    """Epoch time and test RMSE over the rank sweep (one line per point)."""
    import numpy as np
    import torch

    import __graft_entry__ as ge
    ge.build()
    from paper_2012_03550_gb300 import binding as B
    from paper_2012_03550_gb300 import synth

    scale = a.scale if a.scale != 1.0 else 0.05
    w, points = synth.ranksweep(scale=scale)
    t = w.tensor
    c, v = t.split("train")
    tc, tv = t.split("test")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    dc, dv = torch.from_numpy(c).to(dev), torch.from_numpy(v).to(dev)
    dtc, dtv = torch.from_numpy(tc).to(dev), torch.from_numpy(tv).to(dev)
    for ranks, R in points:
        A0, B0 = synth.init_params(t.shape, ranks, R, mode="rating", seed=1, mean_value=float(np.mean(v)))
        opt = B.std_default_options()
        opt.r_core = R
        opt.ptr_kind = 1
        opt.stream = stream.cuda_stream
        ctx = B.std_create(t.order, t.shape, ranks, c.shape[0], dc, dv, opt)
        B.std_set_params(ctx, [np.ascontiguousarray(x) for x in A0], [np.ascontiguousarray(x) for x in B0], 0)
        for _ in range(a.warmup):
            B.std_sgd_epoch(ctx, w.lr, w.lr, w.lam, w.lam, w.minibatch)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            B.std_sgd_epoch(ctx, w.lr, w.lr, w.lam, w.lam, w.minibatch)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.steps
        rm = B.std_rmse(ctx, tc.shape[0], dtc, dtv)
        B.std_destroy(ctx)
        line = {"metric": "rank sweep: epoch time and test RMSE", "workload": w.name, "ranks": list(ranks),
                "r_core": R, "minibatch": w.minibatch, "epochs": a.warmup + a.steps, "ms_per_epoch": ms,
                "value": c.shape[0] / (ms * 1e-3), "unit": "nnz/s", "test_rmse": rm[0], "test_mae": rm[1],
                "data": "synthetic"}
        print(json.dumps(line), flush=True)
    return 0


def run_msweep(a):
    """Throughput against the minibatch size M on the rating tensor (strict
    Algorithm 1 at every M): the per-minibatch chain of dependent steps is
    amortised over more samples as M grows.  The learning rate scales with
    M / 4096 so that the step per epoch stays comparable."""
    import numpy as np
    import torch

    import __graft_entry__ as ge
    ge.build()
    from paper_2012_03550_gb300 import binding as B
    from paper_2012_03550_gb300 import synth

    scale = a.scale if a.scale != 1.0 else 0.25
    w = synth.config2(scale=scale)
    t = w.tensor
    c, v = t.split("train")
    tc, tv = t.split("test")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    dc, dv = torch.from_numpy(c).to(dev), torch.from_numpy(v).to(dev)
    dtc, dtv = torch.from_numpy(tc).to(dev), torch.from_numpy(tv).to(dev)
    A0, B0 = synth.init_params(t.shape, w.ranks, w.r_core, mode="rating", seed=1, mean_value=float(np.mean(v)))
    for M in (1024, 2048, 4096, 8192, 16384):
        lr = w.lr * M / 4096.0
        opt = B.std_default_options()
        opt.r_core = w.r_core
        opt.ptr_kind = 1
        opt.stream = stream.cuda_stream
        ctx = B.std_create(t.order, t.shape, w.ranks, c.shape[0], dc, dv, opt)
        B.std_set_params(ctx, [np.ascontiguousarray(x) for x in A0], [np.ascontiguousarray(x) for x in B0], 0)
        for _ in range(a.warmup):
            B.std_sgd_epoch(ctx, lr, lr, w.lam, w.lam, M)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            st = B.std_sgd_epoch(ctx, lr, lr, w.lam, w.lam, M)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.steps
        rm = B.std_rmse(ctx, tc.shape[0], dtc, dtv)
        B.std_destroy(ctx)
        nb = (c.shape[0] + M - 1) // M
        line = {"metric": "minibatch sweep: epoch throughput and test RMSE", "workload": w.name, "minibatch": M,
                "lr": lr, "epochs": a.warmup + a.steps, "ms_per_epoch": ms, "value": c.shape[0] / (ms * 1e-3),
                "unit": "nnz/s", "us_per_minibatch": 1e6 * st["update_seconds"] / nb, "test_rmse": rm[0],
                "data": "synthetic"}
        print(json.dumps(line), flush=True)
    return 0


def run_order4(a):
    print(json.dumps(order4_record(a, a.scale, a.warmup, a.steps)), flush=True)
    return 0


def order4_record(a, scale, warmup, steps):
    """The 4-order workload (200,000 x 100,000 x 500 x 24, 50M nonzeros at
    scale 1, J = 8, M = 8192): epoch throughput and test RMSE of the FP32 form
    and of the BF16 form, whose factor-phase contraction (512 x 8 per mode and
    sample) runs on the tensor cores."""
    import numpy as np
    import torch

    import __graft_entry__ as ge
    ge.build()
    from paper_2012_03550_gb300 import binding as B
    from paper_2012_03550_gb300 import synth

    t0 = time.time()
    w = synth.config3(scale=scale)
    gen_s = time.time() - t0
    t = w.tensor
    c, v = t.split("train")
    tc, tv = t.split("test")
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    dc, dv = torch.from_numpy(c).to(dev), torch.from_numpy(v).to(dev)
    dtc, dtv = torch.from_numpy(tc).to(dev), torch.from_numpy(tv).to(dev)
    A0, B0 = synth.init_params(t.shape, w.ranks, w.r_core, mode="normal", seed=1)
    res = {}
    for prec in (0, 1):
        opt = B.std_default_options()
        opt.r_core = w.r_core
        opt.ptr_kind = 1
        opt.precision = prec
        opt.stream = stream.cuda_stream
        ctx = B.std_create(t.order, t.shape, w.ranks, c.shape[0], dc, dv, opt)
        B.std_set_params(ctx, [np.ascontiguousarray(x) for x in A0], [np.ascontiguousarray(x) for x in B0], 0)
        for _ in range(warmup):
            B.std_sgd_epoch(ctx, w.lr, w.lr, w.lam, w.lam, w.minibatch)
        torch.cuda.synchronize()
        # each epoch timed on its own; the median is reported (a host-side
        # stall in one of a few epochs does not set the figure)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        upds = []
        evs[0].record(stream)
        for i in range(steps):
            upds.append(B.std_sgd_epoch(ctx, w.lr, w.lr, w.lam, w.lam, w.minibatch)["update_seconds"])
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        ms = float(np.median([evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]))
        upd = float(np.median(upds)) * steps
        rm = B.std_rmse(ctx, tc.shape[0], dtc, dtv)
        B.std_destroy(ctx)
        nb = (c.shape[0] + w.minibatch - 1) // w.minibatch
        res[prec] = {"value": c.shape[0] / (ms * 1e-3), "ms_per_epoch": ms,
                     "us_per_minibatch": 1e6 * upd / steps / nb, "test_rmse": rm[0]}
    line = {"metric": "4-order workload: sampled nonzeros/s per epoch, FP32 and BF16", "workload": w.name,
            "nnz_train": int(c.shape[0]), "minibatch": w.minibatch, "ranks": list(w.ranks), "r_core": w.r_core,
            "epochs": warmup + steps, "epoch_time": "median of the timed epochs (CUDA events)",
            "value": res[0]["value"], "unit": "nnz/s", "fp32": res[0], "bf16": res[1],
            "bf16_speedup": res[1]["value"] / res[0]["value"],
            "bf16_test_rmse_gap": abs(res[1]["test_rmse"] - res[0]["test_rmse"]), "datagen_s": round(gen_s, 1),
            "data": "synthetic"}
    return line


def run_batched(a):
    print(json.dumps(batched_record(a, a.scale, a.warmup, a.steps)), flush=True)
    return 0


def batched_record(a, nnz_scale, warmup, steps):
    """Epochs of 256 independent decompositions in one launch per epoch, FP32 and
    BF16, against the same tensors run one after another on the whole GPU."""
    import numpy as np
    import torch

    import __graft_entry__ as ge
    ge.build()
    from paper_2012_03550_gb300 import binding as B
    from paper_2012_03550_gb300 import synth

    t0 = time.time()
    specs = synth.config4_specs(nnz_scale=nnz_scale)
    tensors = [synth.config4_tensor(sp) for sp in specs]
    gen_s = time.time() - t0
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    M, lr, lam = 256, 1e-3, 1e-3
    data = []
    for tt in tensors:
        c, v = tt.split("train")
        data.append((torch.from_numpy(c).to(dev), torch.from_numpy(v).to(dev)))
    n_train = sum(int(d[0].shape[0]) for d in data)

    def contexts(precision):
        out = []
        for sp, tt, (dc, dv) in zip(specs, tensors, data):
            o = B.std_default_options()
            o.r_core = sp["R"]
            o.ptr_kind = 1
            o.precision = precision
            o.stream = stream.cuda_stream
            out.append(B.std_create(3, tt.shape, (sp["J"],) * 3, int(dc.shape[0]), dc, dv, o))
        return out

    lines = {}
    for precision in (0, 1):
        ctxs = contexts(precision)
        bt = B.std_batch_create(ctxs, 0)
        for _ in range(warmup):
            st = B.std_batch_epoch(bt, lr, lr, lam, lam, M)
        torch.cuda.synchronize()
        secs = []
        for _ in range(steps):
            st = B.std_batch_epoch(bt, lr, lr, lam, lam, M)
            secs.append(st["seconds"])
        sizes = B.std_batch_groups(bt, len(ctxs))
        tile = B.std_batch_tile(bt)
        B.std_batch_destroy(bt)
        # test RMSE over all members (weighted by test entries)
        se, cnt = 0.0, 0
        for ctx, tt in zip(ctxs, tensors):
            tc, tv = tt.split("test")
            if tc.shape[0] == 0:
                continue
            r = B.std_rmse(ctx, tc.shape[0], torch.from_numpy(tc).to(dev), torch.from_numpy(tv).to(dev))
            se += r[0] ** 2 * tc.shape[0]
            cnt += tc.shape[0]
        # the same epoch with every tensor alone on the whole GPU, one after another
        seq = None
        if precision == 0:
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for ctx in ctxs:
                B.std_sgd_epoch(ctx, lr, lr, lam, lam, M)
            e1.record(stream)
            torch.cuda.synchronize()
            seq = n_train / (e0.elapsed_time(e1) * 1e-3)
        for ctx in ctxs:
            B.std_destroy(ctx)
        ms = 1e3 * sum(secs) / len(secs)
        hist = {}
        for g in sizes:
            hist[str(g)] = hist.get(str(g), 0) + 1
        lines[precision] = {"value": n_train / (ms * 1e-3), "ms_per_epoch": ms, "ctas_per_tensor": st["ctas_per_tensor"],
                            "contraction_tile": tile,
                            "tensors_by_group_size": hist, "graph_replayed": st["graph_replayed"],
                            "test_rmse": (se / cnt) ** 0.5 if cnt else None, "sequential_value": seq}
    line = {"metric": "batched SGD_Tucker: sampled nonzeros/s per epoch over all tensors", "value": lines[0]["value"],
            "unit": "nnz/s", "n_gpus": 1, "steps": steps, "warmup": warmup,
            "ms_per_step": lines[0]["ms_per_epoch"], "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched-{len(specs)}-tensors-{n_train}", "tensors": len(specs),
                       "nnz_train": n_train, "minibatch": M, "ranks": "J in {4, 8, 16}, R = min(5, J)",
                       "ctas_per_tensor": lines[0]["ctas_per_tensor"],
                       "contraction_tile": lines[0]["contraction_tile"],
                       "tensors_by_group_size": lines[0]["tensors_by_group_size"],
                       "graph_replayed": lines[0]["graph_replayed"], "datagen_s": round(gen_s, 1),
                       "step": "one epoch of every tensor in one persistent launch (samplers and tilers before it)"},
            "test_rmse": lines[0]["test_rmse"],
            "one_after_another_value": lines[0]["sequential_value"],
            "speedup_vs_one_after_another": lines[0]["value"] / lines[0]["sequential_value"],
            "bf16": {"value": lines[1]["value"], "ms_per_step": lines[1]["ms_per_epoch"],
                     "ctas_per_tensor": lines[1]["ctas_per_tensor"], "test_rmse": lines[1]["test_rmse"],
                     "speedup_vs_fp32": lines[1]["value"] / lines[0]["value"]}}
    return line


def run_serve(a):
    print(json.dumps(serve_record(a, a.serve_seconds)), flush=True)
    return 0


def serve_record(a, seconds):
    """Open-loop serving run: Poisson job arrivals and query batches against the
    continuous-batching server for a fixed wall time, then a drain."""
    import numpy as np

    import __graft_entry__ as ge
    ge.build()
    from paper_2012_03550_gb300 import serve, synth

    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([a.serve_seed, 9])))
    t0 = time.time()
    specs = synth.serve_specs(a.serve_pool, seed=a.serve_seed)
    pool = []
    for sp in specs:
        tt = synth.serve_tensor(sp)
        c, v = tt.split("train")
        pool.append((sp, c, v))
    gen_s = time.time() - t0
    M, lr, lam = 256, 1e-3, 1e-3
    eng = serve.CudaEngine(precision=0 if a.serve_fp32 else 1, max_query=4096)
    def by_size(job):
        return 4 if job.nnz < 400_000 else (8 if job.nnz < 1_200_000 else 16)

    srv = serve.Server(eng, budget_bytes=int(a.serve_budget_gb * 1e9), batches_per_tick=a.serve_batches,
                       ctas_per_tensor=by_size if a.serve_ctas < 0 else a.serve_ctas)
    # arrival times (s from the start): jobs and query batches, both Poisson
    jobs_t = np.cumsum(rng.exponential(1.0 / a.serve_rate, size=int(a.serve_rate * seconds * 2) + 16))
    jobs_t = jobs_t[jobs_t < seconds]
    q_t = np.cumsum(rng.exponential(1.0 / a.serve_qrate, size=int(a.serve_qrate * seconds * 2) + 16))
    q_t = q_t[q_t < seconds]
    tables = {}

    def query_coords(shape):
        k = int(np.exp(rng.uniform(0.0, np.log(4096.0))))
        cols = []
        for size in shape:
            if size not in tables:
                tables[size] = synth.zipf_table(int(size), 1.1)
            cols.append(synth.draw_mode_indices(rng, k, int(size), "zipf", 1.1, table=tables[size]))
        return np.stack(cols, axis=1).astype(np.int32)

    clk = srv.clock
    start = clk()
    ij = iq = 0
    nnz_in_window = 0
    try:
        while True:
            now = clk() - start
            if now >= seconds:
                break
            while ij < len(jobs_t) and jobs_t[ij] <= now:
                sp, c, v = pool[ij % len(pool)]
                job = serve.Job(shape=sp["shape"], ranks=(sp["J"],) * len(sp["shape"]), coords=c, values=v,
                                epochs=a.serve_epochs, minibatch=M, lr_a=lr, lr_b=lr, lam_a=lam, lam_b=lam,
                                r_core=sp["R"], options={"seed_init": 1000 + ij, "seed_sched": 2000 + ij})
                srv.submit(job, now=start + float(jobs_t[ij]))
                ij += 1
            while iq < len(q_t) and q_t[iq] <= now:
                live = [j for j in srv.running] + list(srv.resident_done.values())
                if live:
                    j = live[int(rng.integers(0, len(live)))]
                    srv.query(j.id, query_coords(j.shape), now=start + float(q_t[iq]))
                iq += 1
            if srv.idle():
                nxt = min(jobs_t[ij] if ij < len(jobs_t) else seconds,
                          q_t[iq] if iq < len(q_t) else seconds)
                time.sleep(max(0.0, min(0.01, nxt - (clk() - start))))
                continue
            srv.tick()
        window_s = clk() - start
        nnz_in_window = srv.nnz
        gpu_in_window = srv.gpu_seconds
        srv.run_until_idle()
        total_s = clk() - start
    finally:
        srv.shutdown()
    r = srv.report()
    line = {"metric": "serve p99 job-epoch latency", "value": r["job_epoch_p99_s"], "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "dtype": "bf16-storage/f32" if not a.serve_fp32 else "f32",
            "data": "synthetic",
            "config": {"workload": f"serve-{a.serve_rate:g}jobs_s-{seconds:g}s",
                       "arrivals": f"Poisson {a.serve_rate:g} jobs/s, {a.serve_qrate:g} query batches/s "
                                   f"(1-4096 Zipf(1.1) coordinates, log-uniform size)",
                       "jobs": f"orders 3-4, J in {{4,8,16}} (order 4: {{4,8}}), nnz lognormal [1e4, 2e6], "
                               f"{a.serve_epochs} epochs each, M = {M}, lr = lambda = 1e-3; a pool of "
                               f"{len(pool)} distinct tensors, each arrival with its own seeds",
                       "budget_gb": a.serve_budget_gb, "batches_per_tick": a.serve_batches,
                       "ctas_per_job": "4 / 8 / 16 by the job's nonzeros (<400k / <1.2M / more)"
                       if a.serve_ctas < 0 else srv.group, "window_s": round(window_s, 2),
                       "drain_s": round(total_s - window_s, 2), "datagen_s": round(gen_s, 1)},
            "job_epoch_p50_s": r["job_epoch_p50_s"], "job_epoch_p99_s": r["job_epoch_p99_s"],
            "job_p50_s": r["job_p50_s"], "job_p99_s": r["job_p99_s"],
            "queue_wait_p50_s": r["queue_wait_p50_s"], "queue_wait_p99_s": r["queue_wait_p99_s"],
            "query_p50_s": r["query_p50_s"], "query_p99_s": r["query_p99_s"],
            "nnz_per_s_window": nnz_in_window / window_s if window_s > 0 else None,
            "nnz_per_s_kernel": nnz_in_window / gpu_in_window if gpu_in_window > 0 else None,
            "jobs_submitted": r["jobs_submitted"], "jobs_done": r["jobs_done"],
            "jobs_rejected": r["jobs_rejected"], "queries_answered": r["queries_answered"],
            "ticks": r["ticks"]}
    return line


def main():
    a = _args()
    if a.impl == "reference":
        return run_reference(a)
    if a.sweep:
        return run_sweep(a)
    if a.msweep:
        return run_msweep(a)
    if a.order4:
        return run_order4(a)
    if a.batched:
        return run_batched(a)
    if a.serve:
        return run_serve(a)
    return run_gpu(a)


if __name__ == "__main__":
    sys.exit(main())
