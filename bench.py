#!/usr/bin/env python
"""Throughput of the SCD + LP-rounding hot path on one GB300 (or N replicas).

Default workload: the batched configuration -- 4096 independent vertex-cover /
independent-set LPs (ER, n ~ U[200, 20000], average degree ~ U[4, 16], weights
U[1, 10]) whose edge lists are already resident in HBM.  One step = build the
batch on the device (standard form, colouring, layouts), solve every instance
by colour-class SCD on eq. QP to rho <= 1e-3 (each instance in the shared
memory of one CTA, checked and stopped on its own), repair, best-of-10 rounding
and exact validity of every instance.  The metric is solved instances per
second; the line also carries coordinate updates/s, per-instance latency
against the plain one-at-a-time GPU solve, the sweep's roofline and, as extra
keys, the single-instance independent-set figures (Chung-Lu power law,
n = 2^20, m = 1.6e7: coordinate updates/s and time to residual 1e-3).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl thetis|reference]
                  [--workload NAME]

Under torchrun (N > 1) every rank solves its own instances (independent
problems, weak scaling, no collective on the data path); rank 0 prints the
JSON line.  `--impl reference` times the FP64 oracle (the serial CPU
restatement of the method) on host cores for the same workload.
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

WORKLOADS = {
    "is-chunglu-n2^20-m1.6e7": dict(kind="is", graph="chung_lu", n=1 << 20, m=16_000_000, gamma=2.1, seed=2,
                                    beta=100.0, epochs=50, refresh=10, tol=1e-3, reps=10),
    "vc-er-n2000-m8000": dict(kind="vc", graph="er", n=2000, m=8000, seed=1, beta=100.0, epochs=50, refresh=10,
                              tol=1e-3, reps=1),
    "mc-grid1024-k8": dict(kind="mc", graph="grid", width=1024, height=1024, k=8, seed=3, beta=100.0, epochs=50,
                           refresh=10, tol=1e-3, reps=10),
    # set cover (App. B.1): 2^20 elements, each in U[2, 8] of 2^18 random sets, costs U[1, 10];
    # randomized rounding (best of 10, completed to a cover)
    "sc-n2^20-k2^18": dict(kind="sc", graph="setsys", n_elements=1 << 20, n_sets=1 << 18, f_lo=2, f_hi=8, seed=6,
                           beta=100.0, epochs=50, refresh=10, tol=1e-3, reps=10, round=4),
    # pairwise MAP (Sec. 4.1) on a skip-chain-CRF-shaped factor graph the size of the paper's text-chunking
    # LP: 47,000 variables with 23 labels, 24-token sentences, 5 % skip factors (26.2 M columns, 52.3 M non-zeros)
    "map-skipchain-n47k-k23": dict(kind="map", graph="skipchain", n=47_000, k=23, sent_len=24, skip_frac=0.05,
                                   seed=7, beta=100.0, epochs=50, refresh=10, tol=1e-3, reps=1, cpu_sample_n=4700),
    # the IS config under the augmented-Lagrangian outer loop: 5 solves of 50 epochs, multiplier step between
    "al-is-chunglu-n2^20-m1.6e7": dict(kind="is", graph="chung_lu", n=1 << 20, m=16_000_000, gamma=2.1, seed=2,
                                       beta=100.0, epochs=50, refresh=10, tol=0.0, reps=10, al_outer=5),
    # asynchronous mode (Sec. 3.4) vs concurrency: VC on ER n=1e6, avg degree 8, each level solved to rho <= 1e-3
    "async-study-vc-er-n1e6": dict(kind="vc", graph="er", n=1_000_000, m=4_000_000, seed=4, beta=100.0,
                                   epochs=1500, refresh=10, tol=1e-3, reps=1, study=True,
                                   levels=[16, 64, 152, 608, 2432, 0]),
    # 4096 ER instances, half VC half IS, n ~ U[200, 20000], avg degree ~ U[4, 16], weights U[1, 10],
    # all solved to rho <= 1e-3 as one batch
    "batched-4096": dict(kind="batch", count=4096, n_lo=200, n_hi=20000, d_lo=4.0, d_hi=16.0, seed=5, beta=100.0,
                         epochs=4000, refresh=20, tol=1e-3, reps=10, plain_sample=32),
    # the same distribution, 1024 instances (profiling-sized, r larger than L2)
    "batched-1024": dict(kind="batch", count=1024, n_lo=200, n_hi=20000, d_lo=4.0, d_hi=16.0, seed=5, beta=100.0,
                         epochs=4000, refresh=20, tol=1e-3, reps=10, plain_sample=8),
    # the same distribution, 256 instances (profiling-sized)
    "batched-256": dict(kind="batch", count=256, n_lo=200, n_hi=20000, d_lo=4.0, d_hi=16.0, seed=5, beta=100.0,
                        epochs=4000, refresh=20, tol=1e-3, reps=10, plain_sample=8),
    # serving: Poisson arrivals at 2000 req/s of 40% VC / 40% IS (ER, n log-uniform [1e3, 1e6], avg degree
    # U[4, 16]) / 20% MC (k = 4, grid side U[64, 512]); each request to rho <= 1e-3 and rounded; 120 GB budget.
    # One step = one arrival trace of `requests` requests drawn from a pool of `pool` pre-generated graphs.
    "serving-2000rps": dict(kind="serve", rate=2000.0, seconds=60.0, sustain_frac=0.6, pool=40, seed=9, k=4,
                            n_lo=1e3, n_hi=1e6, d_lo=4.0, d_hi=16.0, side_lo=64, side_hi=512, beta=100.0,
                            epochs=5000, refresh=20, tol=1e-3, reps=10, budget=120 << 30, workers=8,
                            max_batch=64, max_queue=256, plain_sample=24),
}
DEFAULT = "batched-4096"
SINGLE = "is-chunglu-n2^20-m1.6e7"  # the single-instance IS config reported beside the default
METRIC = "SCD coord updates/s & time to residual 1e-3; batched solves/s + p99 vs plain"
# DRAM bytes per epoch of the persistent sweep, from an ncu capture of the
# current kernel (profiles/k_sweep_is-chunglu-n2e20.md: one launch of ten
# epochs moved 5.78 GB)
SWEEP_TRAFFIC_PER_EPOCH = {"is-chunglu-n2^20-m1.6e7": 578.0e6}
# DRAM bytes per batched step of the instance kernels (all launch classes),
# from an ncu capture of the current kernels at full size
# (profiles/k_inst_batched-4096_dram.md)
BATCH_TRAFFIC = {"batched-4096": 343.3e9}
L2_BYTES = 129 * 1024 * 1024
SERVE_ORACLE_N_CAP = 20000  # serving requests the oracle baseline samples


def host_cores():
    """Host CPUs this process may run on (its affinity mask), not every CPU of the box."""
    try:
        return len(os.sched_getaffinity(0)) or 1
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_model():
    """The host CPU's model name, from lscpu (or /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                v = line.split(":", 1)[1].strip()
                if v and not v.isdigit():
                    return v
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def make_graph(wl, rank=0):
    from paper_1311_2661_gb300 import synth

    seed = wl["seed"] + 1000 * rank
    if wl["graph"] == "setsys":
        # set cover: the set lists stand in for the edge arrays (eu = set_ptr,
        # ev = set_elems, w = costs; n = sets, m = non-zeros)
        from types import SimpleNamespace

        ss = synth.set_cover_instance(wl["n_elements"], wl["n_sets"], wl["f_lo"], wl["f_hi"], seed)
        return SimpleNamespace(n=ss.n_sets, m=int(ss.ptr[-1]), eu=ss.ptr, ev=ss.elems, w=ss.cost,
                               n_elements=ss.n_elements, terminals=None)
    if wl["graph"] == "skipchain":
        # pairwise MAP: w = node scores, te = factor scores
        from types import SimpleNamespace

        f = synth.skip_chain_crf(wl["n"], wl["k"], wl["sent_len"], wl["skip_frac"], seed)
        return SimpleNamespace(n=f.n, m=f.m, eu=f.eu, ev=f.ev, w=f.theta_node.ravel(), te=f.theta_edge.ravel(),
                               terminals=None)
    if wl["graph"] == "chung_lu":
        g = synth.chung_lu(wl["n"], wl["m"], wl["gamma"], seed)
    elif wl["graph"] == "er":
        g = synth.er_graph(wl["n"], wl["m"], seed)
    else:
        g = synth.grid_graph(wl["width"], wl["height"], wl["k"], seed)
    rng = np.random.default_rng(seed + 17)
    if wl["kind"] == "is":
        g.w = synth.unit_interval_weights(g.n, rng)
    elif wl["kind"] == "vc":
        g.w = synth.int_weights(g.n, 1, 10, rng)
    return g


def algorithmic_bytes_per_epoch(wl, g):
    """Bytes one epoch must move with nothing cached: a structural column j moves
    8 (column pointers) + 4 nnz_j (row ids) + 8 nnz_j (r read + write) + 8 (x read +
    write) + 4 (c_j) = 20 + 12 nnz_j; a slack moves 8 (s) + 8 (r) = 16."""
    n, m = g.n, g.m
    if wl["kind"] in ("vc", "is"):
        return 20 * n + 12 * (2 * m) + 16 * m
    if wl["kind"] == "sc":  # n sets, m non-zeros, one slack per element
        return 20 * n + 12 * m + 16 * g.n_elements
    if wl["kind"] == "map":  # n*k node columns (2mk non-zeros), m*k*k edge columns (2 each), no slacks
        k = wl["k"]
        return 20 * (n * k + m * k * k) + 12 * (2 * m * k + 2 * m * k * k)
    k = wl["k"]
    nfree_blocks = n - k
    deg = np.bincount(np.concatenate([g.eu, g.ev]), minlength=n)
    free = np.ones(n, bool)
    free[g.terminals] = False
    xb = k * (20 * nfree_blocks + 12 * 2 * int(deg[free].sum()))
    zb = m * k * (20 + 12 * 2)
    sb = 16 * 2 * m * k
    return xb + zb + sb


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        if not self.proc:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if args.impl != "reference" else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(v, ws, device=None):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, ws, device=None):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args, wl, ws, rank, local):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1311_2661_gb300 import thetis as T

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    g = make_graph(wl, rank)
    kind = wl["kind"]
    # inputs resident in HBM
    eu_d = torch.from_numpy(g.eu).to(dev)
    ev_d = torch.from_numpy(g.ev).to(dev)
    wt = g.w if kind != "mc" else g.ce
    w_d = torch.from_numpy(wt).to(dev)
    term_d = torch.from_numpy(g.terminals).to(dev) if kind == "mc" else None
    if kind == "map":
        term_d = torch.from_numpy(g.te).to(dev)  # factor scores ride in the terminals slot
    lab_d = torch.zeros(g.n, dtype=torch.uint8, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    def build(eu, ev, w, term):
        if kind == "map":
            return T.thetis_build_map(g.n, wl["k"], eu, ev, w, term, seed=0, stream=stream)
        if kind == "sc":
            return T.thetis_build_sc(g.n_elements, eu, ev, w, seed=0, stream=stream)
        if kind == "vc":
            return T.thetis_build_vc(g.n, eu, ev, w, seed=0, stream=stream)
        if kind == "is":
            return T.thetis_build_is(g.n, eu, ev, w, seed=0, stream=stream)
        return T.thetis_build_mc(g.n, eu, ev, w, wl["k"], term, seed=0, stream=stream)

    shape = {}

    def step(eu, ev, w, term, out, epochs=wl["epochs"], tol=wl["tol"]):
        h = build(eu, ev, w, term)
        # launch shape: timed trials on the first handle of this shape, cached afterwards
        shape["small_group"], shape["ctas_per_sm"] = T.thetis_autotune(h, beta=wl["beta"])
        if wl.get("al_outer"):
            # augmented-Lagrangian outer loop (Sec. 3.4): al_outer solves of `epochs` epochs each
            info, hist = h.solve_al(beta=wl["beta"], epochs=epochs, tol=tol, refresh_every=wl["refresh"],
                                    outer=wl["al_outer"])
            info["al_infeas"] = hist["infeas"].tolist()
            info["al_obj"] = hist["obj"].tolist()
        else:
            info = h.solve(beta=wl["beta"], epochs=epochs, tol=tol, refresh_every=wl["refresh"])
        lab, rinfo = h.round(kind=wl.get("round"), seed=11, reps=wl["reps"], out=out)
        assert rinfo["valid"], "rounded solution failed the exact validity check"
        h.close()
        return info, rinfo

    # warm-up
    for _ in range(args.warmup):
        step(eu_d, ev_d, w_d, term_d, lab_d)
    torch.cuda.synchronize()

    # timed region: device events around every step, L2 flushed between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    l0 = T.thetis_launch_count()
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
                ev[i][0].record(stream)
            infos.append(step(eu_d, ev_d, w_d, term_d, lab_d))
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    launches = T.thetis_launch_count() - l0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), ws, dev)
    updates = sum(i[0]["updates"] for i in infos)
    updates_all = sum_over_ranks(float(updates), ws, dev)
    value = updates_all / (total_ms / 1e3)

    # roofline of the dominant kernel (the colour-class step, one epoch graph)
    bpe = algorithmic_bytes_per_epoch(wl, g)
    ep_ms = sum(i[0]["epoch_ms"] for i in infos)
    ep_n = sum(i[0]["epochs_run"] for i in infos)
    achieved = bpe * ep_n / (ep_ms / 1e3) / 1e9
    pk, pk_kind = peaks()

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    eu_h = torch.from_numpy(g.eu).pin_memory()
    ev_h = torch.from_numpy(g.ev).pin_memory()
    w_h = torch.from_numpy(wt).pin_memory()
    term_h = torch.from_numpy(g.terminals).pin_memory() if kind == "mc" else None
    if kind == "map":
        term_h = torch.from_numpy(g.te).pin_memory()
    lab_h = torch.zeros(g.n, dtype=torch.uint8).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    e_ms = 0.0
    e_upd = 0
    for i in range(e2e_steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(i))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        info, _ = step(eu_h, ev_h, w_h, term_h, lab_h)
        b.record(stream)
        b.synchronize()
        e_ms += a.elapsed_time(b)
        e_upd += info["updates"]
    e_ms = max_over_ranks(e_ms, ws, dev)
    e_upd_all = sum_over_ranks(float(e_upd), ws, dev)
    h2d = g.eu.nbytes + g.ev.nbytes + wt.nbytes + (g.terminals.nbytes if kind == "mc" else 0) + \
        (g.te.nbytes if kind == "map" else 0)

    # time to residual 1e-3 (same pipeline, epochs until rho <= 1e-3)
    ttr = None
    if args.ttr_epochs > 0 and not wl.get("al_outer"):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        info, _ = step(eu_d, ev_d, w_d, term_d, lab_d, epochs=args.ttr_epochs, tol=1e-3)
        b.record(stream)
        b.synchronize()
        ttr = {"ms": a.elapsed_time(b), "epochs": info["epochs_run"], "rho": info["rho"],
               "converged": info["converged"], "solve_ms": info["solve_ms"]}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, g, args.cpu_epochs)

    info0 = infos[-1][0]
    res = {
        "metric": METRIC,
        "value": value,
        "unit": "coord_updates/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (FP64 refresh/checks)",
        "data": "synthetic (seeded Chung-Lu / ER / grid stand-ins for the paper's graphs)",
        "config": {"workload": args.workload, "kind": kind, "n": g.n, "m": g.m,
                   "free_coords": infos[-1][0]["updates"] // max(1, infos[-1][0]["epochs_run"]),
                   "colors": info0["ncolors"], "beta": wl["beta"], "epochs": wl["epochs"],
                   "refresh_every": wl["refresh"], "reps": wl["reps"], "parallelism": f"replicas x{ws}",
                   "launch_shape": dict(shape),
                   "l2": "inputs larger than L2 and L2 flushed (2x129 MB write) between steps"},
        "e2e": {"value": e_upd_all / (e_ms / 1e3), "unit": "coord_updates/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": g.n + 64},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": SWEEP_TRAFFIC_PER_EPOCH.get(args.workload),
                     "traffic_unit": "DRAM bytes per epoch",
                     "kernel": "k_sweep (persistent colour sweep); unit = one epoch", "bytes_per_epoch": bpe,
                     "epoch_us": ep_ms / ep_n * 1e3, "peak_kind": f"{pk_kind} hbm_gbs"},
        "cpu_baseline": cpu,
        "time_to_residual": ttr,
        "last_step": {"epochs_run": info0["epochs_run"], "rho": info0["rho"], "obj": info0["obj"],
                      "infeas": info0["infeas"], "solve_ms": info0["solve_ms"],
                      "rounded_obj": infos[-1][1]["obj"], "step_ms": step_ms[-1],
                      "launches_per_epoch": info0["launches_per_epoch"],
                      **({"al_infeas_per_outer": info0["al_infeas"], "al_obj_per_outer": info0["al_obj"]}
                         if "al_infeas" in info0 else {})},
        "clocks": clk.summary(),
    }
    return res


# ---------------------------------------------------------------------------
# batched workload: solves/s and latency against one-at-a-time GPU solves
# ---------------------------------------------------------------------------
def run_batched(args, wl, ws, rank, local):
    """Batched workload: one step = build the batch, launch shape (tuned once per
    shape, cached), solve every instance to rho <= tol, round every instance,
    validate.  Value = solved instances / step time.  Per-instance latency =
    step start -> the instance's LP solution final on the device (it stops on
    its own in the instance-resident engine) and -> its rounded result; the
    plain arm solves a sample of the same instances one at a time."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1311_2661_gb300 import synth
    from paper_1311_2661_gb300 import thetis as T

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    items = synth.batch_instances(wl["count"], wl["n_lo"], wl["n_hi"], wl["d_lo"], wl["d_hi"], 1, 10,
                                  wl["seed"] + 1000 * rank)
    kinds = np.array([T.ROUND_VC if k == "vc" else T.ROUND_IS for k, _ in items], np.uint8)
    noff = np.concatenate([[0], np.cumsum([g.n for _, g in items])]).astype(np.int64)
    eoff = np.concatenate([[0], np.cumsum([g.m for _, g in items])]).astype(np.int64)
    host = dict(kinds=kinds, noff=noff, eoff=eoff,
                eu=np.concatenate([g.eu for _, g in items]).astype(np.int32),
                ev=np.concatenate([g.ev for _, g in items]).astype(np.int32),
                w=np.concatenate([g.w for _, g in items]).astype(np.float32))
    d = {k: torch.from_numpy(v).to(dev) for k, v in host.items()}
    lab_d = torch.zeros(int(noff[-1]), dtype=torch.uint8, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    count = wl["count"]
    bpe_inst = np.array([20 * g.n + 40 * g.m for _, g in items], np.float64)
    coords_inst = np.array([g.n + g.m for _, g in items], np.float64)
    bpe = float(bpe_inst.sum())
    torch.cuda.synchronize()

    shape = {}

    def step(a, out, t_start=None):
        pre = torch.cuda.Event(enable_timing=True)
        h = T.thetis_build_batch(a["kinds"], a["noff"], a["eoff"], a["eu"], a["ev"], a["w"], seed=0, stream=stream)
        if args.launch_shape:
            lanes, cl = (int(v) for v in args.launch_shape.split(","))
            T.thetis_set_batch_shape(h, lanes, cl)
            shape["lanes_per_column"], shape["clusters"] = lanes, cl
        else:
            shape["lanes_per_column"], shape["clusters"] = T.thetis_autotune(h, beta=wl["beta"])  # cached per shape
        pre.record(stream)
        # solve + repair + rounding + validity; each instance is rounded by its
        # own CTA / cluster the moment it stops
        info, lab, obj, status, best = T.thetis_solve_round_batch(h, seed=11, reps=wl["reps"], out=out,
                                                                  beta=wl["beta"], epochs=wl["epochs"],
                                                                  tol=wl["tol"], refresh_every=wl["refresh"])
        info["inst_epochs"], info["inst_rho"] = T.thetis_batch_info(h)
        info["inst_done_ms"] = T.thetis_batch_latency(h)
        assert np.all(status == 1), "a rounded instance failed the validity check"
        info["pre_solve_ms"] = t_start.elapsed_time(pre) if t_start is not None else 0.0
        h.close()
        return info

    for _ in range(args.warmup):
        step(d, lab_d)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    l0 = T.thetis_launch_count()
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(i))
                ev[i][0].record(stream)
            infos.append(step(d, lab_d, ev[i][0]))
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    launches = T.thetis_launch_count() - l0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), ws, dev)
    value = sum_over_ranks(float(count * args.steps), ws, dev) / (total_ms / 1e3)
    updates = sum(float(coords_inst @ i["inst_epochs"]) for i in infos)
    ep_ms = sum(i["epoch_ms"] for i in infos)
    # an instance is swept only until its own rho reaches tol: only its own
    # epochs move its bytes
    moved = sum(float(bpe_inst @ i["inst_epochs"]) for i in infos)
    achieved = moved / (ep_ms / 1e3) / 1e9
    pk, pk_kind = peaks()
    # per-instance latency inside the steps: step start -> the instance's
    # rounded, validated result final on the device
    done = np.concatenate([i["pre_solve_ms"] + i["inst_done_ms"] for i in infos])

    # e2e: host (pinned) inputs, labels back to the host
    hp = {k: torch.from_numpy(v).pin_memory() for k, v in host.items()}
    lab_h = torch.zeros(int(noff[-1]), dtype=torch.uint8).pin_memory()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    step(hp, lab_h)
    b.record(stream)
    b.synchronize()
    e_ms = max_over_ranks(a.elapsed_time(b), ws, dev)

    # plain: the same instances one at a time through the single-instance API,
    # each built, solved to the same rho and rounded (latency = its own time)
    rng = np.random.default_rng(7)
    sample = rng.choice(count, size=min(wl["plain_sample"], count), replace=False)
    lat = []
    for t in sample:
        kind, g = items[t]
        eu_t, ev_t, w_t = (torch.from_numpy(x).to(dev) for x in (g.eu, g.ev, g.w))
        out_t = torch.zeros(g.n, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bld = T.thetis_build_vc if kind == "vc" else T.thetis_build_is
        h = bld(g.n, eu_t, ev_t, w_t, seed=0, stream=stream)
        h.solve(beta=wl["beta"], epochs=wl["epochs"], tol=wl["tol"], refresh_every=wl["refresh"])
        h.round(seed=11, reps=wl["reps"], out=out_t)
        b.record(stream)
        b.synchronize()
        lat.append(a.elapsed_time(b))
        h.close()
    lat = np.array(lat)
    plain_total_s = float(lat.mean()) * count / 1e3  # the whole batch one at a time

    info0 = infos[-1]
    res = {
        "metric": METRIC,
        "value": value,
        "unit": "solves/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (exact fixed-point refresh, FP64 checks)",
        "data": "synthetic (seeded ER instances)",
        "config": {"workload": args.workload, "instances": count, "sum_n": int(noff[-1]), "sum_m": int(eoff[-1]),
                   "colors": info0["ncolors"], "beta": wl["beta"], "tol": wl["tol"],
                   "refresh_every": wl["refresh"], "reps": wl["reps"], "parallelism": f"replicas x{ws}",
                   "engine": "instance-resident (one CTA per instance, r and x in shared memory)",
                   "launch_shape": dict(shape),
                   "l2": "inputs larger than L2 and L2 flushed (2x129 MB write) between steps"},
        "coord_updates_per_s": sum_over_ranks(updates, ws, dev) / (total_ms / 1e3),
        "e2e": {"value": count / (e_ms / 1e3), "unit": "solves/s",
                "h2d_bytes_per_step": int(sum(v.nbytes for v in host.values())), "d2h_bytes_per_step": int(noff[-1])},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": BATCH_TRAFFIC.get(args.workload),
                     "traffic_unit": "DRAM bytes per step (all launch classes)",
                     "kernel": "k_inst (instance-resident sweep + in-kernel checks); unit = each instance's own "
                               "epochs, algorithmic bytes 20 n + 40 m per instance epoch",
                     "bytes_per_epoch_all_instances": bpe, "bytes_per_step": moved / len(infos),
                     "device_ms_per_step": ep_ms / len(infos), "peak_kind": f"{pk_kind} hbm_gbs",
                     "note": "r and x stay in shared memory: DRAM moves far fewer bytes than the algorithmic "
                             "count (see traffic); frac is algorithmic bytes over time, not DRAM bandwidth"},
        "latency": {"instance_p50_ms": float(np.percentile(done, 50)),
                    "instance_p99_ms": float(np.percentile(done, 99)),
                    "batch_step_ms": float(np.percentile(step_ms, 50)),
                    "plain_p50_ms": float(np.percentile(lat, 50)), "plain_p99_ms": float(np.percentile(lat, 99)),
                    "plain_solves_per_s": float(1e3 / lat.mean()), "plain_sample": int(len(lat)),
                    "plain_whole_batch_s": plain_total_s,
                    "note": "instance: step start (batch submitted) -> the instance's rounded and validated "
                            "result final on the device (instances stop and round independently); plain: one "
                            "instance at a time (build + solve + round), its own latency"},
        "last_step": {"epochs_run_max": info0["epochs_run"], "epochs_mean": float(np.mean(info0["inst_epochs"])),
                      "rho_max": info0["rho"], "converged": info0["converged"], "solve_ms": info0["solve_ms"],
                      "step_ms": step_ms[-1], "pre_solve_ms": info0["pre_solve_ms"]},
        "clocks": clk.summary(),
        "cpu_baseline": None,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        order = np.random.default_rng(7).permutation(count)
        res["cpu_baseline"] = cpu_baseline_instances(wl, items, order, 15.0, "random instances of the batch")
    return res


def run_async_study(args, wl, ws, rank, local):
    """Convergence of the asynchronous scheme (Sec. 3.4: every coordinate at
    once, atomic residual updates) against its concurrency -- at most `L` CTAs of
    256 threads stepping at a time -- beside the colour-class sweep, each run
    from the same start to rho <= tol.  The value is the coordinate-update rate
    of the uncapped asynchronous solve."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1311_2661_gb300 import thetis as T

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    g = make_graph(wl, rank)
    eu, ev, w = (torch.from_numpy(a).to(dev) for a in (g.eu, g.ev, g.w))
    bpe = algorithmic_bytes_per_epoch(wl, g)
    kw = dict(beta=wl["beta"], epochs=wl["epochs"], tol=wl["tol"], refresh_every=wl["refresh"])

    def solve(**extra):
        # every run from the same start: a fresh handle (x = 0, slacks 0); build time is not in solve_ms
        h = T.thetis_build_vc(g.n, eu, ev, w, seed=0, stream=stream)
        info = h.solve(**kw, **extra)
        h.close()
        torch.cuda.synchronize()
        return info

    for _ in range(args.warmup):
        solve(mode=T.MODE_ASYNC)
    l0 = T.thetis_launch_count()
    barrier(ws)
    infos = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            infos.append(solve(mode=T.MODE_ASYNC))
    launches = T.thetis_launch_count() - l0
    total_ms = max_over_ranks(sum(i["solve_ms"] for i in infos), ws, dev)
    updates = sum_over_ranks(float(sum(i["updates"] for i in infos)), ws, dev)
    study = []
    for L in wl["levels"]:
        i = solve(mode=T.MODE_ASYNC, async_ctas=L)
        study.append({"ctas": L if L else "all", "epochs": i["epochs_run"], "converged": i["converged"],
                      "rho": i["rho"], "solve_ms": i["solve_ms"], "ms_per_epoch": i["epoch_ms"] / max(i["epochs_run"], 1),
                      "updates_per_s": i["updates"] / (i["solve_ms"] / 1e3)})
    col = solve()
    pk, pk_kind = peaks()
    ep_ms = sum(i["epoch_ms"] for i in infos)
    ep_n = sum(i["epochs_run"] for i in infos)
    achieved = bpe * ep_n / (ep_ms / 1e3) / 1e9
    res = {
        "metric": METRIC, "value": updates / (total_ms / 1e3), "unit": "coord_updates/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 refresh/checks)",
        "data": "synthetic (seeded ER graph)",
        "config": {"workload": args.workload, "kind": "vc", "n": g.n, "m": g.m, "beta": wl["beta"], "tol": wl["tol"],
                   "mode": "async, uncapped", "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2; each step a full solve to tol"},
        "e2e": None,
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": None,
                     "kernel": "k_color_step (async: all units per class launch, atomic r)",
                     "bytes_per_epoch": bpe, "peak_kind": f"{pk_kind} hbm_gbs"},
        "async_study": study,
        "colored": {"epochs": col["epochs_run"], "solve_ms": col["solve_ms"], "rho": col["rho"],
                    "ms_per_epoch": col["epoch_ms"] / max(col["epochs_run"], 1)},
        "clocks": clk.summary(),
        "cpu_baseline": None,
    }
    if rank == 0:
        print(json.dumps(res), flush=True)


def _serving_inputs(wl, rank):
    from paper_1311_2661_gb300 import synth

    pool = synth.serving_pool(wl["pool"], wl["seed"] + 1000 * rank, wl["n_lo"], wl["n_hi"], wl["d_lo"], wl["d_hi"],
                              wl["side_lo"], wl["side_hi"], wl["k"])
    return pool, [k for k, _ in pool]


def _request_bytes(kind, g):
    """Host bytes a request carries in (edge list + weights) and out (labels + x)."""
    if kind == "mc":
        k = len(g.terminals)
        return 8 * g.m + 4 * g.m + 4 * k, g.n + 4 * g.n * k
    return 8 * g.m + 4 * g.n, g.n + 4 * g.n


def run_serving(args, wl, ws, rank, local):
    """Open-loop serving at two load points, each for `seconds` (>= 60 s by
    default) after a warm-up: Poisson arrivals at the workload's 2000 req/s
    (far above capacity: the server sheds load beyond `max_queue` waiting
    requests, and the completed requests per second measure its capacity), then
    at a sustainable rate (a fraction of that capacity: nothing is shed).
    Requests are submitted to the request server as they arrive; latency is
    arrival -> poll returning the result.  The plain arm serves a sample of the
    same requests one at a time (build + solve + round + read-back through the
    single-instance API); its latency is its service time alone."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1311_2661_gb300 import synth
    from paper_1311_2661_gb300 import thetis as T

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pool, kinds = _serving_inputs(wl, rank)
    bpe = [algorithmic_bytes_per_epoch({"kind": k, "k": wl["k"]}, g) for k, g in pool]
    solve_kw = dict(beta=wl["beta"], epochs=wl["epochs"], tol=wl["tol"], refresh_every=wl["refresh"])
    seconds = args.serve_seconds if args.serve_seconds > 0 else wl["seconds"]

    def trace(rate, dur, salt):
        cnt = int(rate * dur * 1.2) + 16
        t_arr, idx = synth.poisson_trace(rate, cnt, kinds, wl["seed"] * 7919 + 31 * salt + rank)
        keep = t_arr < dur
        return t_arr[keep], idx[keep]

    def serve(sv, t_arr, idx):
        pending, lat, infos = {}, [], []
        shed = 0
        i, n = 0, len(t_arr)
        t0 = time.perf_counter()
        while i < n or pending:
            now = time.perf_counter() - t0
            while i < n and t_arr[i] <= now:
                kind, g = pool[idx[i]]
                try:
                    rid = sv.submit(kind, g, seed=11, reps=wl["reps"], **solve_kw)
                    pending[rid] = (t_arr[i], int(idx[i]))
                except T.ThetisError as e:
                    if e.status != T.THETIS_E_BUDGET:
                        raise
                    shed += 1
                i += 1
            got = False
            for rid in list(pending):
                r = sv.poll(rid)
                if r is None:
                    continue
                got = True
                done = time.perf_counter() - t0
                ta, j = pending.pop(rid)
                info = r[2]
                info["pool"] = j
                info["t_done"] = done
                lat.append(done - ta)
                infos.append(info)
            if not got:
                time.sleep(0.0002)
        return np.array(lat), time.perf_counter() - t0, infos, shed

    def point(sv, rate, dur, salt):
        t_arr, idx = trace(rate, dur, salt)
        lat, wall, infos, shed = serve(sv, t_arr, idx)
        in_window = sum(1 for i in infos if i["t_done"] <= dur)
        bad = [i for i in infos if i["status"] != T.THETIS_OK or not i["valid"]]
        bs = np.array([i["batch_size"] for i in infos]) if infos else np.zeros(1)
        moved = sum(bpe[i["pool"]] * i["epochs_run"] for i in infos)
        return {"offered_rate_per_s": rate, "seconds": dur, "arrivals": int(len(t_arr)), "shed": int(shed),
                "completed": len(infos), "completed_per_s_in_window": in_window / dur,
                "throughput_per_s": len(infos) / wall, "wall_s": wall,
                "p50_ms": float(np.percentile(lat, 50) * 1e3) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99) * 1e3) if len(lat) else None,
                "mean_batch": float(bs.mean()), "not_converged_or_invalid": len(bad),
                "algorithmic_gbs": moved / wall / 1e9,
                "bytes_in": sum(_request_bytes(*pool[i["pool"]])[0] for i in infos),
                "bytes_out": sum(_request_bytes(*pool[i["pool"]])[1] for i in infos)}

    sv = T.Server(budget_bytes=wl["budget"], workers=wl["workers"], max_batch=wl["max_batch"])
    sv.set_queue_limit(wl["max_queue"])
    for s_ in range(args.warmup):
        serve(sv, *trace(wl["rate"], 1.0, 1000 + s_))
    torch.cuda.synchronize()
    l0 = T.thetis_launch_count()
    barrier(ws)
    with ClockSampler(local) as clk:
        over = point(sv, wl["rate"], seconds, 0)
        capacity = max(over["completed_per_s_in_window"], 1.0)
        sus = point(sv, wl["sustain_frac"] * capacity, seconds, 1)
        torch.cuda.synchronize()
    barrier(ws)
    launches = T.thetis_launch_count() - l0
    sv.close()
    value = sum_over_ranks(over["completed_per_s_in_window"], ws, dev)
    pk, pk_kind = peaks()

    # plain: a sample of the requests one at a time, each its own latency
    rng = np.random.default_rng(5)
    sample = rng.choice(len(pool), size=min(wl["plain_sample"], len(pool)), replace=False)
    plain_lat = []
    t0 = time.perf_counter()
    for j in sample:
        kind, g = pool[j]
        a = time.perf_counter()
        if kind == "mc":
            h = T.thetis_build_mc(g.n, g.eu, g.ev, g.ce, len(g.terminals), g.terminals, seed=11)
        else:
            h = (T.thetis_build_vc if kind == "vc" else T.thetis_build_is)(g.n, g.eu, g.ev, g.w, seed=11)
        h.solve(**solve_kw)
        lab, rinfo = h.round(seed=11, reps=wl["reps"])
        h.get_x()
        h.close()
        assert rinfo["valid"], "plain path: invalid rounded solution"
        plain_lat.append(time.perf_counter() - a)
    plain_wall = time.perf_counter() - t0
    plain_lat = np.array(plain_lat)

    res = {
        "metric": METRIC,
        "value": value,
        "unit": "solves/s",
        "n_gpus": ws,
        "steps": 1,
        "warmup": args.warmup,
        "ms_per_step": over["wall_s"] * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (exact fixed-point refresh, FP64 checks)",
        "data": "synthetic (seeded ER + grid pool, Poisson arrival trace)",
        "config": {"workload": args.workload, "rate_per_s": wl["rate"], "seconds_per_point": seconds,
                   "pool": wl["pool"], "pool_sum_n": int(sum(g.n for _, g in pool)),
                   "pool_sum_m": int(sum(g.m for _, g in pool)), "mix": "40% VC / 40% IS / 20% MC k=4",
                   "tol": wl["tol"], "beta": wl["beta"], "refresh_every": wl["refresh"], "reps": wl["reps"],
                   "budget_bytes": wl["budget"], "workers": wl["workers"], "max_batch": wl["max_batch"],
                   "max_queue": wl["max_queue"], "parallelism": f"replicas x{ws}",
                   "l2": "per-request inputs; the pool (>1 GB) is larger than L2; no flush",
                   "timing": "host wall clock, arrival -> result"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": int(over["bytes_in"]),
                "d2h_bytes_per_step": int(over["bytes_out"]),
                "note": "the server takes host arrays: value is already end to end"},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": over["algorithmic_gbs"], "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": over["algorithmic_gbs"] / pk["hbm_gbs"], "traffic": None,
                     "kernel": "all solves of the overload point; algorithmic bytes of every request's epochs / "
                               "wall time", "peak_kind": f"{pk_kind} hbm_gbs"},
        "overload": over,
        "sustained": sus,
        "latency": {"p50_ms": sus["p50_ms"], "p99_ms": sus["p99_ms"],
                    "overload_p50_ms": over["p50_ms"], "overload_p99_ms": over["p99_ms"],
                    "plain_p50_ms": float(np.percentile(plain_lat, 50) * 1e3),
                    "plain_p99_ms": float(np.percentile(plain_lat, 99) * 1e3),
                    "plain_solves_per_s": float(len(plain_lat) / plain_wall), "plain_sample": int(len(plain_lat)),
                    "note": "p50/p99: the sustainable point (arrival -> result); plain: service time of one "
                            "request at a time, no queueing"},
        "clocks": clk.summary(),
        "cpu_baseline": None,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        small = [int(j) for j in trace(wl["rate"], 1.0, 0)[1] if pool[j][1].n <= SERVE_ORACLE_N_CAP]
        res["cpu_baseline"] = cpu_baseline_instances(
            wl, pool, small, 15.0, f"requests of the trace with n <= {SERVE_ORACLE_N_CAP} (the oracle needs minutes "
                                   f"for the largest)")
    if rank == 0:
        print(json.dumps(res), flush=True)


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def _oracle_setup(wl, g):
    import oracle

    oracle.build()
    if wl["kind"] == "sc":
        lp = oracle.OracleLP.set_cover(g.n_elements, g.eu, g.ev, g.w.astype(np.float64))
    elif wl["kind"] == "map":
        lp = oracle.OracleLP.map_lp(g.n, wl["k"], g.eu, g.ev, g.w.astype(np.float64), g.te.astype(np.float64))
    else:
        lp = oracle.build_problem(wl["kind"], g)
    col, nc = lp.color(0)
    return lp, col


def cpu_baseline(wl, g, epochs):
    """The FP64 oracle on one host core: `epochs` SCD epochs of the same
    instance (standard-form build and colouring are setup, not timed) -- or,
    where the workload names `cpu_sample_n`, of a smaller instance of the same
    generator (the oracle's serial colouring of the full one takes minutes)."""
    what = "the full instance"
    if wl.get("cpu_sample_n"):
        g = make_graph(dict(wl, n=wl["cpu_sample_n"]), 0)
        what = f"an instance of the same generator with n = {wl['cpu_sample_n']}"
    lp, col = _oracle_setup(wl, g)
    t = time.perf_counter()
    x, info = lp.solve(beta=wl["beta"], epochs=epochs, refresh_every=wl["refresh"], color=col)
    dt = time.perf_counter() - t
    return {"value": epochs * lp.free_coords / dt, "unit": "coord_updates/s", "cores": 1, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{epochs} FP64 serial SCD epochs of {what} ({lp.free_coords} coordinates) "
                      f"incl. the final exact refresh + checks; build and colouring excluded",
            "seconds": dt}


def _oracle_solve_round(kind, g, wl, seed=11):
    """Build, colour, solve to rho <= tol and round one instance on the oracle."""
    import oracle

    lp = oracle.build_problem(kind, g)
    col, _ = lp.color(seed)
    x, _ = lp.solve(beta=wl["beta"], epochs=wl["epochs"], tol=wl["tol"], refresh_every=wl["refresh"], color=col)
    if kind == "vc":
        lp.round_vc(x[: g.n])
    elif kind == "is":
        lp.round_is(x[: g.n], seed, wl["reps"])
    else:
        lp.round_mc(x[: g.n * len(g.terminals)], seed, wl["reps"])


def cpu_baseline_instances(wl, items, order, seconds, what):
    """The oracle solving the instances in `order` (each built, coloured, solved
    to rho <= tol and rounded), one instance per process on every host core,
    for about `seconds`.  The pool is spawned, so it is safe after GPU work."""
    import multiprocessing as mp

    cores = host_cores()
    jobs = [(items[j][0], items[j][1], wl) for j in order]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as P:
        P.map(_oracle_request, jobs[:cores], chunksize=1)  # warm-up: imports and oracle build in every worker
        rest = jobs[cores:] or jobs
        done, t0 = 0, time.perf_counter()
        for _ in P.imap_unordered(_oracle_request, rest, chunksize=1):
            done += 1
            if time.perf_counter() - t0 >= seconds:
                break
        dt = time.perf_counter() - t0
        P.terminate()
    return {"value": done / dt, "unit": "solves/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": f"{done} {what}, each built, coloured, solved to rho <= {wl['tol']} and rounded by the FP64 "
                      f"oracle, one process per core ({dt:.1f} s)"}


def run_reference_batch(args, wl, ws):
    """The oracle solving instances of the batch, each to rho <= tol plus
    rounding, one instance per process on every host core; one step = four
    instances per core, all steps streamed through the pool."""
    import multiprocessing as mp

    from paper_1311_2661_gb300 import synth

    items = synth.batch_instances(wl["count"], wl["n_lo"], wl["n_hi"], wl["d_lo"], wl["d_hi"], 1, 10, wl["seed"])
    rng = np.random.default_rng(7)
    order = rng.permutation(len(items))
    cores = host_cores()
    jobs = [(items[j][0], items[j][1], wl) for j in order]
    per_step = 4 * cores  # one step = four instances per core, streamed so no core waits for a step's slowest
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as P:
        P.map(_oracle_request, jobs[:cores], chunksize=1)  # warm-up: imports and oracle build in every worker
        warm = [jobs[(cores + q) % len(jobs)] for q in range(args.warmup * per_step)]
        for _ in P.imap_unordered(_oracle_request, warm, chunksize=1):
            pass
        pos = cores + len(warm)
        timed = [jobs[(pos + q) % len(jobs)] for q in range(args.steps * per_step)]
        t = time.perf_counter()
        for _ in P.imap_unordered(_oracle_request, timed, chunksize=1):
            pass
        dt = time.perf_counter() - t
    done = len(timed)
    walls = [dt / args.steps] * args.steps
    value = done / sum(walls)
    sample = (f"{done} instances of the batch, each built, coloured, solved to rho <= {wl['tol']} and rounded by "
              f"the FP64 oracle, one process per core")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(walls) / len(walls) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "instances": wl["count"]},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(), "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def _oracle_request(job):
    """One serving request on the oracle (runs in a spawned worker process)."""
    import oracle

    kind, g, wl = job
    oracle.build()
    t = time.perf_counter()
    _oracle_solve_round(kind, g, wl)
    return time.perf_counter() - t


def run_reference_serving(args, wl, ws):
    """The oracle serving the request mix offline on every host core (one
    request per process).  Bounded sample: requests of the arrival trace whose
    graph has at most `n_cap` vertices (the oracle needs minutes for the largest
    ones); one step = one request per core."""
    import multiprocessing as mp

    from paper_1311_2661_gb300 import synth

    n_cap = SERVE_ORACLE_N_CAP
    pool, kinds = _serving_inputs(wl, 0)
    t_arr, idx = synth.poisson_trace(wl["rate"], 4096, kinds, wl["seed"] * 7919)
    small = [int(j) for j in idx if pool[j][1].n <= n_cap]
    cores = host_cores()
    jobs = [(pool[j][0], pool[j][1], wl) for j in small]
    ctx = mp.get_context("spawn")
    walls, done = [], 0
    with ctx.Pool(cores) as P:
        P.map(_oracle_request, jobs[:cores])  # warm-up: imports and oracle build in every worker
        pos = cores
        for s in range(args.warmup + args.steps):
            batch = [jobs[(pos + q) % len(jobs)] for q in range(cores)]
            pos += cores
            t = time.perf_counter()
            P.map(_oracle_request, batch, chunksize=1)
            dt = time.perf_counter() - t
            if s >= args.warmup:
                walls.append(dt)
                done += len(batch)
    value = done / sum(walls)
    sample = (f"{done} requests of the arrival trace with n <= {n_cap} (VC/IS/MC mix of the trace), each built, "
              f"coloured, solved to rho <= {wl['tol']} and rounded by the FP64 oracle, one process per core")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(walls) / len(walls) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n_cap": n_cap},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "cpu": cpu_model(), "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_reference(args, wl, ws, rank):
    if rank != 0:
        return
    if wl["kind"] == "batch":
        return run_reference_batch(args, wl, ws)
    if wl["kind"] == "serve":
        return run_reference_serving(args, wl, ws)
    g = make_graph(dict(wl, n=wl["cpu_sample_n"]) if wl.get("cpu_sample_n") else wl, 0)
    lp, col = _oracle_setup(wl, g)
    x = lp.initial_x()
    times = []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        x, info = lp.solve(beta=wl["beta"], epochs=1, refresh_every=wl["refresh"], color=col, x0=x)
        dt = time.perf_counter() - t
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = len(times) * lp.free_coords / total
    sample = (f"1 FP64 serial SCD epoch of the full instance per step ({lp.free_coords} coordinates, incl. the "
              f"exact refresh + checks); build and colouring untimed")
    res = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "coord_updates/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total / len(times) * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "kind": wl["kind"], "n": g.n, "m": g.m},
        "cpu_baseline": {"value": value, "unit": "coord_updates/s", "cores": 1, "kind": "oracle", "cpu": cpu_model(), "sample": sample},
        "e2e": {"value": value, "unit": "coord_updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(res), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="thetis", choices=["thetis", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS))
    ap.add_argument("--ttr-epochs", type=int, default=3000, help="epoch cap of the time-to-residual run (0: skip)")
    ap.add_argument("--cpu-epochs", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-single", action="store_true", help="batched default: skip the single-instance extra keys")
    ap.add_argument("--serve-seconds", type=float, default=0.0, help="serving: seconds per load point (0: workload's)")
    ap.add_argument("--launch-shape", default="",
                    help="batched: 'lanes,clusters' instead of the autotuned shape (e.g. to profile the shape "
                         "an unprofiled run chose: the tuner's timings mean nothing under a profiler)")
    args = ap.parse_args()
    ws, rank, local = dist_setup(args)
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl, ws, rank)
    elif wl["kind"] == "batch":
        res = run_batched(args, wl, ws, rank, local)
        if args.workload == DEFAULT and not args.no_single:
            # the single-instance figures of the IS config (coordinate updates/s,
            # time to residual 1e-3, its sweep roofline) ride along as extra keys
            import copy

            a1 = copy.copy(args)
            a1.workload, a1.steps, a1.warmup = SINGLE, max(3, min(args.steps, 5)), 3
            one = run_gpu(a1, WORKLOADS[SINGLE], ws, rank, local)
            res["single_instance"] = {k: one[k] for k in ("metric", "value", "unit", "ms_per_step", "config", "e2e",
                                                          "roofline", "time_to_residual", "last_step",
                                                          "cpu_baseline", "clocks") if k in one}
        if rank == 0:
            print(json.dumps(res), flush=True)
    elif wl["kind"] == "serve":
        run_serving(args, wl, ws, rank, local)
    elif wl.get("study"):
        run_async_study(args, wl, ws, rank, local)
    else:
        res = run_gpu(args, wl, ws, rank, local)
        if rank == 0:
            print(json.dumps(res), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
