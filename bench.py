"""Benchmark of the short-range non-bonded path (one JSON line on stdout).

Default workload: the 96,000-atom SPC/E water box (Ewald real space, rc 1.0 nm,
rlist 1.1 nm) run as an MD-like loop: every step evaluates forces, energies
and the virial from the inner list, re-prunes half of the outer list (rolling
prune over 2 parts) and advances positions ballistically; every 100 steps the
grid sort and the pair search rebuild the outer list.  `value` is steps (force
evaluations) per second on the device, each step charged 1/100 of one timed list
rebuild; `e2e` the same through the public API with positions copied in from
pinned host memory and forces/energies copied out every step.  Extra workloads
(batched replicas, forward + adjoint, the complete Ewald sum, the argon sweep,
the 648-atom box's latency and the 1.5M-atom box) are reported under "extra".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference arm) on the same
workload and metric.  Under torchrun each rank evaluates its own independent
copy of the workload (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "force-evals/s plain vs batched vs fwd+adjoint; %FP32 peak; RMS rel err≤1e-5"
UNIT = "force-evals/s"
NSTLIST = 100
N_PARTS = 2
TRACE_EVERY = 4  # force launches timed with CUDA events in the timed loop: every 4th
DT = 0.002  # ps

# FP32 operations per effective pair interaction (inside rc) by flavour, counted
# from the pair formulas: distance 8, 1/r and powers 4,
# LJ force 5, Coulomb force (Ewald rational 29 / reaction field 5), scalar sum 1,
# force vector 3 and the i/j accumulation 6; energies add LJ 4, Coulomb (Ewald
# exp*rational 16 / RF 8), accumulation 2; the virial adds 2 per pair (amortised).
FLOPS_PER_PAIR = {
    ("ewald", "F"): 56, ("ewald", "FE"): 78, ("ewald", "FEV"): 80,
    ("rf", "F"): 32, ("rf", "FE"): 46, ("rf", "FEV"): 48,
}
# The roofline's algorithmic work per effective interaction: the method's force
# terms only, LJ 12 + Ewald 20 + distance/mask 9 + force update 12 (the exp and
# erfc count as one special-function operation each, off the FP32 pipe; energies and
# the virial are not counted).  The fuller counts above are reported beside it.
FLOPS_PER_PAIR_ROOFLINE = {"ewald": 53, "rf": 41, "none": 33}


# DRAM bytes (read + write) of one k_forces<Ewald, energy, virial> launch on the
# 96k box, from the committed ncu summary of that kernel (the capture named in
# FORCE_KERNEL_CAPTURE); None whenever the force kernel has changed since it was taken.
FORCE_KERNEL_DRAM_BYTES = 7_698_176
# From the same capture: FP32 (FMA) pipe and issue-slot utilisation of that launch,
# in percent of active cycles (what bounds the kernel; None with the bytes above).
FORCE_KERNEL_NCU_PCT = {"fma_pipe": 58.9, "issue_slots": 69.3}
FORCE_KERNEL_CAPTURE = ("profiles/k_forces_spce_water_96k.md, mid-life launch of "
                        "'bench.py --profile --profile-case step --split 24', fused force updates (cold L2, one launch)")


def rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_shard(n_systems: int, rank: int, world: int):
    """Independent systems owned by one rank (round robin; no data exchange between ranks)."""
    return list(range(rank, n_systems, world))


def workload_seed(rank: int) -> int:
    """Each rank evaluates its own copy of the workload, generated from its own seed."""
    return 2 + 1000 * rank


def max_over_ranks(values, device):
    """Element-wise maximum over ranks of a list of floats (timing only; not on the data path)."""
    import torch
    t = torch.tensor(values, dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 20):
        self.gpu = gpu_index
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.interval_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def fp32_peak_tflops(sm_mhz):
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_mhz if sm_mhz else 2070.0
    return sms * 128 * 2 * mhz * 1e6 / 1e12, sms


def l2_flusher(device):
    """Flush L2 between timed iterations: write a 256 MiB buffer (> the 129 MB L2), then
    read another, so that L2 holds none of the workload and no dirty flush lines either
    (their write-back would otherwise land in the next timed step)."""
    import torch
    buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
    buf2 = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)
    sink = torch.empty(1, dtype=torch.float32, device=device)

    def flush():
        buf.fill_(1.0)
        torch.sum(buf2, dim=0, keepdim=True, out=sink)
    return flush


# ----------------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2006_09167_gb300 import api, synth
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    s = synth.water_96k(seed=workload_seed(rank))
    ctx = api.NbContext.from_system(s)
    x0 = torch.tensor(s.x, device=dev)
    v = torch.tensor(synth.maxwell_boltzmann(s, 300.0, seed=7 + rank), dtype=torch.float32, device=dev)
    flush = l2_flusher(dev)
    box = s.box
    from paper_2006_09167_gb300 import autotune
    # the work-item size is autotuned; the prune cadence is the workload's (2 rolling parts)
    tuned = autotune.tune(s, x0, flush=flush)
    ctx.nb_set_split(tuned["split"])
    n_parts = N_PARTS
    ctx.build(x0, box)
    # the timed loop traces every TRACE_EVERY-th force launch only: each traced launch adds
    # two event records to the stream, which cost ~12 us per step when every launch carries
    # them (gather and prune are timed in a loop of their own below)
    f = torch.empty((s.n, 3), dtype=torch.float32, device=dev)
    e = torch.empty(2, dtype=torch.float64, device=dev)
    w = torch.empty(9, dtype=torch.float64, device=dev)
    flags = api.NB_ENERGY | api.NB_VIRIAL
    x = x0.clone()
    # the headline runs in the sorted layout (nb_forces_sorted): between list builds the
    # positions, velocities and forces stay in the context's cluster order, as an MD engine
    # that integrates in its grid order keeps them; a rebuild goes through caller order
    # caller-order arrays with one extra row that the padding slots map to (no boolean indexing,
    # so no host synchronisation): zero velocity there, and a scratch row for positions
    lay = {"v_ext": torch.cat([v, torch.zeros((1, 3), dtype=torch.float32, device=dev)]),
           "x_ext": torch.empty((s.n + 1, 3), dtype=torch.float32, device=dev)}

    def export_sorted():
        ns = ctx.n_slots()
        if lay.get("ns") != ns:
            lay.update(ns=ns, xq=torch.empty((ns, 4), dtype=torch.float32, device=dev),
                       perm=torch.empty(ns, dtype=torch.int32, device=dev),
                       f=torch.empty((ns, 4), dtype=torch.float32, device=dev),
                       v4=torch.zeros((ns, 4), dtype=torch.float32, device=dev))
        ctx.nb_sorted_export(lay["xq"], lay["perm"])
        lay["idx"] = torch.where(lay["perm"] >= 0, lay["perm"], s.n).long()
        # velocities as (vx, vy, vz, 0) per slot: the update is one contiguous add over the slots
        # that leaves the charges (w) and the padding slots as they are
        lay["v4"][:, :3] = lay["v_ext"].index_select(0, lay["idx"])

    def to_caller():
        lay["x_ext"].index_copy_(0, lay["idx"], lay["xq"][:, :3])
        x.copy_(lay["x_ext"][:s.n])

    def rebuild():
        if args.caller_order:
            ctx.build(x, box)
        else:
            to_caller()
            ctx.build(x, box)
            export_sorted()

    def step(t, rebuild_ok=True, fl=flags):
        if rebuild_ok and t % NSTLIST == 0 and t > 0:
            rebuild()
        if args.caller_order:
            ctx.nb_forces(fl, x, f, e, w)
            ctx.nb_prune_rolling(t % n_parts, n_parts)
            x.add_(v, alpha=DT)
        else:
            ctx.nb_forces_sorted(fl, lay["xq"], lay["f"], e, w)
            ctx.nb_prune_rolling(t % n_parts, n_parts)
            lay["xq"].add_(lay["v4"], alpha=DT)

    if not args.caller_order:
        export_sorted()

    ctx.nb_trace_enable(True, kinds=[api.NB_TRACE_FORCES])  # creates the events before timing
    for t in range(args.warmup):
        step(t)
    torch.cuda.synchronize()
    # one list rebuild (grid sort + pair search + first full prune, with the host read-back of
    # the list sizes inside it) timed on its own, L2 flushed: every step of the headline is
    # charged 1/NSTLIST of it, whatever the number of timed steps
    build_ms = []
    for _ in range(5):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        rebuild()
        b.record()
        torch.cuda.synchronize()
        build_ms.append(a.elapsed_time(b))
    # the timed steps start half-way through a list lifetime: the force kernel's time grows with
    # the list's age as the atoms spread, and mid-life is its average
    for t in range(NSTLIST // 2):
        step(t, rebuild_ok=False)
    torch.cuda.synchronize()
    t_off = NSTLIST // 2
    for kind in range(4):
        ctx.nb_trace_read(kind)
    launches0 = ctx.nb_get_stats()["n_launches"]
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    built = []
    for k in range(args.steps):
        flush()  # L2 flushed between timed steps (outside the events)
        ctx.nb_trace_enable(k % TRACE_EVERY == 0, kinds=[api.NB_TRACE_FORCES])
        t = t_off + k
        built.append(t % NSTLIST == 0)
        evs[k][0].record()
        step(t)
        evs[k][1].record()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches = ctx.nb_get_stats()["n_launches"] - launches0
    # algorithmic work of one force launch: the pairs of the list the timed launches used, at the
    # positions of the end of the timed steps (the clock window below moves the atoms further)
    n_eff, n_raw = ctx.nb_count_pairs()
    # clock window: the timed region is a few ms, shorter than the sampling interval, so the
    # same steps keep running (untimed, L2 flushed alike) for a further second of sampling
    ctx.nb_trace_enable(False)
    t_end = time.perf_counter() + 1.0
    k = 0
    while time.perf_counter() < t_end:
        flush()
        step(t_off + args.steps + k)
        k += 1
        if k % 50 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_off += args.steps + k
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    fk_ms, fk_n = ctx.nb_trace_read(api.NB_TRACE_FORCES)
    assert ctx.nb_get_error() == 0, "device error during the timed loop"
    # gather and prune kernel times (reported, not part of the headline): 50 more steps of
    # the same loop, L2 flushed between them as above
    ctx.nb_trace_enable(True, kinds=[api.NB_TRACE_PRUNE, api.NB_TRACE_GATHER])
    for k in range(50):
        flush()
        step(t_off + k)
    pr_ms, pr_n = ctx.nb_trace_read(api.NB_TRACE_PRUNE)
    ga_ms, ga_n = ctx.nb_trace_read(api.NB_TRACE_GATHER)
    ctx.nb_trace_enable(False)
    plain_steps = [m for m, b in zip(step_ms, built) if not b] or step_ms
    res = dict(total_ms=total_ms, step_ms=step_ms, launches=launches, fk_ms=fk_ms, fk_n=fk_n, pr_ms=pr_ms,
               build_ms=float(np.median(build_ms)), step_mean_ms=float(np.mean(plain_steps)),
               step_median_ms=float(np.median(plain_steps)), n_built_in_loop=int(sum(built)),
               pr_n=pr_n, ga_ms=ga_ms, ga_n=ga_n, n_eff=n_eff, n_raw=n_raw, clocks=clk, n_atoms=s.n,
               tuned={"split": int(tuned["split"]), "n_parts": n_parts})
    # end to end through the public API: pinned host positions in, forces + energies out
    xh = torch.empty((s.n, 3), dtype=torch.float32).pin_memory()
    xh.copy_(x.cpu())
    fh = torch.empty((s.n, 3), dtype=torch.float32).pin_memory()
    eh = torch.empty(2, dtype=torch.float64).pin_memory()
    wh = torch.empty(9, dtype=torch.float64).pin_memory()
    xd = torch.empty_like(x)
    vh = v.cpu()
    side = torch.cuda.Stream(device=dev)
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t = 2 * NSTLIST + k
        xd.copy_(xh, non_blocking=True)
        if t % NSTLIST == 0:
            ctx.build(xd, box)
        fo, eo, wo = ctx.forces(xd, energy=True, virial=True)
        # the rolling prune (reads positions and the outer list, writes the inner list) runs on a
        # second stream beside the copy of the results (which reads only the outputs); the step
        # ends when both are done
        side.wait_stream(torch.cuda.current_stream())
        ctx.nb_prune_rolling(t % n_parts, n_parts, stream=side)
        fh.copy_(fo, non_blocking=True)
        eh.copy_(eo, non_blocking=True)
        wh.copy_(wo.view(-1), non_blocking=True)
        torch.cuda.synchronize()
        if k >= args.warmup and t % NSTLIST:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        xh.add_(vh, alpha=DT)
    res["e2e_ms"] = float(np.mean(e2e_ms))
    # a rebuild through the same API (positions copied in, grid sort, search, first prune),
    # host wall clock; charged 1/NSTLIST per step like the device-timed headline
    eb = []
    for _ in range(3):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xd.copy_(xh, non_blocking=True)
        ctx.build(xd, box)
        torch.cuda.synchronize()
        eb.append((time.perf_counter() - t0) * 1e3)
    res["e2e_build_ms"] = float(np.median(eb))
    # context: energies and virial only every 100th step and forces alone otherwise, the cadence
    # MD engines compute them at; the same loop from the same start, device time, L2 flushed
    x.copy_(x0)
    ctx.build(x, box)
    if not args.caller_order:
        export_sorted()
    ev100 = []
    for k in range(args.warmup + args.steps):
        flush()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step(k, fl=flags if k % 100 == 0 else 0)
        b.record()
        if k >= args.warmup:
            ev100.append((a, b))
    torch.cuda.synchronize()
    res["md_e100_ms"] = float(np.mean([a.elapsed_time(b) for a, b in ev100]))
    res["h2d"] = s.n * 3 * 4
    res["d2h"] = s.n * 3 * 4 + 16 + 72
    res["layout"] = "caller order" if args.caller_order else "sorted (nb_forces_sorted)"
    return res


def extra_workloads(args):
    """Batched replicas (plain vs batched vs per-replica graph) and forward + adjoint."""
    import torch
    from paper_2006_09167_gb300 import api, synth
    out = {}
    dev = torch.device("cuda", torch.cuda.current_device())
    # batched: 256 uneven replicas
    reps = synth.replica_set()
    from paper_2006_09167_gb300 import autotune
    flush = l2_flusher(dev)
    xs_tune = [torch.tensor(sysr.x, device=dev) for sysr in reps]
    tuned_b = autotune.tune_batched(reps, xs_tune, splits=(16, 32, 64, 96, 128), reps=5, flush=flush, segments=(0, 1))
    del xs_tune
    ctxs, xs = [], []
    for sysr in reps:
        c = api.NbContext.from_system(sysr)
        c.nb_set_split(tuned_b["split"])
        c.nb_set_search_segments(tuned_b["segments"])
        xr = torch.tensor(sysr.x, device=dev)
        c.build(xr, sysr.box)
        ctxs.append(c)
        xs.append(xr)
    b = api.NbBatch(ctxs)
    xcat = torch.cat(xs).contiguous()
    fcat = torch.empty_like(xcat)
    R = len(ctxs)
    e = torch.empty(2 * R, dtype=torch.float64, device=dev)
    w = torch.empty(9 * R, dtype=torch.float64, device=dev)
    flags = api.NB_ENERGY | api.NB_VIRIAL
    fs = [torch.empty_like(xr) for xr in xs]
    es = [torch.empty(2, dtype=torch.float64, device=dev) for _ in xs]
    ws = [torch.empty(9, dtype=torch.float64, device=dev) for _ in xs]

    def batched():
        b.nb_forces_batched(flags, xcat, fcat, e, w)

    def plain_fn(cs):
        def plain():
            for c, xr, fr, er, wr in zip(cs, xs, fs, es, ws):
                c.nb_forces(flags, xr, fr, er, wr)
        return plain

    def time_fn(fn, reps_=20, warm=3):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps_):
            flush()
            a, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            bb.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(bb))
        return float(np.median(ts))

    def graphed(fn):
        st = torch.cuda.Stream()
        st.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(st):
            fn()
        torch.cuda.current_stream().wait_stream(st)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g

    gb = graphed(batched)
    t_batched_graph = time_fn(gb.replay)
    n_all = sum(c.n for c in ctxs)
    del gb, b, ctxs
    # the per-replica calls at the item size best for them (small systems alone want short items)
    t_plain_graph, split_plain, ctxs_p = None, None, None
    for sp in (8, 16, 32, 64):
        cs = []
        for sysr, xr in zip(reps, xs):
            c = api.NbContext.from_system(sysr)
            c.nb_set_split(sp)
            c.build(xr, sysr.box)
            cs.append(c)
        gp = graphed(plain_fn(cs))
        t = time_fn(gp.replay)
        del gp
        if t_plain_graph is None or t < t_plain_graph:
            t_plain_graph, split_plain, ctxs_p = t, sp, cs
        del cs
    t_plain_seq = time_fn(plain_fn(ctxs_p), reps_=5, warm=1)
    out["batched_256_replicas"] = {
        "atoms_total": int(n_all), "replicas": R, "split_autotuned": int(tuned_b["split"]),
        "search_segments_autotuned": int(tuned_b["segments"]),
        "split_plain_best": int(split_plain),
        "batched_graph_ms": t_batched_graph, "plain_graph_ms": t_plain_graph, "plain_sequential_ms": t_plain_seq,
        "system_evals_per_s_batched": R * 1e3 / t_batched_graph,
        "system_evals_per_s_plain_graph": R * 1e3 / t_plain_graph,
        "system_evals_per_s_plain_sequential": R * 1e3 / t_plain_seq,
    }
    del ctxs_p, xs
    # forward + adjoint on the 24k box with 6 LJ types
    s4 = synth.water_24k_types()
    c4 = api.NbContext.from_system(s4)
    x4 = torch.tensor(s4.x, device=dev)
    c4.build(x4, s4.box)
    T = s4.n_types
    gF = torch.randn((s4.n, 3), device=dev)
    gx = torch.empty_like(x4)
    gq = torch.empty(s4.n, device=dev)
    g6 = torch.empty((T, T), dtype=torch.float64, device=dev)
    g12 = torch.empty_like(g6)
    f4 = torch.empty_like(x4)
    e4 = torch.empty(2, dtype=torch.float64, device=dev)

    def fwd():
        c4.nb_forces(api.NB_ENERGY, x4, f4, e4)

    def fwd_adj():
        c4.nb_forces(api.NB_ENERGY, x4, f4, e4)
        c4.nb_forces_vjp(x4, gF, 0.5, gx, gq, g6, g12)

    t_f = time_fn(graphed(fwd).replay)
    t_fa = time_fn(graphed(fwd_adj).replay)
    out["fwd_adjoint_24k"] = {"n_atoms": s4.n, "forward_ms": t_f, "forward_adjoint_ms": t_fa,
                              "evals_per_s_forward": 1e3 / t_f, "evals_per_s_forward_adjoint": 1e3 / t_fa}
    # the complete Ewald sum on the 96k box: short-range kernel + smooth PME (order 4,
    # 0.12 nm grid) + exclusion and self terms, each timed alone and as one step in a graph
    s2 = synth.water_96k()
    c2 = api.NbContext.from_system(s2)
    x2 = torch.tensor(s2.x, device=dev)
    q2 = torch.tensor(s2.q, device=dev)
    c2.build(x2, s2.box)
    pme = api.NbPme.from_system(s2, spacing=0.12, order=4)
    f2 = torch.empty_like(x2)
    e_sr = torch.empty(2, dtype=torch.float64, device=dev)
    w_sr = torch.empty(9, dtype=torch.float64, device=dev)
    e_rec = torch.empty(1, dtype=torch.float64, device=dev)
    w_rec = torch.empty(9, dtype=torch.float64, device=dev)
    e_cor = torch.empty(2, dtype=torch.float64, device=dev)
    w_cor = torch.empty(9, dtype=torch.float64, device=dev)
    fl = api.NB_ENERGY | api.NB_VIRIAL

    def sr():
        c2.nb_forces(fl, x2, f2, e_sr, w_sr)

    def rec():
        pme.nb_pme_forces(fl, x2, q2, s2.box, f2, e_rec, w_rec)

    def cor():
        c2.nb_ewald_corrections(fl, x2, f2, e_cor, w_cor)

    def full():
        sr()
        rec()
        cor()

    gfull = graphed(full)
    t_sr, t_rec, t_cor = time_fn(sr), time_fn(rec), time_fn(cor)
    t_full = time_fn(gfull.replay)
    out["ewald_full_96k"] = {
        "pme_grid": list(pme.grid), "pme_order": pme.order, "short_range_ms": t_sr, "pme_ms": t_rec,
        "corrections_ms": t_cor, "full_step_graph_ms": t_full, "evals_per_s_full": 1e3 / t_full,
        "kernels_per_step": "gather, k_forces, unsort | memset, spread, FFT R2C (cuFFT), solve, FFT C2R (cuFFT), "
                            "gather | corrections",
    }
    del gfull, pme
    # first use of a new list: separate full prune + force call on the inner list, against
    # the force call that evaluates the outer list and prunes on the way (nb_set_fused_prune)
    def ev_time(fn):
        a, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush()
        a.record()
        fn()
        bb.record()
        torch.cuda.synchronize()
        return a.elapsed_time(bb)

    sep_ms, fus_ms, plain_ms = [], [], []
    cf = api.NbContext.from_system(s2)
    cf.nb_set_fused_prune(True)
    for rep in range(8):
        c2.nb_set_fused_prune(False)
        c2.build(x2, s2.box)
        sep_ms.append(ev_time(lambda: c2.nb_prune_rolling(0, 1)) + ev_time(sr))
        plain_ms.append(ev_time(sr))
        cf.build(x2, s2.box)
        fus_ms.append(ev_time(lambda: cf.nb_forces(fl, x2, f2, e_sr, w_sr)))
    out["first_use_prune_96k"] = {
        "separate_prune_plus_forces_ms": float(np.median(sep_ms[2:])),
        "fused_forces_on_outer_list_ms": float(np.median(fus_ms[2:])),
        "forces_on_inner_list_ms": float(np.median(plain_ms[2:])),
    }
    del c2, cf
    # LJ argon throughput against the number of pairs per particle (the paper's Fig. 6
    # system: 157k atoms, rho 26 nm^-3, sigma 0.3345 nm; force-only, LJ-only kernel)
    sweep = []
    for rc in (0.5, 0.7, 0.9, 1.1, 1.4, 1.8):
        sa = synth.argon_box(157000, seed=11, rc=rc, rlist=rc + 0.1)
        ca = api.NbContext.from_system(sa)
        xa = torch.tensor(sa.x, device=dev)
        ca.build(xa, sa.box)
        fa = torch.empty_like(xa)
        ta = time_fn(lambda: ca.nb_forces(0, xa, fa), reps_=10)
        n_eff, n_raw = ca.nb_count_pairs()
        sweep.append({"rc": rc, "pairs_per_particle_half_sphere": 2.0 * math.pi / 3.0 * 26.0 * rc ** 3,
                      "force_ms": ta, "raw_Gpairs_per_s": n_raw / (ta * 1e-3) / 1e9,
                      "effective_Gpairs_per_s": n_eff / (ta * 1e-3) / 1e9,
                      "work_efficiency": n_eff / max(n_raw, 1)})
        del ca
    out["argon_157k_sweep"] = sweep
    # the 648-atom reaction-field box: latency of one evaluation (forces + energies + virial;
    # gather, force kernel, unsort) issued eagerly and replayed from a CUDA graph
    s1 = synth.water_648()
    c1 = api.NbContext.from_system(s1)
    x1 = torch.tensor(s1.x, device=dev)
    # a tiny system is latency-bound: short work items (more warps, shorter dependent chains
    # of list and position loads per warp) suit it; the item size is autotuned as for the others
    split1 = int(autotune.tune(s1, x1, splits=(4, 8, 12, 16), flush=flush)["split"])
    c1.nb_set_split(split1)
    c1.build(x1, s1.box)
    f1 = torch.empty_like(x1)
    e1 = torch.empty(2, dtype=torch.float64, device=dev)
    w1 = torch.empty(9, dtype=torch.float64, device=dev)

    def ev648():
        c1.nb_forces(flags, x1, f1, e1, w1)
    t1_eager = time_fn(ev648, reps_=200, warm=20)
    g1 = graphed(ev648)
    t1_graph = time_fn(g1.replay, reps_=200, warm=20)
    out["water_648_rf_latency"] = {"n_atoms": s1.n, "split_autotuned": split1, "us_per_eval_eager": 1e3 * t1_eager,
                                   "us_per_eval_graph": 1e3 * t1_graph,
                                   "note": "median of 200 evaluations, CUDA events, L2 flushed between them"}
    del g1, c1
    # the 1.5M-atom heterogeneous box (85% water, 15% polymer, 22 LJ types, rc 1.2 nm):
    # force + energy + virial evaluations from a fresh list
    s3 = synth.polymer_water_box()
    c3 = api.NbContext.from_system(s3)
    x3 = torch.tensor(s3.x, device=dev)
    c3.build(x3, s3.box)
    # a list build (grid sort, pair search, item sort, first prune, with the host read-back of the
    # list sizes), timed alone as for the 96k loop's amortised rebuild
    tb3 = time_fn(lambda: c3.build(x3, s3.box), reps_=3, warm=1)
    f3 = torch.empty_like(x3)
    e3 = torch.empty(2, dtype=torch.float64, device=dev)
    w3 = torch.empty(9, dtype=torch.float64, device=dev)
    t3 = time_fn(lambda: c3.nb_forces(flags, x3, f3, e3, w3), reps_=8, warm=2)
    n_eff, n_raw = c3.nb_count_pairs()
    out["polymer_water_1.5M"] = {"n_atoms": s3.n, "force_ms": t3, "evals_per_s": 1e3 / t3, "list_build_ms": tb3,
                                 "effective_pairs": int(n_eff), "evaluated_pairs": int(n_raw),
                                 "effective_Gpairs_per_s": n_eff / (t3 * 1e-3) / 1e9,
                                 "note": "median of 8 calls (gather + force kernel + unsort), L2 flushed"}
    del c3
    return out


def cpu_oracle_sample(seconds=12.0):
    """The FP64 cell-list oracle on the host cores: full 96k-atom evaluations."""
    import oracle
    from paper_2006_09167_gb300 import synth
    s = synth.water_96k()
    oracle.celllist(s)  # warm-up (page in, thread start)
    n = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds or n == 0:
        oracle.celllist(s)
        n += 1
    dt = time.perf_counter() - t0
    cores = oracle.num_threads()
    # the same on one host core (a shorter sample: one or two evaluations)
    oracle.set_num_threads(1)
    try:
        n1 = 0
        t1 = time.perf_counter()
        while time.perf_counter() - t1 < seconds / 3 or n1 == 0:
            oracle.celllist(s)
            n1 += 1
        dt1 = time.perf_counter() - t1
    finally:
        oracle.set_num_threads(cores)
    return {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} full FP64 cell-list evaluations (forces, energies, virial) of the 96,000-atom box "
                      f"in {dt:.1f} s",
            "single_core_value": n1 / dt1,
            "single_core_sample": f"{n1} evaluations on 1 core in {dt1:.1f} s"}


def main_ours(args):
    import torch
    rank, world, local_rank = rank_env()
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    res = run_ours(args, rank, world, local_rank)
    # the headline step: the mean timed step (forces + energies + virial, half-list rolling
    # prune, position update) plus 1/NSTLIST of one timed list rebuild
    amort = res["step_mean_ms"] + res["build_ms"] / NSTLIST
    e2e_amort = res["e2e_ms"] + res["e2e_build_ms"] / NSTLIST
    ms_per_step, res["e2e_ms"], res["total_ms"] = max_over_ranks([amort, e2e_amort, res["total_ms"]], "cuda")
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    value = world * 1e3 / ms_per_step
    clk = res["clocks"]
    peak, sms = fp32_peak_tflops(clk.get("sm_mhz"))
    fk_avg_ms = res["fk_ms"] / max(res["fk_n"], 1)
    alg_flops = res["n_eff"] * FLOPS_PER_PAIR_ROOFLINE["ewald"]
    achieved = alg_flops / (fk_avg_ms * 1e-3) / 1e12
    achieved_counted = res["n_eff"] * FLOPS_PER_PAIR[("ewald", "FEV")] / (fk_avg_ms * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "spce_water_96k_ewald_rc1.0_rlist1.1 MD-like step: forces+energies+virial, "
                               "rolling prune of 1/2 of the list per step, grid sort + pair search every 100 steps",
                   "e2e_step": "caller atom order through NbContext.forces (gather and scatter included), pinned "
                               "host positions in and forces, energies, virial out every step",
                   "step": "mean of the timed steps without a rebuild (forces+energies+virial, half-list rolling "
                           "prune, position update) + 1/100 of one list rebuild (grid sort + pair search + first "
                           "full prune) timed on its own with CUDA events; steps start half-way through a list "
                           "lifetime",
                   "layout": res["layout"],
                   "step_mean_ms": res["step_mean_ms"], "step_median_ms": res["step_median_ms"],
                   "rebuild_ms": res["build_ms"], "rebuilds_inside_timed_steps": res["n_built_in_loop"],
                   "timed_region_ms": res["total_ms"],
                   "n_atoms": res["n_atoms"], "rc": 1.0, "rlist": 1.1, "r_in": 1.0, "nstlist": NSTLIST,
                   "prune_parts": res["tuned"]["n_parts"], "split": res["tuned"]["split"],
                   "l2": "flushed between timed steps (256 MiB write + 256 MiB read of another buffer, outside the events)",
                   "parallelism": f"replicas{world}"},
        "e2e": {"value": world * 1e3 / res["e2e_ms"], "unit": UNIT, "h2d_bytes_per_step": res["h2d"],
                "d2h_bytes_per_step": res["d2h"]},
        "gpu_launches": int(res["launches"]),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": FORCE_KERNEL_DRAM_BYTES,
                     "traffic_source": FORCE_KERNEL_CAPTURE, "ncu_pct": FORCE_KERNEL_NCU_PCT,
                     "kernel": "k_forces<Ewald, energy, virial>", "avg_launch_ms": fk_avg_ms,
                     "timed_launches": int(res["fk_n"]),
                     "launch_timing": f"CUDA events around every {TRACE_EVERY}th force launch of the timed loop",
                     "effective_pairs_per_launch": int(res["n_eff"]), "evaluated_pairs_per_launch": int(res["n_raw"]),
                     "flops_per_effective_pair": FLOPS_PER_PAIR_ROOFLINE["ewald"],
                     "frac_with_energy_and_virial_flops": achieved_counted / peak,
                     "flops_per_effective_pair_with_energy_and_virial": FLOPS_PER_PAIR[("ewald", "FEV")],
                     "peak_basis": f"{sms} SMs x 128 FP32 lanes x 2 x median SM clock under load"},
        "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"), "reasons": clk.get("reasons"),
                   "samples": clk.get("samples"),
                   "window": "nvidia-smi every 20 ms over the timed steps and one further second of the same steps"},
        "kernels_ms_per_step": {"forces": fk_avg_ms, "prune": res["pr_ms"] / max(res["pr_n"], 1),
                                ("gather" if args.caller_order else "prep_sorted"): res["ga_ms"] / max(res["ga_n"], 1)},
        "pairs_per_s_effective": res["n_eff"] / (fk_avg_ms * 1e-3),
    }
    if not args.no_extra:
        try:
            line["extra"] = extra_workloads(args)
        except Exception as exc:  # report, do not hide the main number
            line["extra"] = {"error": repr(exc)}
        line["extra"]["md_energies_every_100_steps_96k"] = {
            "ms_per_step": res["md_e100_ms"], "steps_per_s": 1e3 / res["md_e100_ms"],
            "note": "the headline loop with energies and virial on every 100th step, forces alone otherwise"}
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle_sample()
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------------------ reference
def main_reference(args):
    """The FP64 oracle as the reference arm: same workload, metric and step definition."""
    rank, world, _ = rank_env()
    if rank != 0:
        return
    import oracle
    from paper_2006_09167_gb300 import synth
    s = synth.water_96k()
    v = synth.maxwell_boltzmann(s, 300.0, seed=7)
    x = s.x.astype(np.float64)
    for t in range(args.warmup):
        oracle.celllist(s, x=x)
        x = x + DT * v
    t0 = time.perf_counter()
    for t in range(args.steps):
        oracle.celllist(s, x=x)
        x = x + DT * v
    dt = time.perf_counter() - t0
    value = args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "spce_water_96k_ewald_rc1.0_rlist1.1 MD-like step: exact FP64 cell-list "
                                   "forces+energies+virial of every step (no pair list to prune)",
                       "n_atoms": s.n, "rc": 1.0, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{args.steps} timed full evaluations of the 96,000-atom box"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main_profile(args):
    """A short, fixed launch sequence for profilers: one build, then force evaluations
    (--profile-case forces: the 96k box; polymer_1.5m: the 1.5M-atom polymer/water box;
    batched: one batched launch over the 256 replicas; vjp: forward + adjoint calls on the
    24k box with 6 LJ types) or PME + Ewald-correction calls (--profile-case pme); step: the
    headline MD step in the sorted layout on the 96k box, NSTLIST/2 untimed steps to reach a
    mid-life list, then warmup + steps more (5 launches per step: prep, forces, energy fold,
    prune, position update)."""
    import torch
    from paper_2006_09167_gb300 import api, synth
    flags = api.NB_ENERGY | api.NB_VIRIAL
    if args.profile_case == "step":
        s = synth.water_96k()
        ctx = api.NbContext.from_system(s)
        ctx.nb_set_split(args.split or 12)
        x = torch.tensor(s.x, device="cuda")
        v = torch.tensor(synth.maxwell_boltzmann(s, 300.0, seed=7), dtype=torch.float32, device="cuda")
        ctx.build(x, s.box)
        xq, perm = ctx.nb_sorted_export()
        idx = torch.where(perm >= 0, perm, s.n).long()
        v4 = torch.zeros_like(xq)
        v4[:, :3] = torch.cat([v, torch.zeros((1, 3), device="cuda")]).index_select(0, idx)
        f = torch.empty_like(xq)
        e = torch.empty(2, dtype=torch.float64, device="cuda")
        w = torch.empty(9, dtype=torch.float64, device="cuda")
        for t in range(NSTLIST // 2 + args.warmup + args.steps):
            ctx.nb_forces_sorted(flags, xq, f, e, w)
            ctx.nb_prune_rolling(t % N_PARTS, N_PARTS)
            xq.add_(v4, alpha=DT)
        torch.cuda.synchronize()
        assert ctx.nb_get_error() == 0
        print(json.dumps({"profile_case": "spce_water_96k_ewald_sorted_step", "launches": ctx.nb_get_stats()["n_launches"],
                          "steps": NSTLIST // 2 + args.warmup + args.steps}))
        return
    if args.profile_case == "batched":
        reps = synth.replica_set()
        ctxs, xs = [], []
        for sysr in reps:
            c = api.NbContext.from_system(sysr)
            c.nb_set_split(args.split or 64)
            c.nb_set_search_segments(1)  # unsegmented lists, as the batched autotuner picks
            xr = torch.tensor(sysr.x, device="cuda")
            c.build(xr, sysr.box)
            ctxs.append(c)
            xs.append(xr)
        b = api.NbBatch(ctxs)
        xcat = torch.cat(xs).contiguous()
        fcat = torch.empty_like(xcat)
        e = torch.empty(2 * len(ctxs), dtype=torch.float64, device="cuda")
        w = torch.empty(9 * len(ctxs), dtype=torch.float64, device="cuda")
        for _ in range(args.warmup + args.steps):
            b.nb_forces_batched(flags, xcat, fcat, e, w)
        torch.cuda.synchronize()
        assert all(c.nb_get_error() == 0 for c in ctxs)
        print(json.dumps({"profile_case": "spce_water_256_replicas_batched", "atoms": int(xcat.shape[0]),
                          "calls": args.warmup + args.steps}))
        return
    if args.profile_case == "vjp":
        s = synth.water_24k_types()
        ctx = api.NbContext.from_system(s)
        x = torch.tensor(s.x, device="cuda")
        ctx.build(x, s.box)
        T = s.n_types
        gF = torch.randn((s.n, 3), device="cuda", generator=torch.Generator(device="cuda").manual_seed(4))
        gx, gq = torch.empty_like(x), torch.empty(s.n, device="cuda")
        g6 = torch.empty((T, T), dtype=torch.float64, device="cuda")
        g12 = torch.empty_like(g6)
        f = torch.empty_like(x)
        e = torch.empty(2, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup + args.steps):
            ctx.nb_forces(api.NB_ENERGY, x, f, e)
            ctx.nb_forces_vjp(x, gF, 0.5, gx, gq, g6, g12)
        torch.cuda.synchronize()
        assert ctx.nb_get_error() == 0
        print(json.dumps({"profile_case": "spce_water_24k_6types_forward_adjoint", "atoms": s.n,
                          "launches": ctx.nb_get_stats()["n_launches"]}))
        return
    if args.profile_case == "polymer_1.5m":
        s = synth.polymer_water_box()
        ctx = api.NbContext.from_system(s)
        if args.split:
            ctx.nb_set_split(args.split)
        x = torch.tensor(s.x, device="cuda")
        ctx.build(x, s.box)
        f = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        e = torch.empty(2, dtype=torch.float64, device="cuda")
        w = torch.empty(9, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup + args.steps):
            ctx.nb_forces(flags, x, f, e, w)
        torch.cuda.synchronize()
        assert ctx.nb_get_error() == 0
        print(json.dumps({"profile_case": "polymer_water_1.5m_ewald", "atoms": s.n,
                          "launches": ctx.nb_get_stats()["n_launches"]}))
        return
    s = synth.water_96k()
    ctx = api.NbContext.from_system(s)
    if args.profile_case == "pme":
        x = torch.tensor(s.x, device="cuda")
        q = torch.tensor(s.q, device="cuda")
        ctx.build(x, s.box)
        pme = api.NbPme.from_system(s, spacing=0.12, order=4)
        f = torch.zeros((s.n, 3), dtype=torch.float32, device="cuda")
        e1 = torch.empty(1, dtype=torch.float64, device="cuda")
        e2 = torch.empty(2, dtype=torch.float64, device="cuda")
        w = torch.empty(9, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup + args.steps):
            pme.nb_pme_forces(api.NB_ENERGY | api.NB_VIRIAL, x, q, s.box, f, e1, w)
            ctx.nb_ewald_corrections(api.NB_ENERGY | api.NB_VIRIAL, x, f, e2, w)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "spce_water_96k_pme_order4_grid84", "calls": args.warmup + args.steps}))
        return
    if args.split:
        ctx.nb_set_split(args.split)
    x = torch.tensor(s.x, device="cuda")
    ctx.build(x, s.box)
    f = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
    e = torch.empty(2, dtype=torch.float64, device="cuda")
    w = torch.empty(9, dtype=torch.float64, device="cuda")
    for t in range(args.warmup + args.steps):
        ctx.nb_forces(api.NB_ENERGY | api.NB_VIRIAL, x, f, e, w)
        ctx.nb_prune_rolling(t % N_PARTS, N_PARTS)
    torch.cuda.synchronize()
    assert ctx.nb_get_error() == 0
    print(json.dumps({"profile_case": "spce_water_96k_ewald", "launches": ctx.nb_get_stats()["n_launches"]}))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched and adjoint workloads")
    ap.add_argument("--caller-order", action="store_true",
                    help="run the headline loop in caller atom order (nb_forces: gather and scatter every step) "
                         "instead of the sorted layout")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--profile", action="store_true",
                    help="profiling target: warmup + steps force evaluations (energy+virial) of the 96k box only")
    ap.add_argument("--profile-case", choices=["forces", "step", "pme", "polymer_1.5m", "batched", "vjp"],
                    default="forces",
                    help="with --profile: the launch sequence to run")
    ap.add_argument("--split", type=int, default=0,
                    help="with --profile: the work-item split to build with (default: the library's)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.profile:
        main_profile(args)
    elif args.impl == "reference":
        main_reference(args)
    else:
        main_ours(args)


if __name__ == "__main__":
    main()
