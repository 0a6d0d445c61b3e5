"""Autotuner for the two scheduling knobs of the pair kernels.

- split: the largest number of outer j-cluster entries per work item (the
  cluster pairs one warp evaluates before it flushes its i-forces).  Shorter
  items give more parallel work and a shorter kernel tail, longer ones less
  per-item overhead (Sec. V.F: lists are split when there are too few of them).
- n_parts: the rolling prune re-prunes 1/n_parts of the outer list per step
  (Sec. V.E).  More parts mean less prune work per step but an inner list that
  is older when it is used; a cadence is acceptable only if no pair inside rc is
  missed over a list lifetime.

Timings are taken on the device with CUDA events (the library's tracer); the
accuracy check counts, at regular steps of a trajectory, the pairs inside rc
that the outer list holds but the rolling inner list lacks.  Results can be
cached in a JSON file keyed by the GPU name and a hash of the system's shape
and cut-offs.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Callable, Dict, Optional, Sequence

SPLITS = (8, 12, 16, 24, 32, 48, 64, 96, 128)
PARTS = (1, 2, 4, 8)


def choose_split(timings: Dict[int, float]) -> int:
    """The fastest split; ties go to the larger split (fewer items, fewer atomics)."""
    if not timings:
        raise ValueError("no timings")
    best = min(timings.values())
    return max(s for s, t in timings.items() if t <= best * (1 + 1e-9))


def choose_parts(missed: Dict[int, int], step_ms: Dict[int, float]) -> int:
    """Among cadences that missed no pair inside rc, the one with the lowest step time
    (force + prune share); falls back to 1 (prune the whole list every step)."""
    ok = [p for p, m in missed.items() if m == 0]
    if not ok:
        return 1
    return min(ok, key=lambda p: (step_ms.get(p, float("inf")), -p))


def config_key(system, gpu_name: str) -> str:
    h = hashlib.sha1(json.dumps({
        "n": int(system.n), "box": [round(float(v), 6) for v in system.box], "rc": system.rc,
        "rlist": system.rlist, "r_in": system.r_in, "coulomb": int(system.coulomb),
    }, sort_keys=True).encode()).hexdigest()[:16]
    return f"{gpu_name}:{h}"


def load_cache(path: Optional[str]) -> dict:
    if path and os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {}


def save_cache(path: Optional[str], cache: dict) -> None:
    if not path:
        return
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(system, x, velocities=None, *, splits: Sequence[int] = SPLITS, parts: Sequence[int] = PARTS,
         nstlist: int = 100, dt: float = 0.002, reps: int = 15, cache_path: Optional[str] = None,
         flags: Optional[int] = None, flush: Optional[Callable[[], None]] = None) -> dict:
    """Tune split and n_parts for `system` at positions x (CUDA float32 [N,3]).

    velocities (CUDA [N,3], nm/ps) drive the ballistic trajectory of the prune
    check; without them only `split` is tuned and n_parts is 2.  `flush`, when
    given, is called before every timed evaluation (e.g. to evict the L2 cache
    as the caller's own loop does), outside the timed kernel.
    """
    import torch

    from . import api

    gpu = torch.cuda.get_device_name(x.device)
    cache = load_cache(cache_path)
    key = config_key(system, gpu)
    if key in cache:
        return cache[key]
    if flags is None:
        flags = api.NB_ENERGY | api.NB_VIRIAL
    f = torch.empty_like(x)
    e = torch.empty(2, dtype=torch.float64, device=x.device)
    w = torch.empty(9, dtype=torch.float64, device=x.device)
    # one context per candidate, timed in interleaved rounds (slow drifts of clock or
    # temperature hit every candidate alike); the median launch time decides
    ctxs = {}
    for sp in splits:
        c = api.NbContext.from_system(system)
        c.nb_set_split(sp)
        c.build(x, system.box)
        c.nb_trace_enable(True, kinds=[api.NB_TRACE_FORCES])
        for _ in range(3):
            c.nb_forces(flags, x, f, e, w)
        ctxs[sp] = c
    torch.cuda.synchronize()
    for c in ctxs.values():
        c.nb_trace_read(api.NB_TRACE_FORCES)
    samples = {sp: [] for sp in splits}
    for _ in range(reps):
        for sp, c in ctxs.items():
            if flush is not None:
                flush()
            c.nb_forces(flags, x, f, e, w)
            ms, n = c.nb_trace_read(api.NB_TRACE_FORCES)
            samples[sp].append(ms / max(n, 1))
    split_ms = {sp: float(sorted(v)[len(v) // 2]) for sp, v in samples.items()}
    del ctxs
    best_split = choose_split(split_ms)
    ctx = api.NbContext.from_system(system)
    ctx.nb_set_split(best_split)
    ctx.nb_trace_enable(True, kinds=[api.NB_TRACE_FORCES, api.NB_TRACE_PRUNE])
    result = {"split": best_split, "split_ms": split_ms, "n_parts": 2, "missed": {}, "step_ms": {}}
    if velocities is not None:
        for npart in parts:
            xt = x.clone()
            ctx.build(xt, system.box)
            ctx.nb_trace_read(api.NB_TRACE_FORCES)
            ctx.nb_trace_read(api.NB_TRACE_PRUNE)
            missed = 0
            for t in range(nstlist):
                xt.add_(velocities, alpha=dt)
                ctx.nb_forces(flags, xt, f, e, w)
                if t % 10 == 9 or t == nstlist - 1:
                    # pairs inside rc that the outer list has and the rolling inner list lacks
                    within_inner, _ = ctx.nb_count_pairs(api.NB_LIST_INNER)
                    within_outer, _ = ctx.nb_count_pairs(api.NB_LIST_OUTER)
                    missed += max(0, within_outer - within_inner)
                ctx.nb_prune_rolling(t % npart, npart)
            fms, fn = ctx.nb_trace_read(api.NB_TRACE_FORCES)
            pms, pn = ctx.nb_trace_read(api.NB_TRACE_PRUNE)
            result["missed"][npart] = int(missed)
            result["step_ms"][npart] = fms / max(fn, 1) + pms / max(nstlist, 1)
        result["n_parts"] = choose_parts(result["missed"], result["step_ms"])
    ctx.nb_trace_enable(False)
    cache[key] = result
    save_cache(cache_path, cache)
    return result


def tune_batched(systems, xs, *, splits: Sequence[int] = SPLITS, reps: int = 10, flags: Optional[int] = None,
                 flush: Optional[Callable[[], None]] = None, segments: Sequence[int] = (0,)) -> dict:
    """Tune the split (and, given several `segments` values, the pair search's column
    segments, 0 = the library's choice) of a batched evaluation (nb_forces_batched) by
    timing the batched launch itself over `systems` at positions `xs` (CUDA float32
    [N_r,3] each): the best item size for many systems sharing the GPU differs from the
    best one for any of them alone.  Returns {"split", "segments", "split_ms"} with
    split_ms the timings of the chosen segments value, and "timings" {(segments,
    split): ms}."""
    import torch

    from . import api

    if flags is None:
        flags = api.NB_ENERGY | api.NB_VIRIAL
    dev = xs[0].device
    xcat = torch.cat(list(xs)).contiguous()
    fcat = torch.empty_like(xcat)
    r = len(systems)
    e = torch.empty(2 * r, dtype=torch.float64, device=dev)
    w = torch.empty(9 * r, dtype=torch.float64, device=dev)
    timings = {}
    for seg in segments:
        for sp in splits:
            ctxs = []
            for s, xr in zip(systems, xs):
                c = api.NbContext.from_system(s)
                c.nb_set_split(sp)
                c.nb_set_search_segments(seg)
                c.build(xr, s.box)
                ctxs.append(c)
            b = api.NbBatch(ctxs)
            for _ in range(3):
                b.nb_forces_batched(flags, xcat, fcat, e, w)
            tot = 0.0
            for _ in range(reps):
                if flush is not None:
                    flush()
                t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                t0.record()
                b.nb_forces_batched(flags, xcat, fcat, e, w)
                t1.record()
                t1.synchronize()
                tot += t0.elapsed_time(t1)
            timings[(seg, sp)] = tot / reps
            b.close()
            del ctxs
    best_seg = min(segments, key=lambda g: (min(timings[(g, sp)] for sp in splits), g))
    split_ms = {sp: timings[(best_seg, sp)] for sp in splits}
    return {"split": choose_split(split_ms), "segments": best_seg, "split_ms": split_ms, "timings": timings}
