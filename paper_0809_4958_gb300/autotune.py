"""Autotuner for the stream-collide launch of a context.

The launch choices (kernel, threads per block, persistent grid size, sites per
thread; see lb_set_launch in include/lbtracer.h) only change how the work is
split, never a site's arithmetic within one kernel instantiation, so the tuner
times them on the live context: it steps the simulation a few times per
candidate with the library's CUDA-event profiling around every stream-collide
launch and keeps the fastest.  Choices are cached in a JSON file keyed by the
GPU, the storage format and the mix of box sizes.
"""
from __future__ import annotations

import hashlib
import json
import os

from . import lbtracer as lbt

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tune_cache.json")


def candidates(storage: int, sms: int):
    dv = {lbt.LB_STORE_F64: 2, lbt.LB_STORE_F32: 4, lbt.LB_STORE_F16DEV: 8, lbt.LB_STORE_BF16DEV: 8}[storage]
    out = [(lbt.LB_KERNEL_STAGED, 0, 0, spt) for spt in ((1,) if storage == lbt.LB_STORE_F64 else (2, 1))]
    for threads in (128, 256):
        for vw in sorted({dv, max(dv // 2, 1), max(dv // 4, 1)}):
            out.append((lbt.LB_KERNEL_REGISTER, threads, 0, vw))
    return out


def signature(tr) -> str:
    import torch
    sizes = sorted(d.E for d in tr.descs)
    key = "%s|%d|%s|%d" % (torch.cuda.get_device_name(tr.stream.device), tr.storage,
                           hashlib.sha1(repr(sizes).encode()).hexdigest()[:12], len(sizes))
    return key


def _load_cache():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def tune_bead_lanes(tr, step, nsteps: int = 6):
    """MD thread layout of the bead kernel, (lanes per bead, beads per
    thread): the whole step is timed with CUDA events on the context stream
    for every valid choice (the bead kernel runs beside the stream-collide, so
    only the step shows its cost).  Returns the choice applied to the context
    ((0, 1) when the context has no chain)."""
    import torch
    maxb = max(d.nbeads for d in tr.descs)
    if maxb == 0:
        return (0, 1)
    best, table = None, []
    for lanes, bpt in ((2, 0), (1, 2), (1, 1), (2, 1), (4, 1), (8, 1)):
        if bpt > 0 and lanes * ((maxb + bpt - 1) // bpt) > 512:
            continue
        tr.lb_set_bead_launch(lanes, bpt)
        step(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(tr.stream)
        step(nsteps)
        e1.record(tr.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / nsteps
        table.append(((lanes, bpt), ms))
        if best is None or ms < best[1]:
            best = ((lanes, bpt), ms)
    tr.lb_set_bead_launch(*best[0])
    tr.bead_lanes = best[0]
    tr.bead_table = table
    return best[0]


def tune(tr, step, steps_per_candidate: int = 6, use_cache: bool = True):
    """Pick the fastest stream-collide launch for context `tr`.

    step(k) must advance the context by k steps (pushing boundary samples as
    needed).  Returns (choice, table) with choice = (kernel, threads, ctas,
    sites_per_thread) already applied to the context and table a list of
    (choice, mean stream-collide milliseconds)."""
    import torch
    key = signature(tr)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        choice = tuple(cache[key]["choice"])
        tr.lb_set_launch(*choice)
        tr.lb_set_bead_launch(*cache[key].get("bead_lanes", (0, 1)))
        return choice, cache[key].get("table", [])
    sms = torch.cuda.get_device_properties(tr.stream.device).multi_processor_count
    table = []
    for cand in candidates(tr.storage, sms):
        tr.lb_set_launch(*cand)
        step(1)  # warm-up launch of this shape
        tr.lb_profile(1, steps_per_candidate)
        step(steps_per_candidate)
        tr.lb_profile(0)
        ms, n = tr.lb_profile_read()
        table.append((cand, ms / max(n, 1)))
    choice = min(table, key=lambda t: t[1])[0]
    tr.lb_set_launch(*choice)
    lanes = tune_bead_lanes(tr, step, steps_per_candidate)
    cache[key] = {"choice": list(choice), "table": [[list(c), t] for c, t in table], "bead_lanes": lanes}
    try:
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return choice, table
