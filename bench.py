#!/usr/bin/env python
"""Throughput of the tracer-box lattice Boltzmann step on GB300.

Workload (default): one D3Q19 BGK box of 128^3 sites, tau 0.8, FP32
populations stored as deviations f_i - w_i, velocity boundaries on all six
faces from a synthetic Kolmogorov-spectrum field (1024 modes, |k| in
[1, 64], one coarse sample per LB step), one 64-bead Kremer-Grest chain (FENE + WCA) with
Philox noise at kT 1e-4 coupled by Stokes friction.  One "step" is one full
LB step: bead coupling, fused stream-collide + boundary layer, forced
re-collision; the timed steps replay a CUDA graph of 16 steps, the samples
of the next 16 steps pushed into the ring before each replay.  The boundary
samples of all timed steps are generated on the GPU before the timed region
and stay resident in HBM (they stand in for the DNS record the paper reads
from disk); each step's working set
(2 x 159 MB of populations) exceeds the 129 MB L2, so no flush is needed.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead (each step a bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = dict(E=128, tau=0.8, M=1024, k_min=1.0, k_max=64.0, K=1, nbeads=64, kT=1e-4, n_md=50, seed=0, graph=16)
METRIC = "LB MLUPS"
UNIT = "MLUPS"
Q = 19


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None, help="timed steps (default: 10000 single, 1008 batch, 5000 precision)")
    p.add_argument("--warmup", type=int, default=None, help="untimed steps (default: 50 single, 112 batch, 20 precision)")
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--storage", default="f32", choices=["f32", "f64", "f16", "bf16"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-forms", action="store_true", help="skip the short runs of the batched, 16-bit and "
                                                            "upsampler forms in the default line")
    p.add_argument("--no-tune", action="store_true", help="skip the launch autotuner (use --kernel/--threads/...)")
    p.add_argument("--threads", type=int, default=0, help="stream-collide block size (0 = library default)")
    p.add_argument("--ctas", type=int, default=0, help="persistent grid size (0 = one block per tile)")
    p.add_argument("--vw", type=int, default=0, help="sites per thread in stream-collide (0 = default)")
    p.add_argument("--bead-layout", default=None, help="MD thread layout 'lanes,beads_per_thread' of the bead "
                   "kernel (as lb_set_bead_launch; default: autotuned, or the library default with --no-tune)")
    p.add_argument("--kernel", default="staged", choices=["staged", "register"],
                   help="stream-collide kernel: TMA-staged pipeline or register tiles")
    p.add_argument("--dry-run", action="store_true",
                   help="exercise the rank launcher and the whole-job reduction only (CPU, gloo): each rank reports "
                        "fixed stand-in units and times, no GPU work, no measurement")
    p.add_argument("--config", default="single", choices=["single", "batch", "precision", "mlp", "paper"],
                   help="single 128^3 box (default), 512 uneven boxes under a CUDA graph, 256^3 16-bit storage, "
                        "256 boxes of 64^3 with the learned boundary upsampler (K = 16), or the paper-shaped "
                        "replay (z = 6, tau = 1, Eq. 1 time step, co-moving frame force)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def launch_ranks(args):
    """--gpus N > 1 started without a process group in the environment: run
    this script again under torch.distributed.run, one rank per GPU of this
    node (rendezvous on 127.0.0.1).  Boxes are independent, so the ranks
    exchange nothing while stepping; rank 0 prints the whole-job line."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(args.gpus),
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def run_dry(args):
    """The launcher and the whole-job reduction without a GPU: rank r stands
    in with (r + 1) * 1e6 site updates in 10 + r milliseconds."""
    import torch.distributed as dist
    rank, world, _ = dist_env()
    if world > 1:
        dist.init_process_group("gloo")
    units, ms = whole_job((rank + 1) * 1e6, 10.0 + rank)
    if rank == 0:
        print(json.dumps({"dry_run": True, "n_gpus": world, "units": units, "ms": ms, "value": None}), flush=True)
    if world > 1:
        dist.destroy_process_group()


def whole_job(units, ms, device=None):
    """Whole-job totals over the ranks of the process group: the site
    updates every rank made (summed) and the slowest rank's time (max).  The
    boxes of different ranks are independent, so this is the only exchange;
    without a group of more than one rank it returns its arguments."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units), float(ms)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    m = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return float(u.item()), float(m.item())


def alg_bytes_per_launch(E, s_elem, s_real, time_interp=0):
    """Algorithmic bytes of one stream-collide launch over one box with
    velocity faces: interior sites read and write 19 populations, boundary
    sites write 19 and read 3 components of 2 (linear) or 4 (Hermite)
    coarse samples."""
    interior = (E - 2) ** 3
    boundary = E ** 3 - interior
    nsamp = 2 if time_interp == 0 else 4
    return interior * 2 * Q * s_elem + boundary * (Q * s_elem + 3 * nsamp * s_real)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


KERNEL_SOURCES = {
    "k_stream_collide_staged": ("lbt_sc_staged.cuh", "lbt_device.cuh", "lbt_internal.h"),
    "k_stream_collide": ("lbt_kernels.cuh", "lbt_device.cuh", "lbt_internal.h"),
}


def plan_timed_steps(steps, graph=16):
    """Split `steps` timed steps into graph replays and plain steps:
    (G, nrep, rest) with nrep * G + rest == steps.  The last `rest` steps run
    plainly, their stream-collide launches timed by CUDA events (event-record
    nodes inside a graph serialise its kernels: about 10 us per step at
    128^3).  Runs of 64 steps or more use graphs of `graph` steps and 8 to
    graph + 7 plain steps; shorter runs keep up to 8 plain steps and the
    largest even graph length that divides the rest (G = 0: no graph)."""
    if steps >= 64:
        P = 8 + (steps - 8) % graph
        G = graph
    else:
        P = min(8, steps)
        even = (steps - P) // 2 * 2
        G = max([g for g in range(2, min(graph, even) + 1, 2) if even % g == 0] or [0])
    nrep = (steps - P) // G if G else 0
    return G, nrep, steps - nrep * G


def kernel_source_hash(kernel):
    """Hash of the sources a stream-collide kernel is compiled from."""
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_0809_4958_gb300", "csrc", rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(storage, kernel):
    """DRAM bytes per stream-collide launch of `kernel` from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "stream_collide_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d.get("%s/%s" % (storage, kernel))
        if ent and ent.get("kernel_hash") == kernel_source_hash(kernel):
            return float(ent["bytes_per_launch_full_size"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(storage_name):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload:
    a few LB steps of the 128^3 box with the same chain and boundary recipe,
    on all host cores it uses (OpenMP)."""
    import oracle
    from paper_0809_4958_gb300 import inputs
    w = WORKLOAD
    E = w["E"]
    modes = inputs.mode_table(w["seed"] + 1000, 64, w["k_min"], w["k_max"], E)
    box = oracle.BoxParams(E=E, tau=w["tau"], K=1)
    ch = oracle.ChainParams(nbeads=w["nbeads"], kT=w["kT"], n_md=w["n_md"], seed=1)
    pos0 = inputs.chain_start(w["seed"] + 5, w["nbeads"], E)
    S = oracle.face_samples(modes, E, 1, 0, 3)
    sim = oracle.Sim(box, np.zeros((3, E, E, E)), S, ch, pos0)
    t0 = time.perf_counter()
    assert sim.run(1) == 0
    t1 = time.perf_counter() - t0
    nsteps = int(max(1, min(100, 12.0 / max(t1, 1e-3))))
    S = oracle.face_samples(modes, E, 1, 0, nsteps + 3)
    sim = oracle.Sim(box, np.zeros((3, E, E, E)), S, ch, pos0)
    assert sim.run(1) == 0
    t0 = time.perf_counter()
    assert sim.run(nsteps) == 0
    dt = time.perf_counter() - t0
    return {"value": E ** 3 * nsteps / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d FP64 oracle steps of the %d^3 box (same chain and boundary recipe, 64-mode boundary "
                      "field, initial field at rest), after 1 untimed step" % (nsteps, E)}


def single_config(storage_name):
    """The workload of the default line, shared by both arms."""
    w = WORKLOAD
    E = w["E"]
    s_elem = {"f32": 4, "f64": 8, "f16": 2, "bf16": 2}[storage_name]
    return {"workload": "tracer box %d^3 D3Q19 BGK tau %.2f, %s populations (f_i - w_i), 64-bead Kremer-Grest chain "
                        "kT %g, Kolmogorov velocity boundaries on 6 faces (1024 modes, one sample per step)"
                        % (E, w["tau"], storage_name, w["kT"]),
            "boxes_per_gpu": 1, "sites_per_box": E ** 3,
            "l2": "working set 2 x %.0f MB > L2, no flush" % (Q * E ** 3 * s_elem / 1e6)}


def run_reference(args):
    """--impl reference: the oracle as it stands, each timed step a bounded
    sample of the workload (one LB step of a box of edge E_s with the same
    recipe, E_s the largest of 128, 96, 64, 48, 32 that keeps the run within a
    few minutes)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_0809_4958_gb300 import inputs
    oracle.build()
    w = WORKLOAD
    budget = 150.0
    chosen = None
    for Es in (128, 96, 64, 48, 32):
        modes = inputs.mode_table(w["seed"] + 1000, 64, w["k_min"], min(w["k_max"], Es / 2), Es)
        S = oracle.face_samples(modes, Es, 1, 0, args.steps + args.warmup + 3)
        sim = oracle.Sim(oracle.BoxParams(E=Es, tau=w["tau"], K=1), np.zeros((3, Es, Es, Es)), S,
                         oracle.ChainParams(nbeads=min(w["nbeads"], 2 * Es // 2), kT=w["kT"], n_md=w["n_md"], seed=1),
                         inputs.chain_start(w["seed"] + 5, min(w["nbeads"], 2 * Es // 2), Es))
        t0 = time.perf_counter()
        assert sim.run(1) == 0
        t1 = time.perf_counter() - t0
        if t1 * (args.steps + args.warmup) <= budget or Es == 32:
            chosen = (Es, sim)
            break
    Es, sim = chosen
    assert sim.run(max(0, args.warmup - 1)) == 0
    t0 = time.perf_counter()
    assert sim.run(args.steps) == 0
    dt = time.perf_counter() - t0
    value = Es ** 3 * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": single_config(args.storage),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "each step: one oracle LB step of a %d^3 box with the same recipe" % Es},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    defaults = {"single": (10000, 50), "batch": (1008, 112), "precision": (5000, 20), "mlp": (1024, 64),
                "paper": (4000, 64)}[args.config]
    if args.steps is None:
        args.steps = defaults[0]
    if args.warmup is None:
        args.warmup = defaults[1]
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(launch_ranks(args))
    if args.dry_run:
        run_dry(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.config == "batch":
        run_batch(args)
        return
    if args.config == "precision":
        run_precision(args)
        return
    if args.config == "mlp":
        run_mlp(args)
        return
    if args.config == "paper":
        run_paper(args)
        return
    import torch
    import torch.distributed as dist

    from paper_0809_4958_gb300 import inputs, lbtracer as lbt

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    storage = {"f32": lbt.LB_STORE_F32, "f64": lbt.LB_STORE_F64, "f16": lbt.LB_STORE_F16DEV,
               "bf16": lbt.LB_STORE_BF16DEV}[args.storage]
    s_elem = {"f32": 4, "f64": 8, "f16": 2, "bf16": 2}[args.storage]
    s_real = 8 if args.storage == "f64" else 4
    real = torch.float64 if args.storage == "f64" else torch.float32
    w = WORKLOAD
    E = w["E"]
    seed = w["seed"] + rank  # one independent tracer box per GPU

    # ---- inputs (untimed): boundary record, initial field, chain ----
    from paper_0809_4958_gb300 import autotune
    modes = inputs.mode_table(seed, w["M"], w["k_min"], w["k_max"], E)
    ncand = 0 if args.no_tune else len(autotune.candidates(storage, torch.cuda.get_device_properties(dev).multi_processor_count))
    tune_steps = 7 * ncand + 7 * 6  # launch shapes, then the bead kernel's six thread layouts
    G, _, _ = plan_timed_steps(args.steps, w["graph"])
    nsamp = args.warmup + tune_steps + args.steps + 2 * w["graph"] + 2  # + one untimed replay
    faces = lbt.synth_faces(modes, E, w["K"], 0, nsamp, real)
    u0 = lbt.synth_volume(modes, E, 0.0, real)
    pos0 = inputs.chain_start(seed + 5, w["nbeads"], E)
    stream = torch.cuda.Stream()
    tr = lbt.Tracers([lbt.box_desc(E, w["tau"], nbeads=w["nbeads"], K=w["K"])], storage, stream=stream,
                     ring_slots=G + 4)
    kernel = lbt.LB_KERNEL_STAGED if args.kernel == "staged" else lbt.LB_KERNEL_REGISTER
    tr.lb_set_launch(kernel, args.threads, args.ctas, args.vw)
    torch.cuda.synchronize()
    tr.lb_init(0, u0)
    tr.chain_couple(0, lbt.chain_desc(w["nbeads"], kT=w["kT"], n_md=w["n_md"], seed=seed), pos0)
    pushed = [-1]

    def push_until(j, src):
        while pushed[0] < j:
            pushed[0] += 1
            tr.lb_set_boundary(0, pushed[0], src(pushed[0]))

    dev_src = lambda j: faces[j]  # noqa: E731

    def step(k):
        for _ in range(k):
            push_until(tr.lb_current_step() + 1, dev_src)
            tr.lb_step(1)

    table = []
    choice = (kernel, args.threads, args.ctas, args.vw)
    if not args.no_tune:  # the autotuner steps the simulation; its steps are untimed warm-up
        choice, table = autotune.tune(tr, step, steps_per_candidate=6, use_cache=False)
    if args.bead_layout:
        tr.bead_lanes = tuple(int(v) for v in args.bead_layout.split(","))
        tr.lb_set_bead_launch(*tr.bead_lanes)
    step(args.warmup)
    tr.lb_sync()

    # ---- timed region (device-resident inputs) ----
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # G steps per CUDA graph replay; the samples of the next G steps are pushed
    # (device to device) before each replay; `rest` plain steps after them
    # (at least 8 when the run is that long), all with timed stream-collides
    _, nrep, rest = plan_timed_steps(args.steps, w["graph"])
    if nrep:
        tr.lb_graph_capture(G)
        push_until(tr.lb_current_step() + G, dev_src)  # one untimed replay: the graph's first run
        tr.lb_graph_launch()
        tr.lb_sync()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)  # let the sampler take its first reading
    # The samples of a replay are pushed while the replay before it runs (the
    # host enqueues them behind that graph): the first replay's before the
    # timed region, one replay's worth after the last one inside it, so the
    # timed region still pushes exactly one sample per timed step.
    if nrep:
        push_until(tr.lb_current_step() + G, dev_src)
        torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(nrep):
        tr.lb_graph_launch()
        push_until(tr.lb_current_step() + G, dev_src)
    tr.lb_profile(1, rest)  # host side only: the plain steps below record the events
    step(rest)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    tr.lb_profile(0)
    sc_ms, sc_n = tr.lb_profile_read()
    tr.lb_sync()
    units, ms = whole_job(E ** 3 * args.steps, ev0.elapsed_time(ev1), dev)
    if world > 1:
        dist.barrier()
    ms_per_step = ms / args.steps
    value = units / (ms * 1e-3) / 1e6
    bead_layout = list(getattr(tr, "bead_lanes", (0, 1)))
    bead_table = [[list(c), t] for c, t in getattr(tr, "bead_table", [])]
    tr.close()  # the end-to-end leg gets the device to itself (a run with the sample
    # record of 10,000 steps still held measured 20 % slower end to end)

    # ---- end to end through the C ABI with host buffers ----
    # The same step as above (graph replays of G2 steps), fed from pinned host
    # memory and read back to it: every step's boundary sample goes host ->
    # device on a copy stream (a replay's G2 samples in one copy, two replays
    # ahead, into a pair of device staging blocks), is pushed into the
    # boundary ring behind the replay before its own (device to device,
    # lb_set_boundary), and every step's chain positions, left by the bead
    # kernel in a trajectory ring (lb_set_chain_history), come back to pinned
    # host memory after each replay.  The first replay's samples are pushed
    # before the timed region and one replay's worth after the last one inside
    # it, so the timed region moves exactly one sample in and one result out
    # per timed step.
    e2e = None
    if not args.no_e2e:
        W2 = args.warmup  # plain untimed steps first
        G2 = w["graph"]  # replays of 16 steps (shorter graphs cost more per step end to end)
        nrep2 = max(1, min(args.steps, 2000) // G2)
        e2e_steps = nrep2 * G2
        nstep2 = W2 + (nrep2 + 3) * G2
        if nstep2 + 2 > faces.shape[0]:
            faces = torch.cat([faces, lbt.synth_faces(modes, E, w["K"], faces.shape[0], nstep2 + 2 - faces.shape[0], real)])
        host_faces = faces[:nstep2 + 2].cpu()  # the host record of the boundary samples (pageable)
        del faces, dev_src
        torch.cuda.empty_cache()
        nb = w["nbeads"]
        host_hist = torch.empty((nrep2, G2, nb, 3), dtype=torch.float64, pin_memory=True)
        # fresh context so the pushed samples line up with the host record
        tr2 = lbt.Tracers([lbt.box_desc(E, w["tau"], nbeads=nb, K=w["K"])], storage, stream=stream, ring_slots=G2 + 4)
        tr2.lb_set_launch(*choice)
        tr2.lb_set_bead_launch(*bead_layout)
        torch.cuda.synchronize()
        tr2.lb_init(0, u0)
        tr2.chain_couple(0, lbt.chain_desc(nb, kT=w["kT"], n_md=w["n_md"], seed=seed), pos0)
        hist = torch.zeros((G2, nb, 3), dtype=torch.float64, device=dev)
        tr2.lb_set_chain_history(hist, G2)
        tr2.lb_set_boundary(0, 0, host_faces[0].contiguous())
        for n in range(W2):
            tr2.lb_set_boundary(0, n + 1, host_faces[n + 1])
            tr2.lb_step(1)
        tr2.lb_sync()
        copy_stream = torch.cuda.Stream()
        NB = 3  # pinned staging blocks: a small ring stays fast for the copy engine (copies from a
        # pinned buffer of the whole record slowed to about 5 GB/s once the device had been busy)
        pinned = torch.empty((NB, G2, 6, 3, E, E), dtype=real, pin_memory=True)
        stage = torch.empty((2, G2, 6, 3, E, E), dtype=real, device=dev)
        ev_h2d = [torch.cuda.Event() for _ in range(NB)]
        ev_copied = [torch.cuda.Event() for _ in range(2)]
        ev_used = [torch.cuda.Event() for _ in range(2)]
        lib, ctx = tr2.lib, tr2.ctx

        def copy_block(k):  # host -> device: the samples of replay k (steps W2 + k G2 ..)
            j0 = W2 + k * G2 + 1
            b = k % NB
            ev_h2d[b].synchronize()  # the pinned block's previous copy has left
            pinned[b].copy_(host_faces[j0:j0 + G2])  # host record -> pinned staging (CPU)
            copy_stream.wait_event(ev_used[k % 2])  # the device block's previous samples are in the ring
            with torch.cuda.stream(copy_stream):
                stage[k % 2].copy_(pinned[b], non_blocking=True)
            ev_h2d[b].record(copy_stream)
            ev_copied[k % 2].record(copy_stream)

        def push_block(k):  # staging -> boundary ring, on the context stream
            j0 = W2 + k * G2 + 1
            stream.wait_event(ev_copied[k % 2])
            for i in range(G2):
                lbt._check(lib.lb_set_boundary(ctx, 0, j0 + i, stage[k % 2, i].data_ptr()), ctx)
            ev_used[k % 2].record(stream)

        tr2.lb_graph_capture(G2)
        copy_block(0)
        push_block(0)
        copy_block(1)
        tr2.lb_graph_launch()  # replay 0, untimed: the graph's first run
        push_block(1)
        copy_block(2)
        tr2.lb_sync()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev0.record(stream)
        for r in range(1, nrep2 + 1):
            tr2.lb_graph_launch()
            with torch.cuda.stream(stream):
                host_hist[r - 1].copy_(hist, non_blocking=True)  # every step's chain positions of this replay
            push_block(r + 1)
            copy_block(r + 2)
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ev_ms = ev0.elapsed_time(ev1)
        units2, ms2 = whole_job(E ** 3 * e2e_steps, max(ev_ms, wall * 1e3), dev)
        e2e = {"value": units2 / (ms2 * 1e-3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": 6 * 3 * E * E * s_real, "d2h_bytes_per_step": nb * 3 * 8,
               "steps": e2e_steps, "event_ms": ev_ms, "wall_ms": wall * 1e3,
               "how": "graph replays of %d steps through the C ABI; per step one boundary sample from the host "
                      "record (pageable) into a ring of pinned staging blocks, host to device %d samples at a "
                      "time two replays ahead, pushed with lb_set_boundary; the chain's positions back to "
                      "pinned host memory (trajectory ring, read after each replay)" % (G2, G2)}
        tr2.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peak, peak_kind = measured_peaks()
    alg = alg_bytes_per_launch(E, s_elem, s_real)
    avg_sc = sc_ms / max(sc_n, 1)
    achieved = alg / (avg_sc * 1e-3) / 1e9
    sc_kernel = "k_stream_collide_staged" if choice[0] == lbt.LB_KERNEL_STAGED else "k_stream_collide"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": single_config(args.storage),
        "launch": {"kernel": ["staged", "register"][choice[0]], "threads": choice[1], "ctas": choice[2],
                   "sites_per_thread": choice[3], "bead_layout": bead_layout, "bead_autotune": bead_table,
                   "graph_steps": G, "graph_replays": nrep, "plain_steps": rest,
                   "autotune": [[list(c), t] for c, t in table]},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": ncu_traffic(args.storage, sc_kernel),
                     "kernel": sc_kernel,
                     "avg_launch_ms": avg_sc, "alg_bytes_per_launch": alg,
                     "peak_kind": peak_kind, "launches_timed": sc_n},
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": args.steps * 3,
    }
    torch.cuda.synchronize()
    if not args.no_forms:
        line["forms"] = measure_forms(args, value) if world == 1 else {"skipped": "forms run at one GPU only"}
    if not args.no_cpu:
        import oracle
        oracle.build()
        try:
            line["cpu_baseline"] = cpu_baseline(args.storage)
        except Exception as e:  # report, do not lose the GPU line
            line["cpu_baseline"] = {"value": None, "error": repr(e)}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


BATCH = dict(nboxes=512, choices=(24, 32, 48, 64), tau=0.8, M=256, K=1, kT=1e-4, n_md=50, seed=0, graph=16)


def run_batch(args, standalone=True):
    """512 tracer boxes of uneven size (E uniform in {24, 32, 48, 64}), each
    with its own boundary field and chain (32 .. min(128, 2E) beads), FP32,
    stepped by a CUDA graph of 16 steps after the launch shape is autotuned.
    Returns the line (rank 0); standalone: set up and print it."""
    import torch
    import torch.distributed as dist

    from paper_0809_4958_gb300 import autotune, inputs, lbtracer as lbt

    rank, world, local = dist_env()
    if not standalone:
        rank, world = 0, 1
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = BATCH
    G = w["graph"]
    seed = w["seed"] + 7919 * rank
    edges = inputs.batch_edges(seed, w["nboxes"], w["choices"])
    nbs = inputs.batch_chain_lengths(seed, edges)
    steps = (args.steps + G - 1) // G * G
    warm = (args.warmup + G - 1) // G * G
    ncand = len(autotune.candidates(lbt.LB_STORE_F32, torch.cuda.get_device_properties(dev).multi_processor_count))
    tune_steps = 7 * ncand + 7 * 6  # launch shapes, then the bead kernel's six thread layouts
    nsamp = warm + tune_steps + steps + 3 * G + 2  # + the untimed first replay and one replay pushed ahead
    descs = [lbt.box_desc(int(E), w["tau"], nbeads=int(N), K=w["K"]) for E, N in zip(edges, nbs)]
    stream = torch.cuda.Stream()
    tr = lbt.Tracers(descs, lbt.LB_STORE_F32, stream=stream, ring_slots=G + 4)
    fs = [18 * int(E) * int(E) for E in edges]
    offs = np.concatenate([[0], np.cumsum(fs)])
    faces = torch.empty((nsamp, int(offs[-1])), dtype=torch.float32, device=dev)
    sites = int(sum(int(E) ** 3 for E in edges))
    for b, (E, N) in enumerate(zip(edges, nbs)):
        E, N = int(E), int(N)
        modes = inputs.mode_table(seed * 1000 + b, w["M"], 1.0, E / 2.0, E)
        faces[:, offs[b]:offs[b + 1]] = lbt.synth_faces(modes, E, w["K"], 0, nsamp, torch.float32).view(nsamp, -1)
        u0 = lbt.synth_volume(modes, E, 0.0, torch.float32)
        torch.cuda.synchronize()
        tr.lb_init(b, u0)
        tr.lb_sync()
        tr.chain_couple(b, lbt.chain_desc(N, kT=w["kT"], n_md=w["n_md"], seed=seed * 1000 + b),
                        inputs.chain_start(seed * 1000 + b, N, E))
    torch.cuda.synchronize()
    pushed = [-1]

    def push_until(j):
        while pushed[0] < j:
            pushed[0] += 1
            tr.lb_set_boundary(lbt.LB_ALL_BOXES, pushed[0], faces[pushed[0]])

    def step(k):
        for _ in range(k):
            push_until(tr.lb_current_step() + 1)
            tr.lb_step(1)

    choice, table = autotune.tune(tr, step, steps_per_candidate=6, use_cache=False)
    step(warm)
    tr.lb_sync()
    tr.lb_graph_capture(G)
    push_until(tr.lb_current_step() + G)  # one untimed replay: the graph's first run
    tr.lb_graph_launch()
    push_until(tr.lb_current_step() + G)  # the first timed replay's samples
    tr.lb_sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0.record(stream)
    for _ in range(steps // G - 1):  # a replay's samples are pushed behind the replay before it
        tr.lb_graph_launch()
        push_until(tr.lb_current_step() + G)
    # the last G steps plainly, their stream-collide launches timed by CUDA
    # events (event-record nodes inside a graph would serialise its kernels)
    tr.lb_profile(1, G)
    step(G)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    tr.lb_profile(0)
    sc_ms, sc_n = tr.lb_profile_read()
    tr.lb_sync()
    units, ms = whole_job(sites * steps, ev0.elapsed_time(ev1), dev)
    value = units / (ms * 1e-3) / 1e6
    if rank == 0:
        peak, peak_kind = measured_peaks()
        alg = sum(alg_bytes_per_launch(int(E), 4, 4) for E in edges)
        avg_sc = sc_ms / max(sc_n, 1)
        achieved = alg / (avg_sc * 1e-3) / 1e9
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warm,
                "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "%d tracer boxes, E uniform in {24,32,48,64} (%d sites), tau %.2f, FP32, own "
                                       "Kolmogorov boundary field (256 modes, |k| <= E/2, one sample per step) and "
                                       "FENE+WCA chain (32..min(128,2E) beads, kT %g) per box; CUDA graph of %d steps"
                                       % (w["nboxes"], sites, w["tau"], w["kT"], G),
                           "boxes_per_gpu": w["nboxes"], "sites_per_gpu": sites,
                           "l2": "working set 2 x %.1f GB > L2, no flush" % (19 * 4 * sites / 1e9),
                           "launch": {"kernel": ["staged", "register"][choice[0]], "threads": choice[1],
                                      "ctas": choice[2], "sites_per_thread": choice[3]},
                           "autotune": [[list(c), t] for c, t in table]},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                             "traffic": None, "kernel": "stream-collide", "avg_launch_ms": avg_sc,
                             "alg_bytes_per_launch": alg, "peak_kind": peak_kind, "launches_timed": sc_n},
                "clocks": clk, "e2e": None, "gpu_launches": steps * 3}
        if standalone:
            print(json.dumps(line), flush=True)
    tr.close()
    del faces
    torch.cuda.synchronize()
    if world > 1:
        dist.destroy_process_group()
    return line if rank == 0 else None


PRECISION = dict(E=256, tau=0.8, M=2048, k_min=1.0, k_max=128.0, K=1, seed=3)


def run_paper(args):
    """The paper-shaped replay: one box of 128^3 (the paper's 121 sites
    rounded to the 8-site alignment) zoomed z = 6 from a 23^2 coarse face
    grid, tau = 1, one coarse sample every 0.05 tau_eta mapped by Eq. (1)
    (113 LB steps), the flow in the tracer's co-moving frame with the frame
    force from the tracer's acceleration, a 64-bead chain at the centre; FP32,
    graphs of 16 steps, samples pushed before each replay."""
    import torch

    from paper_0809_4958_gb300 import inputs, lbtracer as lbt, scaling

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    eta, tau_eta = scaling.kolmogorov(1.0 / 400.0, 0.1)
    um = scaling.UnitMap(eta=eta, tau_eta=tau_eta, delta=2 * np.pi / 1024, z=6, tau=1.0)
    K = int(round(um.steps(0.05 * tau_eta)))
    E, z, nb, G = 128, 6, 64, 16
    steps = (args.steps + G - 1) // G * G
    warm = (args.warmup + G - 1) // G * G
    u_eta = um.eta_lb / um.tau_eta_lb
    modes = inputs.mode_table(21, 256, 1.0, 10.0, E, u_max=3 * u_eta)
    J = (warm + steps + 3 * G) // K + 3
    faces = lbt.synth_faces(modes, E, K, 0, J, torch.float32, zoom=z)
    v = inputs.tracer_velocity(modes, np.arange(J) * K)
    faces -= torch.from_numpy(v).to(faces)[:, None, :, None, None]  # co-moving frame
    u0 = lbt.synth_volume(modes, E, 0.0, torch.float32, zoom=z) - torch.from_numpy(v[0]).to(faces)[:, None, None, None]
    fsamp = inputs.tracer_frame_accel(modes, np.arange(J) * K)
    stream = torch.cuda.Stream()
    tr = lbt.Tracers([lbt.box_desc(E, 1.0, K=K, nbeads=nb, zoom=z, frame_accel=True)], lbt.LB_STORE_F32,
                     stream=stream)
    torch.cuda.synchronize()
    tr.lb_init(0, u0.contiguous())
    tr.chain_couple(0, lbt.chain_desc(nb, kT=1e-4, seed=5), inputs.chain_start(3, nb, E))
    pushed = [-1]

    def push_until(n):  # samples needed by the steps before n
        while pushed[0] < (n - 1) // K + 1:
            pushed[0] += 1
            tr.lb_set_boundary(0, pushed[0], faces[pushed[0]])
            tr.lb_set_frame_accel(0, pushed[0], fsamp[pushed[0]])

    for _ in range(warm):
        push_until(tr.lb_current_step() + 1)
        tr.lb_step(1)
    tr.lb_sync()
    tr.lb_graph_capture(G)
    push_until(tr.lb_current_step() + G)  # one untimed replay: the graph's first run
    tr.lb_graph_launch()
    push_until(tr.lb_current_step() + G)  # the first timed replay's samples
    tr.lb_sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ev0.record(stream)
    for _ in range(steps // G):  # a replay's samples are pushed behind the replay before it
        tr.lb_graph_launch()
        push_until(tr.lb_current_step() + G)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    tr.lb_sync()
    ms = ev0.elapsed_time(ev1)
    value = E ** 3 * steps / (ms * 1e-3) / 1e6
    tr.close()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warm,
            "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper-shaped replay: 128^3 box zoomed z = 6 from a 23^2 coarse face grid, tau 1, "
                                   "one coarse sample every %d LB steps (0.05 tau_eta by Eq. 1), co-moving frame "
                                   "with the tracer's frame force, 64-bead chain, synthetic field (|k| in [1, 10], "
                                   "3 u_eta); CUDA graphs of %d steps" % (K, G),
                       "eta_lb_sites": um.eta_lb, "tau_eta_lb_steps": um.tau_eta_lb, "mach": um.mach,
                       "l2": "working set 2 x 159 MB > L2, no flush"},
            "roofline": None, "clocks": clk, "e2e": None, "gpu_launches": steps * 3}
    print(json.dumps(line), flush=True)


def run_precision(args, standalone=True):
    """One 256^3 box (no chain) stored as FP32, binary16 and bfloat16
    deviations; MLUPS of each and the velocity and non-equilibrium stress
    error of the 16-bit forms against the FP32 form after the same steps."""
    import torch

    from paper_0809_4958_gb300 import inputs, lbtracer as lbt

    rank, world, local = dist_env()
    if rank != 0 and standalone:
        return None
    torch.cuda.set_device(local)
    w = PRECISION
    E = w["E"]
    modes = inputs.mode_table(w["seed"], w["M"], w["k_min"], w["k_max"], E)
    nsamp = args.warmup + args.steps + 2
    faces = lbt.synth_faces(modes, E, w["K"], 0, nsamp, torch.float32)
    u0 = lbt.synth_volume(modes, E, 0.0, torch.float32)
    cvec = torch.tensor([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 0],
                         [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1], [0, 1, 1],
                         [0, -1, -1], [0, 1, -1], [0, -1, 1]], dtype=torch.float64, device="cuda")
    wts = torch.tensor([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12, dtype=torch.float64, device="cuda")

    def stress_neq(d):
        # non-equilibrium momentum flux of the stored populations (analysis only)
        f = d.double() + wts[:, None, None, None]
        rho = f.sum(0)
        j = torch.einsum("ia,ixyz->axyz", cvec, f)
        u = j / rho
        Pi = torch.einsum("ia,ib,ixyz->abxyz", cvec, cvec, f)
        eye = torch.eye(3, dtype=torch.float64, device="cuda")[:, :, None, None, None]
        return Pi - rho * (eye / 3 + u[:, None] * u[None, :])

    results = {}
    fields = {}
    for name, code in (("f32", lbt.LB_STORE_F32), ("f16", lbt.LB_STORE_F16DEV), ("bf16", lbt.LB_STORE_BF16DEV)):
        stream = torch.cuda.Stream()
        tr = lbt.Tracers([lbt.box_desc(E, w["tau"], K=w["K"])], code, stream=stream)
        torch.cuda.synchronize()
        tr.lb_init(0, u0)
        pushed = [-1]

        def push_until(j):
            while pushed[0] < j:
                pushed[0] += 1
                tr.lb_set_boundary(0, pushed[0], faces[pushed[0]])

        for n in range(args.warmup):
            push_until(n + 1)
            tr.lb_step(1)
        tr.lb_sync()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tr.lb_profile(1, args.steps)
        ev0.record(stream)
        for n in range(args.warmup, args.warmup + args.steps):
            push_until(n + 1)
            tr.lb_step(1)
        ev1.record(stream)
        torch.cuda.synchronize()
        tr.lb_profile(0)
        sc_ms, sc_n = tr.lb_profile_read()
        ms = ev0.elapsed_time(ev1)
        s_elem = 4 if name == "f32" else 2
        alg = alg_bytes_per_launch(E, s_elem, 4)
        peak, _ = measured_peaks()
        results[name] = {"MLUPS": E ** 3 * args.steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / args.steps,
                         "stream_collide_ms": sc_ms / max(sc_n, 1),
                         "hbm_frac": alg / (sc_ms / max(sc_n, 1) * 1e-3) / 1e9 / peak}
        u = torch.empty((3, E, E, E), dtype=torch.float32, device="cuda")
        tr.lb_read_fields(0, lbt.LB_FIELD_U, u)
        d = torch.empty((19, E, E, E), dtype=torch.float32, device="cuda")
        tr.lb_read_fields(0, lbt.LB_FIELD_DEV, d)
        sl = (slice(None), slice(1, -1), slice(1, -1), slice(1, -1))
        fields[name] = (u[sl].double(), stress_neq(d)[:, :, 1:-1, 1:-1, 1:-1])
        del d
        tr.close()
        torch.cuda.synchronize()
    u_ref, s_ref = fields["f32"]
    for name in ("f16", "bf16"):
        u, st = fields[name]
        results[name]["velocity_rel_l2_vs_f32"] = float(torch.linalg.norm(u - u_ref) / torch.linalg.norm(u_ref))
        results[name]["stress_rel_l2_vs_f32"] = float(torch.linalg.norm(st - s_ref) / torch.linalg.norm(s_ref))
    peak, peak_kind = measured_peaks()
    line = {"metric": METRIC, "value": results["f16"]["MLUPS"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": results["f16"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
            "config": {"workload": "tracer box %d^3 D3Q19 BGK tau %.2f, binary16 deviations f_i - w_i (value), "
                                   "bfloat16 and FP32 for comparison, Kolmogorov velocity boundaries (2048 modes, "
                                   "|k| in [1,128], one sample per step), no chain" % (E, w["tau"]),
                       "forms": results},
            "roofline": {"bound": "hbm", "achieved": results["f16"]["hbm_frac"] * peak, "peak": peak, "unit": "GB/s",
                         "frac": results["f16"]["hbm_frac"], "traffic": None, "kernel": "stream-collide",
                         "peak_kind": peak_kind},
            "e2e": None, "gpu_launches": args.steps * 2}
    del faces
    torch.cuda.synchronize()
    if standalone:
        print(json.dumps(line), flush=True)
    return line


MLP = dict(nboxes=256, E=64, tau=0.8, M=256, k_min=1.0, k_max=32.0, K=16, u_max=0.05, train_boxes=12,
           train_intervals=10, train_steps=3000, batch=16384, lr=2e-3, eval_boxes=4, eval_steps=256, seed=500)


def run_mlp(args, standalone=True):
    """256 boxes of 64^3 with coarse boundary samples every K = 16 steps.
    The upsampler is trained on the GPU on every-step boundary data of
    training seeds, its gain is measured on held-out boxes (interior velocity
    error against the run that sees the boundary every step, for linear,
    Hermite and Hermite + learned residual), and the throughput of all boxes
    is timed with the network in the step (and with Hermite alone)."""
    import torch

    from paper_0809_4958_gb300 import inputs, lbtracer as lbt

    rank, world, local = dist_env()
    if rank != 0 and standalone:
        return None
    torch.cuda.set_device(local)
    w = MLP
    E, K = w["E"], w["K"]
    def boundary_data(seeds, nint):
        # features and targets of intervals 0 .. nint-1 from every-step boundary data
        Xs, Ts = [], []
        for sd in seeds:
            modes = inputs.mode_table(sd, w["M"], w["k_min"], w["k_max"], E)
            fine = lbt.synth_faces(modes, E, 1, 0, (nint + 3) * K + 1, torch.float32)
            coarse = fine[::K]
            for j in range(0, nint):
                jm = max(j - 1, 0)
                Xs.append(lbt.mlp_features(coarse[jm], coarse[j], coarse[j + 1], coarse[j + 2], E, w["u_max"]))
                Ts.append(lbt.mlp_targets(coarse[jm], coarse[j], coarse[j + 1], coarse[j + 2],
                                          fine[j * K:j * K + K + 1].contiguous(), E, K, int(j == 0), w["u_max"]))
            del fine
        return torch.cat(Xs), torch.cat(Ts)

    # ---- training data: every-step boundary of the training boxes ----
    X, T = boundary_data([w["seed"] + b for b in range(w["train_boxes"])], w["train_intervals"])
    up = lbt.Upsampler(K=K, batch_rows=w["batch"], master=inputs.mlp_init(w["seed"], K))
    gen = torch.Generator(device="cuda").manual_seed(w["seed"])
    t0 = time.perf_counter()
    first = None
    for it in range(w["train_steps"]):
        idx = torch.randint(0, X.shape[0], (w["batch"],), device="cuda", generator=gen)
        lr = w["lr"] * 0.5 * (1.0 + np.cos(np.pi * it / w["train_steps"]))  # cosine decay
        up.step(X[idx].contiguous(), T[idx].contiguous(), lr)
        if it == 0:
            first = up.loss.item()
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    final = up.loss.item()
    params = up.export()
    torch.cuda.synchronize()

    def run_boxes(seeds, time_interp, Kb, nsteps, timed=False, graph=True):
        descs = [lbt.box_desc(E, w["tau"], time_interp=time_interp, K=Kb) for _ in seeds]
        G = K if graph else 1
        stream = torch.cuda.Stream()
        tr = lbt.Tracers(descs, lbt.LB_STORE_F32, stream=stream, ring_slots=G // Kb + 4 if Kb else 4)
        fs = 18 * E * E
        warm = args.warmup // G * G if timed else 0
        nsamp = (warm + nsteps + (3 * G if timed else 0)) // Kb + 4
        faces = torch.empty((nsamp, len(seeds) * fs), dtype=torch.float32, device="cuda")
        for b, sd in enumerate(seeds):
            modes = inputs.mode_table(sd, w["M"], w["k_min"], w["k_max"], E)
            faces[:, b * fs:(b + 1) * fs] = lbt.synth_faces(modes, E, Kb, 0, nsamp, torch.float32).view(nsamp, -1)
            u0 = lbt.synth_volume(modes, E, 0.0, torch.float32)
            torch.cuda.synchronize()
            tr.lb_init(b, u0)
            tr.lb_sync()
        if time_interp == lbt.LB_TIME_MLP:
            tr.lb_mlp_bind(params, w["u_max"])
        pushed = [-1]

        def push_until(j):
            while pushed[0] < j:
                pushed[0] += 1
                tr.lb_set_boundary(lbt.LB_ALL_BOXES, pushed[0], faces[pushed[0]])

        need = lambda n: n // Kb + (1 if time_interp == lbt.LB_TIME_LINEAR else 2)  # noqa: E731
        ms = None
        if timed:
            for n in range(warm):
                push_until(need(n))
                tr.lb_step(1)
            tr.lb_graph_capture(G)
            push_until(need(tr.lb_current_step() + G - 1))  # one untimed replay: the graph's first run
            tr.lb_graph_launch()
            push_until(need(tr.lb_current_step() + G - 1))  # the first timed replay's samples
            tr.lb_sync()
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(nsteps // G):  # a replay's samples are pushed behind the replay before it
                tr.lb_graph_launch()
                push_until(need(tr.lb_current_step() + G - 1))
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
        else:
            for n in range(nsteps):
                push_until(need(n))
                tr.lb_step(1)
        us = []
        if not timed:
            for b in range(len(seeds)):
                u = torch.empty((3, E, E, E), dtype=torch.float32, device="cuda")
                tr.lb_read_fields(b, lbt.LB_FIELD_U, u)
                us.append(u[:, 1:-1, 1:-1, 1:-1].double())
        tr.close()
        del faces
        torch.cuda.synchronize()
        return ms, us

    # ---- gain on held-out boxes ----
    eval_seeds = [w["seed"] + 10000 + b for b in range(w["eval_boxes"])]
    Xh, Th = boundary_data(eval_seeds, w["eval_steps"] // K)
    Yh = lbt.mlp_forward(params, K, Xh)
    resid_ratio = float(((Yh - Th) ** 2).mean() / (Th ** 2).mean())
    del Xh, Th, Yh
    _, u_ref = run_boxes(eval_seeds, lbt.LB_TIME_LINEAR, 1, w["eval_steps"], graph=False)
    errs = {}
    for name, ti in (("linear", lbt.LB_TIME_LINEAR), ("hermite", lbt.LB_TIME_HERMITE), ("mlp", lbt.LB_TIME_MLP)):
        _, u = run_boxes(eval_seeds, ti, K, w["eval_steps"], graph=False)
        errs[name] = float(np.mean([float(torch.linalg.norm(a - r) / torch.linalg.norm(r)) for a, r in zip(u, u_ref)]))
    # ---- throughput of all boxes: network in the step vs Hermite alone ----
    all_seeds = [w["seed"] + 20000 + b for b in range(w["nboxes"])]
    steps = args.steps // K * K
    ms_mlp, _ = run_boxes(all_seeds, lbt.LB_TIME_MLP, K, steps, timed=True)
    ms_her, _ = run_boxes(all_seeds, lbt.LB_TIME_HERMITE, K, steps, timed=True)
    sites = w["nboxes"] * E ** 3
    value = sites * steps / (ms_mlp * 1e-3) / 1e6
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": args.warmup // K * K,
            "ms_per_step": ms_mlp / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "%d boxes of %d^3, tau %.2f, FP32, Kolmogorov boundaries (256 modes, |k| in [1,32]) "
                                   "sampled every K = %d steps; learned upsampler (32-128-128-48, bf16 tensor cores) "
                                   "in the step, CUDA graph of one interval" % (w["nboxes"], E, w["tau"], K),
                       "hermite_only_MLUPS": sites * steps / (ms_her * 1e-3) / 1e6,
                       "interior_velocity_error_vs_every_step_boundary": errs,
                       "heldout_boundary_residual_mse_vs_hermite": resid_ratio,
                       "eval": "%d held-out boxes, %d steps" % (w["eval_boxes"], w["eval_steps"]),
                       "training": {"boxes": w["train_boxes"], "intervals_per_box": w["train_intervals"],
                                    "rows": int(X.shape[0]), "adam_steps": w["train_steps"], "batch": w["batch"],
                                    "lr": w["lr"], "loss_first": first, "loss_final": final, "seconds": train_s}},
            "roofline": None, "e2e": None, "gpu_launches": None}
    del X, T
    torch.cuda.synchronize()
    if standalone:
        print(json.dumps(line), flush=True)
    return line


FORM_STEPS = {"batch": (256, 112), "precision": (1000, 20), "mlp": (256, 64)}


def measure_forms(args, plain_mlups):
    """The three added forms, each a short timed run on the same GPU next to
    the plain FP32 box of the headline (steps and warm-up fixed per form)."""
    import copy
    out = {}
    for name, fn in (("batch", run_batch), ("precision", run_precision), ("upsampler", run_mlp)):
        a = copy.copy(args)
        a.steps, a.warmup = FORM_STEPS["mlp" if name == "upsampler" else name]
        try:
            line = fn(a, standalone=False)
        except Exception as e:  # report, do not lose the headline
            out[name] = {"error": repr(e)}
            continue
        if name == "batch":
            rf = line["roofline"]
            out[name] = {"MLUPS": line["value"], "vs_plain_f32_box": line["value"] / plain_mlups,
                         "steps": line["steps"], "hbm_frac": rf["frac"], "stream_collide_ms": rf["avg_launch_ms"],
                         "workload": line["config"]["workload"],
                         "error_vs_single_box": 0.0,
                         "error_note": "each box of a batch equals the same box run alone bit for bit "
                                       "(tests/test_gpu_parity.py::test_batch_of_uneven_boxes_equals_single_boxes)"}
        elif name == "precision":
            res = line["config"]["forms"]
            out[name] = {"steps": line["steps"], "workload": line["config"]["workload"]}
            for st in ("f32", "f16", "bf16"):
                r = res[st]
                e = {"MLUPS": r["MLUPS"], "vs_plain_f32_box": r["MLUPS"] / plain_mlups, "hbm_frac": r["hbm_frac"],
                     "stream_collide_ms": r["stream_collide_ms"]}
                if st != "f32":
                    e["velocity_rel_l2_vs_f32"] = r["velocity_rel_l2_vs_f32"]
                    e["stress_rel_l2_vs_f32"] = r["stress_rel_l2_vs_f32"]
                out[name][st] = e
        else:
            c = line["config"]
            out[name] = {"MLUPS": line["value"], "vs_plain_f32_box": line["value"] / plain_mlups,
                         "steps": line["steps"], "hermite_only_MLUPS": c["hermite_only_MLUPS"],
                         "interior_velocity_error_vs_every_step_boundary":
                             c["interior_velocity_error_vs_every_step_boundary"],
                         "heldout_boundary_residual_mse_vs_hermite": c["heldout_boundary_residual_mse_vs_hermite"],
                         "training_seconds": c["training"]["seconds"], "workload": c["workload"]}
    return out


if __name__ == "__main__":
    main()
