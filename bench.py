"""Throughput of the simulation step on GB300: agent-steps/s at 200x400.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload paper_200x400|large_1000x2000|small_20x40]

A step is one pass of the whole path (regrowth, observation + LSTM, moves,
physiology, births) over one world.  The world is synthetic (seeded), shaped
like the paper's natural environment: a 200x400 grid, 1000 agents at the
start, capacity 8192, free-running population.  Inputs fit in L2 (129 MB),
so L2 is flushed before every timed step (a 256 MB write, then a 256 MB read
of another buffer so that the lines left in L2 are clean); each step is timed
with CUDA events on the world's stream and the step times are summed.

Under torchrun (N > 1) every rank steps its own world (seed = rank): worlds
are independent, there is no collective on the data path ("replicas only").
--impl reference times the CPU oracle on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# algorithmic bytes of the observation + LSTM kernel per agent:
# 93,332 B of weights (4 blocks + read-out), h and c read and written
# (4 x 128 B), position, energy, action and logits (36 B)
LSTM_BYTES_PER_AGENT = 93332 + 512 + 36
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (read + write) of one observation+LSTM launch per agent, from an
# ncu capture of this kernel on the 200x400 world with 1,000 agents held
# (97.17 MB, mean of two launches); traffic grows with the agents of a
# launch, so it is scaled by them.
LSTM_TRAFFIC_PER_AGENT = 97.17e6 / 1000


# the same for the paper's controller: 2,445 FP32 parameters, h and c of 4
# units read and written, position, previous action (read + written), ate,
# logits and action
PAPER_BYTES_PER_AGENT = 2445 * 4 + 32 + 8 + 8 + 1 + 20 + 4


def lstm_bytes(n_agents: int, H: int, W: int, controller: int = 0) -> int:
    # + the three observation channels of the grid, one bit per cell
    per = PAPER_BYTES_PER_AGENT if controller == 1 else LSTM_BYTES_PER_AGENT
    return n_agents * per + 3 * H * W // 8


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_worker(args):
    """One host process: the oracle stepping one world (its own seed) until
    the step count or the time budget runs out.  Returns (agent-steps,
    steps, seconds)."""
    params_dict, seed, budget_s, warmup, max_steps = args
    sys.path.insert(0, ROOT)
    from oracle import pyoracle
    # the error magnitudes the oracle keeps for the parity tests are not part
    # of the step: off for the timing
    ow = pyoracle.OracleWorld(params_dict, seed, magnitudes=False)
    for _ in range(warmup):
        ow.step()
    agent_steps, steps = 0, 0
    t0 = time.perf_counter()
    while steps < max_steps and (time.perf_counter() - t0) < budget_s:
        agent_steps += ow.population
        ow.step()
        steps += 1
    dt = time.perf_counter() - t0
    ow.close()
    return agent_steps, steps, dt


def run_oracle_pool(params, budget_s: float, warmup: int, max_steps: int, cores: int):
    """The oracle on `cores` host processes, one independent world each
    (seeds 0..cores-1), as they stand.  Processes are spawned (never forked
    from a process that has used the GPU).  Returns (agent-steps/s, steps of
    each world, seconds)."""
    import multiprocessing as mp
    from oracle import build as oracle_build
    oracle_build.build()
    jobs = [(params.asdict(), i, budget_s, warmup, max_steps) for i in range(cores)]
    if cores == 1:
        res = [_oracle_worker(jobs[0])]
    else:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_worker, jobs)
    agent_steps = sum(r[0] for r in res)
    wall = max(r[2] for r in res)
    return agent_steps / wall, [r[1] for r in res], wall


def bench_reference(args, params, rank, world_size):
    if rank != 0:
        return
    cores = args.cpu_cores or os.cpu_count() or 1
    v, steps, dt = run_oracle_pool(params, 1e9, args.warmup, args.steps, cores)
    line = {
        "impl": "reference", "metric": "agent-steps/s at 200x400", "value": v,
        "unit": "agent-steps/s", "n_gpus": world_size, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(args, params),
        "cpu_baseline": {"kind": "oracle", "cores": cores, "value": v, "unit": "agent-steps/s",
                         "sample": f"{args.workload}, {cores} independent worlds (seeds "
                                   f"0..{cores - 1}) on {cores} host processes, steps "
                                   f"{args.warmup + 1}..{args.warmup + args.steps} each, "
                                   "single-threaded C oracle"},
        "e2e": {"value": v, "unit": "agent-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(args, params):
    return {"workload": args.workload, "H": params.H, "W": params.W,
            "n_agents0": params.n_agents0, "capacity": params.capacity, "seed": "rank",
            "population": "held" if args.held else "free-running",
            "l2": "flushed before every step (256 MB write + 256 MB read)",
            "parallelism": f"replicas{args.gpus}"}


CONFIG_KEYS = ("fused", "spawn_ctas_per_sm", "steps_per_graph")
SHAPE_KEYS = ("regrow_rows_per_cta", "lstm_ctas_per_sm")


def configure(target, cfg: dict) -> None:
    """Launch configuration and kernel shapes (a tuner record, or the
    get_config() + get_shape() of a world) applied to a world or batch."""
    target.set_config(**{k: cfg[k] for k in CONFIG_KEYS})
    target.set_shape(**{k: cfg[k] for k in SHAPE_KEYS})


def flushed_shape_check(make_world, cfg: dict, flush, flush_read, sink, steps: int = 8,
                        rounds: int = 4):
    """Controller CTAs per SM (1 or 2) timed with L2 flushed before every
    step, as the timed region runs: one fresh world per shape (from
    `make_world()`, the same seed), `rounds` rounds of `steps` one-step
    graphs each, round-robin between the two, all before the first births
    (so both time the population the timed steps have); the lower median
    decides (the tuner's own choice, made with the weights left in L2, gets
    no precedence).  Returns the configuration and the medians."""
    import statistics
    import torch
    worlds = {}
    for lc in (1, 2):
        w = make_world()
        configure(w, {**cfg, "steps_per_graph": 1, "lstm_ctas_per_sm": lc})
        w.step(1)   # the one-step graph captured before the timing
        w.sync()
        worlds[lc] = w
    times = {1: [], 2: []}
    for _ in range(rounds):
        for lc, w in worlds.items():
            stream = w.stream
            for _ in range(steps):
                with torch.cuda.stream(stream):
                    flush.fill_(1)
                    torch.sum(flush_read, dim=0, out=sink)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                w.step(1)
                e1.record(stream)
                e1.synchronize()
                times[lc].append(e0.elapsed_time(e1))
    for w in worlds.values():
        w.close()
    med = {lc: statistics.median(v) for lc, v in times.items()}
    out = dict(cfg)
    out["lstm_ctas_per_sm"] = min(med, key=med.get)
    return out, {"flushed_step_ms_lstm_ctas_1": med[1], "flushed_step_ms_lstm_ctas_2": med[2],
                 "chosen": out["lstm_ctas_per_sm"]}


def to_pinned(state: dict) -> dict:
    """The same arrays in page-locked host memory (numpy views of pinned
    torch tensors), so that host-to-device copies from them are DMA
    transfers."""
    import numpy as np
    import torch
    out = {}
    for k, v in state.items():
        v = np.ascontiguousarray(v)
        t = torch.empty(v.shape, dtype=torch.from_numpy(v[:0].copy()).dtype, pin_memory=True)
        out[k] = t.numpy()
        out[k][...] = v
    return out


def analysis_summary(windows, life_expectancy):
    """The e2e leg's 50-step analysis windows (App. C) in short: the last
    window's population, resources and displacement bins, and the life
    expectancy pooled over all windows."""
    if not windows:
        return None
    last = windows[-1]
    return {"windows": len(windows), "window_steps": last["window"], "t": last["t"],
            "population": last["population"], "resources": last["resources"],
            "movers": last["movers"], "move_bins": [int(v) for v in last["move_bins"]],
            "life_expectancy": life_expectancy(windows)}


def reduce_over_ranks(stats, dist, n_times: int):
    """Whole-job figures from one rank's 1-D tensor [times..., units...]:
    the first n_times entries take the maximum over ranks (the job lasts as
    long as its slowest rank), the others the sum (every rank steps its own
    independent world).  Without a process group the rank's own values."""
    if dist is None:
        return [float(v) for v in stats]
    mx = stats.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = stats.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return [float(mx[i]) if i < n_times else float(sm[i]) for i in range(stats.numel())]


def bench_ours(args, params, rank, world_size, dist):
    import torch
    from paper_2302_09334_gb300 import build as lib_build
    lib_build.build()
    from paper_2302_09334_gb300._lib import lib
    from paper_2302_09334_gb300.world import World

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    flush_read = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    flush_sink = torch.empty((), dtype=torch.float32, device=dev)
    # launch configuration: tuned on a world of the same shape (seed + 1000)
    # so that the measured world starts from step 0
    shape_check = None
    if args.no_tune:
        probe = World(params, seed=1000 + rank, device=local)
        cfg = {**probe.get_config(), **probe.get_shape()}
        probe.close()
        if args.lstm_ctas:
            cfg["lstm_ctas_per_sm"] = args.lstm_ctas
    else:
        tuner = World(params, seed=1000 + rank, device=local)
        tuned = tuner.autotune(trial_steps=8)
        cfg = {k: tuned[k] for k in CONFIG_KEYS + SHAPE_KEYS}
        tuner.close()
        del tuner
        if args.lstm_ctas:
            cfg["lstm_ctas_per_sm"] = args.lstm_ctas
        elif params.controller == 0:
            # the tuner's trials run back to back, with the weights left in
            # L2 from step to step, and reach populations the timed steps do
            # not; the timed steps start from a flushed L2, where the
            # controller kernel's shape matters more: both shapes are timed
            # again that way on another fresh world of the same shape (one-step
            # graphs, flush before each)
            cfg, shape_check = flushed_shape_check(
                lambda: World(params, seed=2000 + rank, device=local), cfg, flush, flush_read,
                flush_sink)
    # the timed world steps by plain one-step CUDA graphs; its twin (same
    # seed, hence the same states step by step) launches each step's kernels
    # on the stream with CUDA events around every kernel for the per-kernel
    # times
    world = World(params, seed=rank, device=local)
    twin = World(params, seed=rank, device=local, stream=world.stream)
    configure(world, cfg)
    configure(twin, cfg)
    stream = world.stream
    kps = lib().eco_kernels_per_step(world.handle)

    def flush_l2():
        # write a buffer larger than L2, then read another one: no input of
        # the step stays in L2 and the lines left there are clean
        with torch.cuda.stream(stream):
            flush.fill_(1)
            torch.sum(flush_read, dim=0, out=flush_sink)

    for _ in range(args.warmup):
        flush_l2()
        world.step(1)
        twin.step(1)
    world.sync()

    # host copy of the state the timed steps start from (input of the e2e leg)
    alive_slots = world.read_state(fields=("alive",))["alive"].nonzero()[0]
    hi = int(alive_slots.max()) + 1 if alive_slots.size else 0
    e2e_state = to_pinned(world.read_state(weights=(0, hi)))

    twin.profile(True, max_steps=args.steps)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    pops = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            pops.append(int(world.counters()[1]))
            flush_l2()
            twin.step(1)
            flush_l2()
            starts[k].record(stream)
            world.step(1)
            ends[k].record(stream)
        world.sync()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    prof = twin.profile_read()
    twin.profile(False)
    if int(twin.counters()[1]) != int(world.counters()[1]):
        raise RuntimeError("the profiled twin diverged from the timed world")
    twin.close()
    agent_steps = sum(pops)
    cell_steps = params.H * params.W * args.steps

    # e2e through the C ABI with host buffers, over the same steps as the
    # timed region: the state they start from (with the weights of every
    # living agent) is uploaded from host memory; the steps run as a user
    # runs them (world.step over 50-step windows, in the world's graph
    # chunks), and every step's counters reach page-locked host memory
    # through the counter log, written by the kernel that ends the step;
    # after every 50 steps (the movement window of the paper's analyses,
    # App. C) the window's analysis record (population, resources, deaths
    # and ages, displacement bins) is copied back too.
    import numpy as np
    from paper_2302_09334_gb300._lib import C_AGENT_STEPS, C_T, NANALYSIS, NCOUNTERS
    h2d = sum(v.nbytes for k, v in e2e_state.items() if k not in ("slot_map",))
    counter_log = torch.full((args.steps, NCOUNTERS), -1, dtype=torch.int64, pin_memory=True)
    counters0 = torch.empty(NCOUNTERS, dtype=torch.int64, pin_memory=True)
    analysis_host = torch.empty((args.steps // 50 + 1, NANALYSIS), dtype=torch.int64,
                                pin_memory=True)
    world.counter_log(counter_log)
    e_steps0 = torch.cuda.Event(enable_timing=True)
    e_steps1 = torch.cuda.Event(enable_timing=True)
    # warm-up of the path (its first calls load kernels, touch the buffers
    # and capture the step graphs the timed calls replay), then the timed
    # region without Python's cyclic collector
    world.load_state(e2e_state)
    done = 0
    while done < args.steps:
        n = min(50, args.steps - done)
        world.step(n)
        done += n
    world.sync()
    gc.collect()
    gc.disable()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    world.load_state(e2e_state)
    t_loaded = time.perf_counter()
    e_steps0.record(stream)
    world.counters_async(counters0)
    d2h = NCOUNTERS * 8
    done = 0
    while done < args.steps:
        n = min(50, args.steps - done)
        world.step(n)
        done += n
        d2h += n * NCOUNTERS * 8
        if n == 50:
            world.analysis_async(analysis_host[done // 50 - 1])
            d2h += NANALYSIS * 8
    e_steps1.record(stream)
    world.sync()
    e2e_dt = time.perf_counter() - t0
    gc.enable()
    e2e_load_s = t_loaded - t0
    e2e_steps_ms = e_steps0.elapsed_time(e_steps1)
    world.counter_log(None)
    t_first = int(counters0[C_T])
    rows = counter_log.numpy()[[(t_first + k) % args.steps for k in range(args.steps)]]
    if (rows[:, C_T] != np.arange(t_first + 1, t_first + args.steps + 1)).any():
        raise RuntimeError("the counter log misses steps of the e2e leg")
    e2e_agent_steps = int(rows[-1, C_AGENT_STEPS] - counters0[C_AGENT_STEPS])
    d2h //= args.steps
    from paper_2302_09334_gb300.world import analysis_record, life_expectancy
    windows = [analysis_record(r) for r in analysis_host[:args.steps // 50].numpy()]

    stats = torch.tensor([total_ms, e2e_dt, float(agent_steps), float(cell_steps),
                          float(e2e_agent_steps)], dtype=torch.float64, device=dev)
    total_ms, e2e_dt, agent_steps, cell_steps, e2e_agent_steps = \
        reduce_over_ranks(stats, dist, n_times=2)
    if rank != 0:
        return
    value = agent_steps / (total_ms / 1e3)
    ctrl_kernel = "observe_paper" if params.controller == 1 else "observe_lstm"
    lstm_ms, lstm_n = prof[ctrl_kernel]
    peak, peak_kind = load_peaks()
    bytes_lstm = sum(lstm_bytes(n, params.H, params.W, params.controller) for n in pops)
    achieved = bytes_lstm / (lstm_ms / 1e3) / 1e9 if lstm_ms > 0 else None
    line = {
        "metric": "agent-steps/s at 200x400", "value": value, "unit": "agent-steps/s",
        "n_gpus": world_size, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_of(args, params),
        "cell_steps_per_s": cell_steps / (total_ms / 1e3),
        "mean_population": agent_steps / max(args.steps * world_size, 1),
        "kernel_ms_per_step": {k: v[0] / v[1] for k, v in prof.items() if v[1]},
        "roofline": {"kernel": ctrl_kernel, "bound": "hbm", "achieved": achieved,
                     "peak": peak, "peak_kind": f"{peak_kind} hbm_gbs", "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None,
                     "traffic": (LSTM_TRAFFIC_PER_AGENT * (sum(pops) / max(len(pops), 1))
                                 if params.controller == 0 and LSTM_TRAFFIC_PER_AGENT else None),
                     "bytes_per_launch": bytes_lstm / max(lstm_n, 1)},
        "gpu_launches": kps * args.steps,
        "launch_config": cfg,
        "shape_check": shape_check,
        "e2e": {"value": e2e_agent_steps / e2e_dt, "unit": "agent-steps/s",
                "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h,
                "load_state_ms": e2e_load_s * 1e3, "steps_device_ms": e2e_steps_ms,
                "wall_ms": e2e_dt * 1e3},
        "clocks": clocks.summary(),
        "analysis": analysis_summary(windows, life_expectancy),
    }
    if world_size == 1 and not args.no_many:
        legs = {"batched": bench_batched, "served": bench_served,
                "paper_preset": bench_paper_preset, "large": bench_large, "held": bench_held}
        for name, leg in legs.items():
            if args.legs is None or name in args.legs:
                line[name] = leg(args, local)
    if not args.no_cpu_baseline:
        cores = args.cpu_cores or os.cpu_count() or 1
        v, steps, dt = run_oracle_pool(params, args.cpu_budget, 0, 100000, cores)
        line["cpu_baseline"] = {
            "value": v, "unit": "agent-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{args.workload}, {cores} independent worlds (seeds 0..{cores - 1}) on "
                      f"{cores} host processes, first {min(steps)}-{max(steps)} steps each "
                      f"({dt:.1f} s), single-threaded C oracle"}
        # the parity configuration in full (20x40, 64 agents, 500 steps), one process
        from paper_2302_09334_gb300.params import small_20x40
        a_s, n_s, dt_s = _oracle_worker((small_20x40().asdict(), 0, 1e9, 0, 500))
        line["cpu_baseline"]["small_20x40_full"] = {
            "value": a_s / dt_s, "unit": "agent-steps/s", "cores": 1, "steps": n_s,
            "seconds": dt_s}
    print(json.dumps(line), flush=True)


def bench_batched(args, local):
    """64 worlds of mixed sizes stepped together (one launch per kernel per
    step), run in CUDA-graph chunks whose length and launch shapes the tuner
    picks on a twin batch (same shapes, other seeds).  The timed region is
    one call of batched_steps steps; agent-steps come from the worlds'
    cumulative counters.  ~12 GB of weights per step: inputs far larger than
    L2, no flush."""
    import torch
    from paper_2302_09334_gb300._lib import C_AGENT_STEPS
    from paper_2302_09334_gb300.params import batched_64
    from paper_2302_09334_gb300.world import Batch, World
    specs = batched_64()
    stream = torch.cuda.Stream(local)
    # tuner: a twin batch of the same worlds with seeds 1000+, first stepped
    # past the first births (step 50) so that its trials see the mutation
    # load the timed steps have
    tw = [World(p, 1000 + s, device=local, stream=stream) for p, s in specs]
    tb = Batch(tw)
    tb.step(args.batched_warmup + 60)
    tb.sync()
    tuned = tb.autotune(trial_steps=4)
    tb.close()
    for w in tw:
        w.close()
    del tw
    torch.cuda.empty_cache()
    worlds = [World(p, s, device=local, stream=stream) for p, s in specs]
    batch = Batch(worlds)
    configure(batch, tuned)
    batch.step(args.batched_warmup)
    batch.sync()
    pops0 = [int(w.counters()[1]) for w in worlds]
    as0 = sum(int(w.counters()[C_AGENT_STEPS]) for w in worlds)
    torch.cuda.synchronize()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    batch.step(args.batched_steps)
    end.record(stream)
    end.synchronize()
    total_ms = start.elapsed_time(end)
    agent_steps = sum(int(w.counters()[C_AGENT_STEPS]) for w in worlds) - as0
    batch.close()
    for w in worlds:
        w.close()
    del worlds, batch
    torch.cuda.empty_cache()
    # per-kernel times over the same steps: a twin batch (same worlds and
    # seeds, hence the same states step by step) repeats warm-up and timed
    # steps with its kernels bracketed by events
    worlds = [World(p, s, device=local, stream=stream) for p, s in specs]
    batch = Batch(worlds)
    configure(batch, tuned)
    batch.step(args.batched_warmup)
    batch.sync()
    worlds[0].profile(True, max_steps=args.batched_steps)
    as1 = sum(int(w.counters()[C_AGENT_STEPS]) for w in worlds)
    batch.step(args.batched_steps)
    batch.sync()
    prof = worlds[0].profile_read()
    worlds[0].profile(False)
    prof_agent_steps = sum(int(w.counters()[C_AGENT_STEPS]) for w in worlds) - as1
    if prof_agent_steps != agent_steps:
        raise RuntimeError("the profiled twin batch diverged from the timed batch")
    lstm_ms, _ = prof["observe_lstm"]
    cells = sum(p.H * p.W for p, _ in specs)
    bytes_lstm = prof_agent_steps * LSTM_BYTES_PER_AGENT + \
        args.batched_steps * sum(3 * p.H * p.W // 8 for p, _ in specs)
    peak, kind = load_peaks()
    achieved = bytes_lstm / (lstm_ms / 1e3) / 1e9 if lstm_ms > 0 else None
    out = {"workload": "batched_64", "worlds": len(specs), "steps": args.batched_steps,
           "warmup": args.batched_warmup, "value": agent_steps / (total_ms / 1e3),
           "unit": "agent-steps/s", "ms_per_step": total_ms / args.batched_steps,
           "cell_steps_per_s": cells * args.batched_steps / (total_ms / 1e3),
           "mean_population": agent_steps / args.batched_steps,
           "initial_population": sum(pops0),
           "launch_config": {k: tuned[k] for k in CONFIG_KEYS + SHAPE_KEYS},
           "tuner": {"steps_taken": tuned["steps_taken"],
                     "ms_per_step_initial": tuned["ms_per_step_initial"],
                     "ms_per_step_best": tuned["ms_per_step_best"]},
           "kernel_ms_per_step": {k: v[0] / v[1] for k, v in prof.items() if v[1]},
           "kernel_sum_ms_per_step": sum(v[0] for v in prof.values()) / args.batched_steps,
           "kernel_times": "twin batch over the same steps, kernels on the stream between "
                           "CUDA events (no overlap between them)",
           "roofline": {"kernel": "observe_lstm", "bound": "hbm", "achieved": achieved,
                        "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak if achieved else None},
           "l2": "inputs larger than L2 (about 12 GB of weights per step)"}
    batch.close()
    for w in worlds:
        w.close()
    torch.cuda.empty_cache()
    return out


def bench_paper_preset(args, local):
    """The paper's own natural environment (App. B.4, B.5): 200x400 grid, 330
    agents at the start (at most 1000), the CNN+LSTM(4) controller with
    sampled actions.  The world (~10 MB of weights) stays in L2 over a long
    run, as it would over the paper's 10^6 steps, so it is not flushed; the
    timed region is one call of paper_steps steps (CUDA-graph chunks of the
    tuned length).  The paper reports 10^6 steps in about 20 minutes on an
    unnamed GPU (App. B.4): about 833 steps/s."""
    import torch
    from paper_2302_09334_gb300._lib import C_AGENT_STEPS
    from paper_2302_09334_gb300.params import paper_natural
    from paper_2302_09334_gb300.world import World
    p = paper_natural()
    stream = torch.cuda.Stream(local)
    tuner = World(p, 1000, device=local, stream=stream)
    tuned = tuner.autotune(trial_steps=16)
    tuner.close()
    cfg = {k: tuned[k] for k in CONFIG_KEYS + SHAPE_KEYS}
    w = World(p, 0, device=local, stream=stream)
    configure(w, cfg)
    w.step(args.paper_warmup)
    w.sync()
    c0 = w.counters()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    w.step(args.paper_steps)
    end.record(stream)
    end.synchronize()
    ms = start.elapsed_time(end)
    c1 = w.counters()
    agent_steps = int(c1[C_AGENT_STEPS] - c0[C_AGENT_STEPS])
    w.profile(True, max_steps=200)
    w.step(200)
    prof = w.profile_read()
    w.profile(False)
    w.close()
    steps_per_s = args.paper_steps / (ms / 1e3)
    return {"workload": "paper_natural", "steps": args.paper_steps,
            "warmup": args.paper_warmup, "steps_per_s": steps_per_s,
            "agent_steps_per_s": agent_steps / (ms / 1e3), "ms_per_step": ms / args.paper_steps,
            "mean_population": agent_steps / args.paper_steps,
            "population_end": int(c1[1]), "births": int(c1[2] - c0[2]),
            "deaths": int(c1[3] - c0[3]),
            "launch_config": cfg,
            "kernel_ms_per_step": {k: v[0] / v[1] for k, v in prof.items() if v[1]},
            "minutes_per_1e6_steps": 1e6 / steps_per_s / 60.0,
            "paper_context": "10^6 steps in about 20 min on an unnamed GPU, JAX (App. B.4): "
                             "about 833 steps/s",
            "l2": "not flushed: the world (about 10 MB of weights) stays L2-resident over a run"}


def bench_large(args, local):
    """The 1000x2000 world (20,000 agents at the start, capacity 131,072,
    12.2 GB of weight rows; slot phases on the grid-wide kernels): one world
    whose weights per step (1.9 GB and growing) are far larger than L2, so no
    flush.  Plain steps timed one call at a time, then as many profiled
    steps of a twin (same seed) for the per-kernel times."""
    import torch
    from paper_2302_09334_gb300._lib import C_AGENT_STEPS
    from paper_2302_09334_gb300.params import large_1000x2000
    from paper_2302_09334_gb300.world import World
    p = large_1000x2000()
    stream = torch.cuda.Stream(local)
    w = World(p, 0, device=local, stream=stream)
    twin = World(p, 0, device=local, stream=stream)
    w.step(args.large_warmup)
    twin.step(args.large_warmup)
    w.sync()
    a0 = int(w.counters()[C_AGENT_STEPS])
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    w.step(args.large_steps)
    end.record(stream)
    end.synchronize()
    ms = start.elapsed_time(end)
    agent_steps = int(w.counters()[C_AGENT_STEPS]) - a0
    twin.profile(True, max_steps=args.large_steps)
    t0 = int(twin.counters()[C_AGENT_STEPS])
    twin.step(args.large_steps)
    prof = twin.profile_read()
    twin.profile(False)
    prof_agent_steps = int(twin.counters()[C_AGENT_STEPS]) - t0
    w.close()
    twin.close()
    torch.cuda.empty_cache()
    lstm_ms, _ = prof["observe_lstm"]
    bytes_lstm = prof_agent_steps * LSTM_BYTES_PER_AGENT + args.large_steps * 3 * p.H * p.W // 8
    peak, kind = load_peaks()
    achieved = bytes_lstm / (lstm_ms / 1e3) / 1e9 if lstm_ms > 0 else None
    return {"workload": "large_1000x2000", "steps": args.large_steps,
            "warmup": args.large_warmup, "value": agent_steps / (ms / 1e3),
            "unit": "agent-steps/s", "ms_per_step": ms / args.large_steps,
            "cell_steps_per_s": p.H * p.W * args.large_steps / (ms / 1e3),
            "mean_population": agent_steps / args.large_steps,
            "kernel_ms_per_step": {k: v[0] / v[1] for k, v in prof.items() if v[1]},
            "roofline": {"kernel": "observe_lstm", "bound": "hbm", "achieved": achieved,
                         "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak if achieved else None},
            "l2": "inputs larger than L2 (about 1.9 GB of weights per step), not flushed"}


def bench_held(args, local):
    """Held populations (no energy decay, no reproduction: the agent count
    stays at n_agents0), the roofline microbenchmark: 1,000 agents at
    200x400 (93 MB of weights, less than L2: flushed before every step),
    20,000 agents at 1000x2000 and 131,072 (every slot) at 1000x2000 (1.9 and
    12.2 GB per step, larger than L2: not flushed).  Plain steps timed with
    CUDA events, per-kernel times from a profiled twin (same seed)."""
    import torch
    from paper_2302_09334_gb300.params import held, large_1000x2000, paper_200x400
    from paper_2302_09334_gb300.world import World
    peak, kind = load_peaks()
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(local)
    big = large_1000x2000()
    cases = [("paper_200x400", held(paper_200x400()), True),
             ("large_1000x2000", held(big), False),
             ("large_1000x2000_full", held(big.replace(n_agents0=big.capacity)), False)]
    out = []
    for name, p, flushed in cases:
        w = World(p, 0, device=local, stream=stream)
        twin = World(p, 0, device=local, stream=stream)
        # no births in a held population: one mutation CTA per SM
        w.set_config(steps_per_graph=1, spawn_ctas_per_sm=1)
        twin.set_config(steps_per_graph=1, spawn_ctas_per_sm=1)
        w.step(args.held_warmup)
        twin.step(args.held_warmup)
        n = int(w.counters()[1])
        if flushed:
            flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
            flush_read = torch.ones(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
            sink = torch.empty((), dtype=torch.float32, device=dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.held_steps if flushed else 1)]
        twin.profile(True, max_steps=args.held_steps)
        torch.cuda.synchronize()
        if flushed:
            for k in range(args.held_steps):
                with torch.cuda.stream(stream):
                    flush.fill_(1)
                    torch.sum(flush_read, dim=0, out=sink)
                    twin.step(1)
                    flush.fill_(1)
                    torch.sum(flush_read, dim=0, out=sink)
                ev[k][0].record(stream)
                w.step(1)
                ev[k][1].record(stream)
        else:
            ev[0][0].record(stream)
            w.step(args.held_steps)
            ev[0][1].record(stream)
            twin.step(args.held_steps)
        w.sync()
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        prof = twin.profile_read()
        twin.profile(False)
        if int(w.counters()[1]) != n or int(twin.counters()[1]) != n:
            raise RuntimeError(f"held population changed in {name}")
        w.close()
        twin.close()
        lstm_ms, lstm_n = prof["observe_lstm"]
        bytes_lstm = lstm_n * lstm_bytes(n, p.H, p.W)
        achieved = bytes_lstm / (lstm_ms / 1e3) / 1e9 if lstm_ms > 0 else None
        out.append({"workload": name, "agents": n, "steps": args.held_steps,
                    "ms_per_step": ms / args.held_steps,
                    "agent_steps_per_s": n * args.held_steps / (ms / 1e3),
                    "kernel_ms_per_step": {k: v[0] / v[1] for k, v in prof.items() if v[1]},
                    "roofline": {"kernel": "observe_lstm", "bound": "hbm", "achieved": achieved,
                                 "peak": peak, "peak_kind": f"{kind} hbm_gbs", "unit": "GB/s",
                                 "frac": achieved / peak if achieved else None},
                    "l2": ("flushed before every step" if flushed
                           else "inputs larger than L2, not flushed")})
        torch.cuda.empty_cache()
    return out


def bench_served(args, local):
    """Serving: Poisson request arrivals (20/s), admission by a 120 GB
    device-memory budget and a chunk-latency target, continuous batching
    with reports every 100 steps of each request; the same arrival trace
    processed one request at a time as the comparison.  The offered load
    (about 20 requests/s x 1,600 agents x 10,500 steps) is several times what
    one GPU steps, so the queue grows and admission decides the latency: the
    line reports the p50/p99 report interval of all requests and of those
    admitted after a warm-up (steady state) beside the target."""
    import torch
    from paper_2302_09334_gb300.params import serve_trace
    from paper_2302_09334_gb300.serve import Server, serve_sequential
    trace = serve_trace(duration_s=args.serve_seconds)
    srv = Server(budget_bytes=120e9, chunk=100, device=local,
                 target_chunk_s=args.serve_target)
    srv.run(trace, duration_s=args.serve_seconds, max_wall_s=args.serve_seconds)
    rep = srv.report(warm_s=min(args.serve_warm, args.serve_seconds / 2))
    srv.close()
    torch.cuda.empty_cache()
    seq = serve_sequential(trace, duration_s=args.serve_seconds,
                           max_wall_s=args.serve_seconds / 2, device=local)
    torch.cuda.empty_cache()
    rep.update({"trace": f"Poisson 20/s arrivals over the first {args.serve_seconds:.0f} s "
                         "(grids 50x100/100x200/200x400, 200-3000 agents, 1000-20000 steps)",
                "budget_gb": 120, "chunk_steps": 100,
                "sequential": seq})
    return rep


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper_200x400")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--cpu-cores", type=int, default=0,
                    help="host processes for the oracle (default: all cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--held-steps", type=int, default=50)
    ap.add_argument("--held-warmup", type=int, default=3)
    ap.add_argument("--held", action="store_true",
                    help="no energy decay and no births: the population stays at n_agents0")
    ap.add_argument("--n-agents", type=int, default=None, help="override n_agents0")
    ap.add_argument("--legs", nargs="+", default=None,
                    choices=("batched", "served", "paper_preset", "large", "held"),
                    help="run only these extra legs (default: all)")
    ap.add_argument("--no-many", action="store_true",
                    help="skip the batched (64 worlds) and served measurements")
    ap.add_argument("--batched-steps", type=int, default=1000)
    ap.add_argument("--batched-warmup", type=int, default=10)
    ap.add_argument("--serve-seconds", type=float, default=120.0,
                    help="length of the served request trace and of the serving run "
                         "(600: the whole 10-minute trace)")
    ap.add_argument("--serve-warm", type=float, default=30.0,
                    help="requests admitted after this many seconds give the steady-state "
                         "latency")
    ap.add_argument("--serve-target", type=float, default=0.1,
                    help="chunk-latency target (s per 100-step report) for admission")
    ap.add_argument("--no-tune", action="store_true",
                    help="default launch configuration (no tuner world before the timed one)")
    ap.add_argument("--lstm-ctas", type=int, choices=(1, 2), default=None,
                    help="controller-kernel CTAs per SM of the headline world (default: "
                         "the tuner's choice checked with flushed steps, or 1 with --no-tune)")
    ap.add_argument("--large-steps", type=int, default=100)
    ap.add_argument("--large-warmup", type=int, default=10)
    ap.add_argument("--paper-steps", type=int, default=20000)
    ap.add_argument("--paper-warmup", type=int, default=100)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    from paper_2302_09334_gb300.params import PRESETS
    params = PRESETS[args.workload]()
    if args.n_agents is not None:
        params = params.replace(n_agents0=args.n_agents)
    if args.held:
        from paper_2302_09334_gb300.params import held
        params = held(params)

    rank = int(os.environ.get("RANK", "0"))
    world_size = int(os.environ.get("WORLD_SIZE", "1"))
    dist = None
    if world_size > 1 and args.impl == "ours":
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    try:
        if args.impl == "reference":
            bench_reference(args, params, rank, world_size)
        else:
            bench_ours(args, params, rank, world_size, dist)
    finally:
        if dist:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
