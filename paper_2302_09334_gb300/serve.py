"""Serving loop: simulation requests (world spec, seed, number of steps)
admitted by a device-memory budget and stepped together by continuous
batching.

Every live world stays resident on the device (grid, agents, weights)
between chunks.  Each iteration of the loop admits the requests that have
arrived, in arrival order, while their arenas fit in the budget (and, with a
chunk-latency target, while the live agents fit in it); steps every live
world together, with one launch per kernel for all of them, up to the next
step at which some live request reports (a request reports every `chunk`
of its own steps and at its last step, so requests at different points of
their 100-step cycles share shorter launches); reports; and retires the
requests that are done, freeing their memory for the queue.  A request's
result does not depend on which others share its launches (every random
draw is keyed by its own seed and step).

Latency accounting: a request's chunk latency is the time between two
consecutive reports (the first from its admission); the queueing delay is
admission time minus arrival time.

Latency control: with target_chunk_s, a request is admitted only while the
agents of the live worlds plus its own, stepped `chunk` times at the
measured rate (agent-steps/s, a moving average over launches, from
rate_prior until measured; fixed at rate_prior with learn_rate=False), fit
in 70 % of the target (the rest is left for the births of admitted worlds);
the first request is always admitted.  The memory budget
still applies.

With `log` (a text file), every chunk appends one JSON record: its time,
steps, live and queued requests, agent-steps, seconds, agent-steps/s and the
device memory in use.

Failures and cancellation, all handled on the host between chunks (no
launch is ever interrupted):
* a request whose arena alone exceeds the budget is rejected on arrival;
* a world whose creation runs out of device memory goes back to the head of
  the queue until a retirement frees memory, or is rejected when nothing is
  live (no memory can come back);
* a cancellation (Server.cancel, from any thread, or a trace entry's
  cancel_after_steps) that arrives while a chunk runs takes effect at the end
  of that chunk: the request retires with the steps it has completed, and its
  state is that of a world stepped alone for that many steps.
"""
from __future__ import annotations

import ctypes
import json
import threading
import time
from collections import deque

import numpy as np

from . import _lib
from .world import Batch, World


class Request:
    __slots__ = ("rid", "arrival", "params", "seed", "steps", "nbytes", "world", "done",
                 "admitted", "last_report", "latencies", "agent_steps", "final",
                 "cancel_after_steps", "outcome", "pop")

    def __init__(self, rid, arrival, params, seed, steps, cancel_after_steps=None):
        self.rid, self.arrival, self.params, self.seed, self.steps = rid, arrival, params, seed, steps
        c = _lib.to_c_params(params)
        nbytes = int(_lib.lib().eco_world_bytes(ctypes.byref(c)))
        if nbytes == 0:
            raise ValueError(f"request {rid}: invalid world parameters")
        self.nbytes = nbytes + 256
        self.cancel_after_steps = cancel_after_steps
        self.world = None
        self.done = 0
        self.admitted = None
        self.last_report = None
        self.latencies = []
        self.agent_steps = 0
        self.pop = int(params.n_agents0)   # population at the last launch
        self.final = None
        self.outcome = None   # "done" | "cancelled" | "rejected: <why>" | None (cut off)


def _out_of_memory(e: BaseException) -> bool:
    if isinstance(e, MemoryError) or type(e).__name__ == "OutOfMemoryError":
        return True
    return isinstance(e, _lib.EcoError) and e.code == _lib.ECO_ENOMEM


class Server:
    """world_factory(params, seed) and batch_factory(worlds) default to
    World on this server's stream and Batch."""

    def __init__(self, budget_bytes: float = 120e9, chunk: int = 100, device: int = 0,
                 keep_final: bool = False, world_factory=None, batch_factory=None,
                 log=None, target_chunk_s: float | None = None, rate_prior: float = 5e7,
                 learn_rate: bool = True):
        self.budget = float(budget_bytes)
        self.chunk = int(chunk)
        self.target = None if target_chunk_s is None else float(target_chunk_s)
        self.rate = float(rate_prior)   # agent-steps/s of a launch, moving average
        self.learn_rate = learn_rate
        self.live_agents = 0            # agents of the live worlds at the last launch
        self.device = device
        self.keep_final = keep_final
        if world_factory is None:
            import torch
            self.stream = torch.cuda.Stream(device)
            world_factory = lambda p, seed: World(p, seed, device=device, stream=self.stream)
        self._new_world = world_factory
        self._new_batch = batch_factory or Batch
        self.used = 0
        self.live: list[Request] = []
        self.finished: list[Request] = []
        self.cancelled: list[Request] = []
        self.rejected: list[Request] = []
        self._batch = None
        self._batch_members = ()
        self._lock = threading.Lock()
        self._cancel_ids = set()
        self._wait_for_retire = False   # set by an out-of-memory admission
        self.log = log                  # text file: one JSON record per chunk

    def cancel(self, rid: int) -> None:
        """Ask for request rid to stop (safe from any thread).  A queued
        request is dropped; a live one retires at the end of its chunk."""
        with self._lock:
            self._cancel_ids.add(rid)

    def _take_cancels(self) -> set:
        with self._lock:
            ids, self._cancel_ids = self._cancel_ids, set()
        return ids

    def _admit(self, req: Request, now: float) -> None:
        req.world = self._new_world(req.params, req.seed)
        req.admitted = now
        req.last_report = now
        self.used += req.nbytes
        self.live.append(req)

    def _retire(self, req: Request, outcome: str) -> None:
        if self.keep_final:
            req.final = req.world.read_state()
        req.world.close()
        req.world = None
        self.used -= req.nbytes
        self.live_agents -= req.pop
        self._wait_for_retire = False
        req.outcome = outcome
        (self.finished if outcome == "done" else self.cancelled).append(req)

    def _reject(self, req: Request, why: str) -> None:
        req.outcome = f"rejected: {why}"
        self.rejected.append(req)

    # share of the target left for the growth of admitted populations
    # (births after admission; capacities are 4x the initial populations)
    TARGET_HEADROOM = 0.65

    def _fits_target(self, req: Request) -> bool:
        if self.target is None or not self.live:
            return True
        agents = self.live_agents + int(req.params.n_agents0)
        return agents * self.chunk / self.rate <= self.TARGET_HEADROOM * self.target

    def _admit_queue(self, queue: deque, now: float) -> None:
        """Admit from the head of the queue, in arrival order, while the
        arenas fit in the budget, the live agents fit in the chunk-latency
        target and the device has the memory."""
        while queue and not self._wait_for_retire:
            req = queue[0]
            if req.nbytes > self.budget:
                queue.popleft()
                self._reject(req, "arena larger than the memory budget")
                continue
            if self.used + req.nbytes > self.budget or not self._fits_target(req):
                return
            try:
                self._admit(req, now)
                self.live_agents += int(req.params.n_agents0)
            except Exception as e:
                if not _out_of_memory(e):
                    raise
                if self.live:
                    self._wait_for_retire = True   # retry once memory is freed
                    return
                queue.popleft()
                self._reject(req, "out of device memory with nothing live")
                continue
            queue.popleft()

    def _populations(self) -> list:
        """Population of every live world: one asynchronous counter copy per
        world into page-locked memory, one wait (fake worlds: counters())."""
        worlds = [r.world for r in self.live]
        if not worlds or not hasattr(worlds[0], "counters_async"):
            return [int(w.counters()[1]) for w in worlds]
        import torch
        if getattr(self, "_ctr_host", None) is None or self._ctr_host.shape[0] < len(worlds):
            self._ctr_host = torch.zeros((max(64, 2 * len(worlds)), _lib.NCOUNTERS),
                                         dtype=torch.int64, pin_memory=True)
        for i, w in enumerate(worlds):
            w.counters_async(self._ctr_host[i])
        worlds[0].stream.synchronize()
        return [int(v) for v in self._ctr_host[:len(worlds), _lib.C_POP].tolist()]

    def _step_live(self, n: int) -> None:
        members = tuple(id(r) for r in self.live)
        if members != self._batch_members:
            if self._batch is not None:
                self._batch.close()
            self._batch = self._new_batch([r.world for r in self.live])
            self._batch_members = members
        self._batch.step(n)
        self._batch.sync()

    def run(self, trace, duration_s: float | None = None, max_wall_s: float | None = None):
        """Serve the requests of `trace` (dicts with arrival, params, seed,
        steps, optionally cancel_after_steps; arrivals in seconds from the
        start).  Arrivals after duration_s are ignored; the loop stops when
        every request is done, cancelled or rejected, or at max_wall_s
        (requests still running are cut off)."""
        pending = deque(sorted(
            (Request(i, r["arrival"], r["params"], r["seed"], r["steps"],
                     r.get("cancel_after_steps"))
             for i, r in enumerate(trace)
             if duration_s is None or r["arrival"] < duration_s),
            key=lambda q: q.arrival))
        queue: deque[Request] = deque()
        t0 = time.perf_counter()
        self.t_start = t0
        chunks = 0
        while True:
            now = time.perf_counter() - t0
            if max_wall_s is not None and now >= max_wall_s:
                break
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            cancels = self._take_cancels()
            if cancels:
                for r in [q for q in queue if q.rid in cancels]:
                    queue.remove(r)
                    r.outcome = "cancelled"
                    self.cancelled.append(r)
                for r in [q for q in self.live if q.rid in cancels]:
                    self.live.remove(r)
                    self._retire(r, "cancelled")
                # a cancel for a request not yet arrived waits for it
                with self._lock:
                    self._cancel_ids |= {q.rid for q in pending if q.rid in cancels}
            self._admit_queue(queue, time.perf_counter() - t0)
            if not self.live:
                if not pending and not queue:
                    break
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                continue
            # up to the next report of any live request
            n = min(min(self.chunk - r.done % self.chunk, r.steps - r.done) for r in self.live)
            pops = self._populations()
            self.live_agents = sum(pops)
            t_chunk = time.perf_counter()
            self._step_live(n)
            chunks += 1
            t_rep = time.perf_counter() - t0
            dt_launch = time.perf_counter() - t_chunk
            if self.learn_rate and dt_launch > 0 and self.live_agents > 0:
                self.rate += 0.2 * (self.live_agents * n / dt_launch - self.rate)
            if self.log is not None:
                dt = time.perf_counter() - t_chunk
                self.log.write(json.dumps({
                    "t_s": round(t_rep, 6), "chunk": chunks, "steps": n,
                    "live": len(self.live), "queued": len(queue),
                    "agent_steps": sum(pops) * n, "seconds": round(dt, 6),
                    "agent_steps_per_s": sum(pops) * n / dt if dt > 0 else None,
                    "used_gb": round(self.used / 1e9, 3)}) + "\n")
            for r, pop in zip(list(self.live), pops):
                r.done += n
                r.pop = pop
                r.agent_steps += pop * n  # population at the launch start
                if r.done % self.chunk == 0 or r.done == r.steps:
                    r.latencies.append(t_rep - r.last_report)
                    r.last_report = t_rep
                if r.done == r.steps:
                    self.live.remove(r)
                    self._retire(r, "done")
                elif r.cancel_after_steps is not None and r.done >= r.cancel_after_steps:
                    self.live.remove(r)
                    self._retire(r, "cancelled")
        self.wall = time.perf_counter() - t0
        self.unfinished = list(self.live) + list(queue) + list(pending)
        self.chunks = chunks
        return self.report()

    def report(self, warm_s: float = 0.0) -> dict:
        """Throughput and latency over the run; with warm_s, the steady-state
        p50/p99 over the reports of requests admitted after warm_s."""
        reqs = self.finished + self.cancelled + [r for r in self.unfinished
                                                 if r.world is not None]
        lat = np.array([x for r in reqs for x in r.latencies], np.float64)
        agent_steps = sum(r.agent_steps for r in reqs)
        delays = [r.admitted - r.arrival for r in reqs if r.admitted is not None]
        steady = np.array([x for r in reqs if r.admitted is not None and r.admitted >= warm_s
                           for x in r.latencies], np.float64)
        return {
            "agent_steps_per_s": agent_steps / self.wall if self.wall > 0 else 0.0,
            "chunk_latency_p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "chunk_latency_p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "chunks_reported": int(lat.size),
            "steady_after_s": warm_s,
            "steady_chunk_latency_p50_s": float(np.percentile(steady, 50)) if steady.size else None,
            "steady_chunk_latency_p99_s": float(np.percentile(steady, 99)) if steady.size else None,
            "steady_chunks_reported": int(steady.size),
            "target_chunk_s": self.target,
            "requests_admitted": sum(1 for r in reqs if r.admitted is not None),
            "requests_completed": len(self.finished),
            "requests_cancelled": len(self.cancelled),
            "requests_rejected": len(self.rejected),
            "queue_delay_mean_s": float(np.mean(delays)) if delays else None,
            "wall_s": self.wall,
            "batch_launches": self.chunks,
        }

    def close(self) -> None:
        if self._batch is not None:
            self._batch.close()
            self._batch = None
        for r in self.live:
            r.world.close()
            r.world = None
        self.live.clear()


def serve_sequential(trace, duration_s: float | None = None, max_wall_s: float | None = None,
                     device: int = 0) -> dict:
    """Comparison point: the same requests processed one at a time, each as a
    plain single world stepped alone, in arrival order."""
    import torch
    stream = torch.cuda.Stream(device)
    reqs = sorted((r for r in trace if duration_s is None or r["arrival"] < duration_s),
                  key=lambda r: r["arrival"])
    t0 = time.perf_counter()
    agent_steps, lat = 0, []
    completed = 0
    for r in reqs:
        now = time.perf_counter() - t0
        if max_wall_s is not None and now >= max_wall_s:
            break
        if r["arrival"] > now:
            time.sleep(r["arrival"] - now)
        w = World(r["params"], r["seed"], device=device, stream=stream)
        last = time.perf_counter()
        done = 0
        while done < r["steps"]:
            if max_wall_s is not None and time.perf_counter() - t0 >= max_wall_s:
                break
            n = min(100, r["steps"] - done)
            pop = int(w.counters()[1])
            w.step(n)
            w.sync()
            done += n
            agent_steps += pop * n
            t = time.perf_counter()
            lat.append(t - last)
            last = t
        completed += done == r["steps"]
        w.close()
    wall = time.perf_counter() - t0
    lat = np.array(lat)
    return {"agent_steps_per_s": agent_steps / wall if wall > 0 else 0.0,
            "chunk_latency_p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "chunk_latency_p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "requests_completed": completed, "wall_s": wall}
