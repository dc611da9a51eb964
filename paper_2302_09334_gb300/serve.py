"""Serving loop: simulation requests (world spec, seed, number of steps)
admitted by a device-memory budget and stepped together by continuous
batching.

Every live world stays resident on the device (grid, agents, weights)
between chunks.  Each iteration of the loop admits the requests that have
arrived, in arrival order, while their arenas fit in the budget; steps every
live world by one chunk (at most `chunk` steps, fewer when a request needs
fewer) with one launch per kernel for all of them; reports each request's
progress; and retires the requests that are done, freeing their memory for
the queue.  A request's result does not depend on which others share its
launches (every random draw is keyed by its own seed and step).

Latency accounting: a request's chunk latency is the time between two
consecutive chunk reports (the first from its admission); the queueing
delay is admission time minus arrival time.
"""
from __future__ import annotations

import ctypes
import time
from collections import deque

import numpy as np

from . import _lib
from .world import Batch, World


class Request:
    __slots__ = ("rid", "arrival", "params", "seed", "steps", "nbytes", "world", "done",
                 "admitted", "last_report", "latencies", "agent_steps", "final")

    def __init__(self, rid, arrival, params, seed, steps):
        self.rid, self.arrival, self.params, self.seed, self.steps = rid, arrival, params, seed, steps
        c = _lib.to_c_params(params)
        self.nbytes = int(_lib.lib().eco_world_bytes(ctypes.byref(c))) + 256
        self.world = None
        self.done = 0
        self.admitted = None
        self.last_report = None
        self.latencies = []
        self.agent_steps = 0
        self.final = None


class Server:
    def __init__(self, budget_bytes: float = 120e9, chunk: int = 100, device: int = 0,
                 keep_final: bool = False):
        import torch
        self.budget = float(budget_bytes)
        self.chunk = int(chunk)
        self.device = device
        self.keep_final = keep_final
        self.stream = torch.cuda.Stream(device)
        self.used = 0
        self.live: list[Request] = []
        self.finished: list[Request] = []
        self._batch = None
        self._batch_members = ()

    def _admit(self, req: Request, now: float) -> None:
        req.world = World(req.params, req.seed, device=self.device, stream=self.stream)
        req.admitted = now
        req.last_report = now
        self.used += req.nbytes
        self.live.append(req)

    def _retire(self, req: Request) -> None:
        if self.keep_final:
            req.final = req.world.read_state()
        req.world.close()
        req.world = None
        self.used -= req.nbytes
        self.finished.append(req)

    def _step_live(self, n: int) -> None:
        members = tuple(id(r) for r in self.live)
        if members != self._batch_members:
            if self._batch is not None:
                self._batch.close()
            self._batch = Batch([r.world for r in self.live])
            self._batch_members = members
        self._batch.step(n)
        self._batch.sync()

    def run(self, trace, duration_s: float | None = None, max_wall_s: float | None = None):
        """Serve the requests of `trace` (dicts with arrival, params, seed,
        steps; arrivals in seconds from the start).  Arrivals after
        duration_s are ignored; the loop stops when every admitted request
        is done, or at max_wall_s (requests still running are cut off)."""
        pending = deque(sorted(
            (Request(i, r["arrival"], r["params"], r["seed"], r["steps"])
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
            while queue and self.used + queue[0].nbytes <= self.budget:
                self._admit(queue.popleft(), time.perf_counter() - t0)
            if not self.live:
                if not pending and not queue:
                    break
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                continue
            n = min(self.chunk, min(r.steps - r.done for r in self.live))
            pops = [int(r.world.counters()[1]) for r in self.live]
            self._step_live(n)
            chunks += 1
            t_rep = time.perf_counter() - t0
            for r, pop in zip(list(self.live), pops):
                r.done += n
                r.agent_steps += pop * n  # population at the chunk start
                if r.done % self.chunk == 0 or r.done == r.steps:
                    r.latencies.append(t_rep - r.last_report)
                    r.last_report = t_rep
                if r.done == r.steps:
                    self.live.remove(r)
                    self._retire(r)
        self.wall = time.perf_counter() - t0
        self.unfinished = list(self.live) + list(queue)
        self.chunks = chunks
        return self.report()

    def report(self) -> dict:
        reqs = self.finished + [r for r in self.unfinished if r.world is not None]
        lat = np.array([x for r in reqs for x in r.latencies], np.float64)
        agent_steps = sum(r.agent_steps for r in reqs)
        delays = [r.admitted - r.arrival for r in reqs if r.admitted is not None]
        return {
            "agent_steps_per_s": agent_steps / self.wall if self.wall > 0 else 0.0,
            "chunk_latency_p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "chunk_latency_p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "chunks_reported": int(lat.size),
            "requests_admitted": len(reqs),
            "requests_completed": len(self.finished),
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
