"""Host logic of the serving loop on CPU, with fake worlds in place of the
device ones: admission by the memory budget, rejection of requests that can
never fit, out-of-memory requeueing, and cancellation (from the trace and
from another thread, while a chunk runs).  No GPU is touched; the request
sizes come from the library's eco_world_bytes."""
import numpy as np
import pytest

from paper_2302_09334_gb300.params import EcoParams


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2302_09334_gb300 import build
    build.build()


class FakeWorld:
    created = []

    def __init__(self, p, seed):
        self.p, self.seed, self.t, self.closed = p, seed, 0, False
        FakeWorld.created.append(self)

    def counters(self):
        return np.array([self.t, self.p.n_agents0, 0, 0, 0, 0, 0, 0], np.int64)

    def read_state(self):
        return {"counters": self.counters()}

    def close(self):
        assert not self.closed
        self.closed = True


class FakeBatch:
    log = []          # (number of worlds, steps) of every batch step
    on_step = None    # hook called inside a step ("while the chunk runs")

    def __init__(self, worlds):
        self.worlds = worlds

    def step(self, n):
        assert all(not w.closed for w in self.worlds)
        FakeBatch.log.append((len(self.worlds), n))
        if FakeBatch.on_step:
            FakeBatch.on_step()
        for w in self.worlds:
            w.t += n

    def sync(self):
        pass

    def close(self):
        pass


def _req(arrival, n0, steps, seed=0, **kw):
    return dict(arrival=arrival, params=EcoParams(H=20, W=40, n_agents0=n0, capacity=4 * n0),
                seed=seed, steps=steps, **kw)


def _server(budget, factory=FakeWorld, **kw):
    from paper_2302_09334_gb300.serve import Server
    FakeWorld.created.clear()
    FakeBatch.log.clear()
    FakeBatch.on_step = None
    return Server(budget_bytes=budget, chunk=100, world_factory=factory,
                  batch_factory=FakeBatch, **kw)


def _size(n0):
    from paper_2302_09334_gb300.serve import Request
    return Request(0, 0.0, _req(0, n0, 1)["params"], 0, 1).nbytes


def test_budget_bounds_the_live_set():
    sz = _size(64)
    srv = _server(2.5 * sz, keep_final=True)
    rep = srv.run([_req(0.0, 64, s, seed=k) for k, s in enumerate((300, 200, 400, 100))])
    assert rep["requests_completed"] == 4 and rep["requests_rejected"] == 0
    assert max(n for n, _ in FakeBatch.log) == 2
    assert all(r.final["counters"][0] == r.steps for r in srv.finished)
    assert all(w.closed for w in FakeWorld.created) and srv.used == 0
    # requests 2 and 3 waited for memory: admitted after the first retirement
    by_rid = {r.rid: r for r in srv.finished}
    assert by_rid[2].admitted >= by_rid[1].admitted and len(FakeWorld.created) == 4
    assert rep["chunk_latency_p99_s"] is not None
    assert rep["agent_steps_per_s"] > 0


def test_oversize_request_is_rejected_not_stuck():
    big, small = 512, 64
    srv = _server(1.5 * _size(small))
    rep = srv.run([_req(0.0, big, 100), _req(0.0, small, 200, seed=1)], max_wall_s=30)
    assert rep["requests_rejected"] == 1 and rep["requests_completed"] == 1
    assert srv.rejected[0].rid == 0 and srv.rejected[0].outcome.startswith("rejected")
    assert rep["wall_s"] < 30


def test_out_of_memory_requeues_until_memory_is_freed():
    fail = {"left": 1}

    def flaky(p, seed):
        if seed == 1 and fail["left"]:
            fail["left"] -= 1
            raise MemoryError("simulated device allocation failure")
        return FakeWorld(p, seed)

    srv = _server(10 * _size(64), factory=flaky)
    rep = srv.run([_req(0.0, 64, 300, seed=0), _req(0.0, 64, 100, seed=1)], max_wall_s=30)
    assert rep["requests_completed"] == 2 and rep["requests_rejected"] == 0
    # request 1 ran only after request 0 had retired
    assert FakeBatch.log[:3] == [(1, 100)] * 3 and FakeBatch.log[3] == (1, 100)
    assert len(FakeBatch.log) == 4


def test_out_of_memory_with_nothing_live_is_rejected():
    def broke(p, seed):
        raise MemoryError("simulated device allocation failure")

    srv = _server(10 * _size(64), factory=broke)
    rep = srv.run([_req(0.0, 64, 100)], max_wall_s=30)
    assert rep["requests_rejected"] == 1 and "memory" in srv.rejected[0].outcome
    assert srv.used == 0


def test_other_errors_propagate():
    def bad(p, seed):
        raise ValueError("not a memory error")

    srv = _server(10 * _size(64), factory=bad)
    with pytest.raises(ValueError):
        srv.run([_req(0.0, 64, 100)])


def test_cancel_after_steps_takes_effect_at_chunk_end():
    srv = _server(10 * _size(64), keep_final=True)
    rep = srv.run([_req(0.0, 64, 1000, seed=0, cancel_after_steps=150),
                   _req(0.0, 64, 400, seed=1)])
    assert rep["requests_cancelled"] == 1 and rep["requests_completed"] == 1
    c = srv.cancelled[0]
    assert c.rid == 0 and c.outcome == "cancelled" and c.done == 200
    assert c.final["counters"][0] == 200 and c.world is None
    assert srv.finished[0].done == 400 and srv.used == 0


def test_cancel_from_another_thread_mid_chunk():
    srv = _server(10 * _size(64))
    calls = {"n": 0}

    def hook():
        calls["n"] += 1
        if calls["n"] == 2:       # the cancel arrives during the second chunk
            srv.cancel(1)
            srv.cancel(2)         # still queued (budget below)
            srv.cancel(99)        # unknown: ignored

    FakeBatch.on_step = hook
    srv.budget = 2.5 * _size(64)
    rep = srv.run([_req(0.0, 64, 500, seed=0), _req(0.0, 64, 500, seed=1),
                   _req(0.0, 64, 500, seed=2)])
    assert rep["requests_cancelled"] == 2 and rep["requests_completed"] == 1
    by_rid = {r.rid: r for r in srv.cancelled}
    assert by_rid[1].done == 200            # ran to the end of its chunk
    assert by_rid[2].admitted is None and by_rid[2].world is None
    assert len(FakeWorld.created) == 2 and all(w.closed for w in FakeWorld.created)


def test_chunk_log_is_jsonl():
    import io
    import json
    buf = io.StringIO()
    srv = _server(10 * _size(64), log=buf)
    srv.run([_req(0.0, 64, 250, seed=0), _req(0.0, 64, 120, seed=1)])
    recs = [json.loads(ln) for ln in buf.getvalue().splitlines()]
    # launches end where a request reports or finishes: 100, 20 (request
    # 1 done), 80 (request 0 reports at its step 200), 50
    assert [r["steps"] for r in recs] == [100, 20, 80, 50]
    assert [r["live"] for r in recs] == [2, 2, 1, 1]
    assert all(r["agent_steps"] == 64 * r["steps"] * r["live"] for r in recs)


def test_every_request_reports_every_chunk_of_its_own_steps():
    """Requests whose step counts are not multiples of the chunk share
    launches cut at the next report of any of them: each reports at every
    multiple of 100 of its own steps and at its last step."""
    srv = _server(1e12)
    steps = (250, 420, 135, 999, 100)
    trace = [_req(0.0, 64, s, seed=k) for k, s in enumerate(steps)]
    trace.append(_req(0.0, 64, 330, seed=9))
    rep = srv.run(trace)
    assert rep["requests_completed"] == len(trace)
    for r in srv.finished:
        assert len(r.latencies) == r.steps // 100 + (1 if r.steps % 100 else 0), \
            (r.steps, len(r.latencies))
    # no launch crosses a report: launches end at a multiple of 100 of some request
    assert all(n <= 100 for _, n in FakeBatch.log)
    assert sum(n for _, n in FakeBatch.log) == 999


def test_latency_target_bounds_the_live_agents():
    """With a chunk-latency target, a request waits while the live agents
    plus its own would take longer than 65 % of the target per chunk at the
    server's rate: here 2 x 64 agents x 100 steps / 1e4 agent-steps/s = 1.28 s
    fits in 0.65 x 2.0 s, 3 x 64 does not."""
    srv = _server(1e12, target_chunk_s=2.0, rate_prior=1e4, learn_rate=False)
    seen = []
    FakeBatch.on_step = lambda: seen.append(len(srv.live))
    rep = srv.run([_req(0.0, 64, 100, seed=k) for k in range(5)])
    assert rep["requests_completed"] == 5
    assert max(seen) <= 2
