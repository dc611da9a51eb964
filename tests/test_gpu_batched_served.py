"""Batched and served forms: the 64-world batch and the serving loop give
every world the result it has when stepped alone, and the alone runs match
the oracle (worlds 0-3 of the batch)."""
import numpy as np
import pytest

from paper_2302_09334_gb300.params import EcoParams, batched_64
from tests.parity import compare, rnn_close, run_forced, small_margin, sync_weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eco():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_09334_gb300 import build, world
    build.build()
    return world


def test_batched_64_worlds_equal_alone(eco):
    import torch
    specs = batched_64()
    stream = torch.cuda.Stream()
    worlds = [eco.World(p, s, stream=stream) for p, s in specs]
    batch = eco.Batch(worlds)
    batch.step(30)
    batch.sync()
    for i in (0, 1, 2, 3, 63):
        p, s = specs[i]
        alone = eco.World(p, s)
        alone.step(30)
        a, b = alone.read_state(), worlds[i].read_state()
        for k in a:
            np.testing.assert_array_equal(a[k], b[k], err_msg=f"world {i} {k}")
        alone.close()
    batch.close()
    for w in worlds:
        w.close()


@pytest.mark.parametrize("i", [0, 1, 2, 3])
def test_batched_64_worlds_0_to_3_match_oracle(eco, oracle, i):
    p, s = batched_64()[i]
    gw = eco.World(p, s)
    ow = oracle.OracleWorld(p.asdict(), s)
    compare(gw.read_state(), ow, f"batched world {i} init")
    run_forced(gw, ow, 20, f"batched world {i}", p.mut_std, compare_every=5)


def test_served_results_equal_alone(eco):
    from paper_2302_09334_gb300.serve import Server
    trace = []
    for k, (arr, h, w, n0, steps) in enumerate([(0.0, 20, 40, 60, 250), (0.0, 30, 60, 150, 420),
                                                (0.05, 12, 70, 40, 130), (0.1, 20, 40, 64, 300),
                                                (0.15, 50, 100, 300, 210)]):
        trace.append({"arrival": arr, "params": EcoParams(H=h, W=w, n_agents0=n0, capacity=4 * n0),
                      "seed": 100 + k, "steps": steps})
    srv = Server(budget_bytes=3 * 2**30, chunk=100, keep_final=True)
    rep = srv.run(trace)
    srv.close()
    assert rep["requests_completed"] == len(trace)
    assert rep["chunk_latency_p99_s"] is not None
    for r in srv.finished:
        alone = eco.World(r.params, r.seed)
        alone.step(r.steps)
        a = alone.read_state()
        assert int(a["counters"][0]) == r.steps
        for k in a:
            np.testing.assert_array_equal(a[k], r.final[k], err_msg=f"request {r.rid} {k}")
        alone.close()


def test_served_cancel_mid_chunk_equals_alone(eco):
    """A cancellation that arrives inside a chunk retires the request at the
    end of that chunk; its state is a world stepped alone for the steps it
    completed, and the requests that shared its launches are unaffected."""
    from paper_2302_09334_gb300.serve import Server
    trace = [{"arrival": 0.0, "params": EcoParams(H=20, W=40, n_agents0=60, capacity=240),
              "seed": 7, "steps": 500, "cancel_after_steps": 130},
             {"arrival": 0.0, "params": EcoParams(H=30, W=60, n_agents0=150, capacity=600),
              "seed": 8, "steps": 300}]
    srv = Server(budget_bytes=3 * 2**30, chunk=100, keep_final=True)
    rep = srv.run(trace)
    srv.close()
    assert rep["requests_cancelled"] == 1 and rep["requests_completed"] == 1
    for r in srv.cancelled + srv.finished:
        assert r.done == (200 if r.rid == 0 else 300)
        alone = eco.World(r.params, r.seed)
        alone.step(r.done)
        a = alone.read_state()
        for k in a:
            np.testing.assert_array_equal(a[k], r.final[k], err_msg=f"request {r.rid} {k}")
        alone.close()


def test_served_trace_shaped_requests_match_oracle(eco, oracle):
    """Three requests shaped like the serving trace's (grids 50x100, 100x200,
    200x400; 250-400 agents, capacity 4x) served together for 20 steps in
    one launch; each final state equals, bit for bit, a world of the same
    spec stepped alone one step at a time, and that world matches the
    oracle at every step: the oracle moves with the actions the GPU took and
    is compared after each step from the same state (run_gpu_driven:
    integer state and energies bit for bit, h, c and logits within the RNN
    tolerance, an argmax difference only at a flagged near-tie)."""
    from paper_2302_09334_gb300.serve import Server
    from tests.parity import run_gpu_driven
    specs = [(EcoParams(H=50, W=100, n_agents0=300, capacity=1200), 200),
             (EcoParams(H=100, W=200, n_agents0=250, capacity=1000), 201),
             (EcoParams(H=200, W=400, n_agents0=400, capacity=1600), 202)]
    trace = [{"arrival": 0.0, "params": p, "seed": s, "steps": 20} for p, s in specs]
    srv = Server(budget_bytes=3 * 2**30, chunk=100, keep_final=True)
    rep = srv.run(trace)
    srv.close()
    assert rep["requests_completed"] == 3 and rep["batch_launches"] == 1
    for r in srv.finished:
        ow = oracle.OracleWorld(r.params.asdict(), r.seed)
        alone = eco.World(r.params, r.seed)
        st = run_gpu_driven(alone, ow, r.steps, f"served request {r.rid}")
        a = alone.read_state()
        for k in a:
            np.testing.assert_array_equal(a[k], r.final[k], err_msg=f"request {r.rid} {k}")
        print(f"served request {r.rid}: {st}")
        assert st["flagged"] <= 2
        alone.close()
        ow.close()
