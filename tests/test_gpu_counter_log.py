"""The per-step counter log (eco_world_counter_log): the step kernels write
every step's counters into page-locked host memory, on both slot paths, in
graph chunks and in batches; rows wrap around; invalid buffers are refused
and leave the log as it was."""
import ctypes

import numpy as np
import pytest

from paper_2302_09334_gb300.params import EcoParams

pytestmark = pytest.mark.gpu

P = EcoParams(H=30, W=60, capacity=600, n_agents0=150, t_repr=25, e_repr=0.4, max_age=140)


@pytest.fixture(scope="module")
def eco():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_09334_gb300 import build, world
    build.build()
    return world


def _pinned_log(rows):
    import torch
    from paper_2302_09334_gb300._lib import NCOUNTERS
    return torch.full((rows, NCOUNTERS), -1, dtype=torch.int64, pin_memory=True)


def _per_step_counters(eco, steps, seed):
    """The counters after each step, read one step at a time."""
    w = eco.World(P, seed=seed)
    out = []
    for _ in range(steps):
        w.step(1)
        out.append(w.counters().copy())
    w.close()
    return np.array(out)


@pytest.mark.parametrize("fused", [1, 0])
def test_log_holds_every_steps_counters(eco, fused):
    steps = 120
    ref = _per_step_counters(eco, steps, seed=23)
    assert ref[-1, 2] > 0                     # births happened
    w = eco.World(P, seed=23)
    w.set_config(fused=fused, steps_per_graph=16)
    log = _pinned_log(200)
    w.counter_log(log)
    w.step(steps)                             # 7 graph chunks of 16 steps + 8 single steps
    w.sync()
    np.testing.assert_array_equal(log.numpy()[:steps], ref)
    assert (log.numpy()[steps:] == -1).all()
    np.testing.assert_array_equal(w.counters(), ref[-1])
    w.close()


def test_log_wraps_and_turns_off(eco):
    ref = _per_step_counters(eco, 25, seed=4)
    w = eco.World(P, seed=4)
    log = _pinned_log(7)
    w.counter_log(log)
    w.step(20)
    w.sync()
    for t in range(13, 20):
        np.testing.assert_array_equal(log.numpy()[t % 7], ref[t], err_msg=f"step {t}")
    before = log.numpy().copy()
    w.counter_log(None)
    w.step(5)
    w.sync()
    np.testing.assert_array_equal(log.numpy(), before)
    np.testing.assert_array_equal(w.counters(), ref[24])
    w.close()


def test_log_in_a_batch(eco):
    seeds = (8, 9)
    refs = [_per_step_counters(eco, 40, seed=s) for s in seeds]
    worlds = [eco.World(P, seed=s) for s in seeds]
    logs = [_pinned_log(40) for _ in seeds]
    for w, log in zip(worlds, logs):
        w.counter_log(log)
    b = eco.Batch(worlds)
    b.step(40)
    b.sync()
    for log, ref in zip(logs, refs):
        np.testing.assert_array_equal(log.numpy(), ref)
    b.close()
    for w in worlds:
        w.close()


def test_invalid_buffers_are_refused(eco):
    import torch
    from paper_2302_09334_gb300._lib import ECO_EINVAL, lib
    ref = _per_step_counters(eco, 3, seed=2)
    w = eco.World(P, seed=2)
    log = _pinned_log(4)
    w.counter_log(log)
    L, h = lib(), w.handle
    pageable = np.zeros((4, 9), dtype=np.int64)
    device = torch.zeros((4, 9), dtype=torch.int64, device=w.device)
    assert L.eco_world_counter_log(h, ctypes.c_void_p(pageable.ctypes.data), 4) == ECO_EINVAL
    assert L.eco_world_counter_log(h, ctypes.c_void_p(device.data_ptr()), 4) == ECO_EINVAL
    assert L.eco_world_counter_log(h, ctypes.c_void_p(log.data_ptr() + 4), 3) == ECO_EINVAL
    assert L.eco_world_counter_log(h, ctypes.c_void_p(log.data_ptr()), 0) == ECO_EINVAL
    assert L.eco_world_counter_log(None, ctypes.c_void_p(log.data_ptr()), 4) == ECO_EINVAL
    w.step(3)                                 # the first log is still on
    w.sync()
    np.testing.assert_array_equal(log.numpy()[:3], ref)
    assert (pageable == 0).all()
    w.counter_log(None)
    w.close()
