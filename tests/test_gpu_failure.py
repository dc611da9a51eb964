"""Failure detection on the GPU without a fault: a bounded device wait that
runs out reports ECO_ETIMEOUT through the world's status word, and the
context stays usable afterwards."""
import time

import pytest

from paper_2302_09334_gb300.params import small_20x40

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eco():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_09334_gb300 import build, world
    build.build()
    return world


def test_bounded_wait_times_out_and_context_survives(eco):
    from paper_2302_09334_gb300._lib import ECO_ETIMEOUT, EcoError, check, lib
    w = eco.World(small_20x40(), 5)
    w.step(3)
    w.sync()
    t0 = time.perf_counter()
    check(lib().eco_world_selftest_timeout(w.handle, 50_000_000), "selftest")  # 50 ms
    with pytest.raises(EcoError) as e:
        w.sync()
    assert e.value.code == ECO_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    check(lib().eco_world_clear_status(w.handle), "clear")
    w.step(5)
    w.sync()  # the context still works
    assert int(w.counters()[0]) == 8
