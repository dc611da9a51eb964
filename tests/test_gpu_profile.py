"""Per-kernel profiling (kernels launched on the stream with events around
each) and graph stepping give the same states as plain steps."""
import numpy as np
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


def test_profiled_steps_equal_plain_steps(eco):
    p = small_20x40()
    a = eco.World(p, 21)
    b = eco.World(p, 21)
    a.profile(True, max_steps=8)
    a.step(12)          # 8 profiled, 4 past the cap
    b.step(12)
    prof = a.profile_read()
    assert prof["observe_lstm"][1] == 8 and prof["observe_lstm"][0] > 0
    assert prof["regrow_spawn"][1] == 8 and prof["agents_fused"][1] == 8
    a.step(3)
    prof2 = a.profile_read()
    assert prof2["observe_lstm"][1] == 11   # the cap restarts after each read
    a.profile(False)
    a.step(2)
    b.step(5)
    sa, sb = a.read_state(), b.read_state()
    for k in sa:
        np.testing.assert_array_equal(sa[k], sb[k], err_msg=k)
