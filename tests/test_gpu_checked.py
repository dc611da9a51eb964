"""The range-checked build (libecoevo_checked.so, ECO_CHECKED=1): every index
the kernels read from device memory is checked before use.  Forced parity
runs on both slot-phase paths, free runs at 200x400 (in both kernel shapes),
a mixed batch, the
paper's controller, the analysis and lab calls all finish with no index out
of range (eco_world_sync / eco_batch_sync would return ECO_EBOUNDS), and the
checked library's results equal the regular one's.  Runs in a child process
so that it loads the checked library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2302_09334_gb300 import build
build.build(checked=True)
from paper_2302_09334_gb300 import _lib, world
from paper_2302_09334_gb300.params import EcoParams, paper_200x400, small_20x40
from oracle import pyoracle
from tests.parity import run_forced
assert _lib.LIB_PATH.endswith("libecoevo_checked.so")

p = small_20x40().replace(capacity=300, max_age=140)
for fused in (1, 0):
    gw = world.World(p, seed=3)
    gw.set_config(fused=fused)
    ow = pyoracle.OracleWorld(p.asdict(), 3)
    run_forced(gw, ow, 200, f"checked fused={fused}", p.mut_std, compare_every=25)
    gw.sync()
    gw.close()

big = paper_200x400()
states = []
for fused in (1, 0):
    w = world.World(big, seed=1)
    w.set_config(fused=fused, spawn_ctas_per_sm=2 if fused else 8)
    if not fused:   # the other kernel shapes too
        w.set_shape(regrow_rows_per_cta=2, lstm_ctas_per_sm=2)
    w.step(100)
    w.analysis()
    w.lab_window()
    w.sync()
    states.append(w.read_state(fields=("alive", "y", "x", "energy", "age", "res")))
    w.close()
for k in states[0]:
    np.testing.assert_array_equal(states[0][k], states[1][k], err_msg=k)

specs = [(EcoParams(H=20 + 7 * i, W=40 + 11 * i, n_agents0=30 + 20 * i,
                    capacity=4 * (30 + 20 * i)), i) for i in range(6)]
ws = [world.World(q, s) for q, s in specs]
b = world.Batch(ws)
b.set_shape(regrow_rows_per_cta=4, lstm_ctas_per_sm=2)
b.step(100)
b.sync()
b.close()
for w in ws:
    w.close()

pc = EcoParams(H=30, W=60, capacity=400, n_agents0=100, controller=1, e0=3.0, e_max=3.0,
               e_decay=0.025, e_gain=1.0, e_repr=0.0, t_repr=30, e_death=0.0, t_death=20,
               max_age=90, res_init_p=0.2, wall_kills=1, w_init_std=0.5)
w = world.World(pc, seed=2)
w.step(120)
w.sync()
w.close()
print("CHECKED OK")
'''


def test_checked_build_finds_no_index_out_of_range():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, ECO_CHECKED="1")
    code = f"ROOT = {ROOT!r}\n" + CHILD
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "CHECKED OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
