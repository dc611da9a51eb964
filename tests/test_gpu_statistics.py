"""Free-running GPU worlds against free-running oracle worlds, statistically.

Without forced actions the two drift apart wherever an argmax margin is
below the FP32/FP64 difference, so they are compared as ensembles over eight
seeds: population and resource mass at every 50th step, and the latitude
profile of the resources (five bands of rows) at the end, each within four
standard errors of the difference of the two ensemble means (plus one unit
for counts that can be equal in every run)."""
import numpy as np
import pytest

from paper_2302_09334_gb300.params import EcoParams

pytestmark = pytest.mark.gpu

P = EcoParams(H=40, W=80, capacity=1024, n_agents0=150)
SEEDS = range(8)
STEPS = 300
EVERY = 50
BANDS = 5


@pytest.fixture(scope="module")
def eco():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2302_09334_gb300 import build, world
    build.build()
    return world


def _bands(res):
    rows = res.reshape(BANDS, -1, res.shape[1]).sum(axis=(1, 2)).astype(np.float64)
    return rows / max(rows.sum(), 1.0)


def _run_gpu(eco, seed):
    w = eco.World(P, seed=seed)
    pops, ress = [], []
    for _ in range(STEPS // EVERY):
        w.step(EVERY)
        a = w.analysis()
        pops.append(a["population"])
        ress.append(a["resources"])
    res = w.read_state(fields=("res",))["res"]
    w.close()
    return np.array(pops), np.array(ress), _bands(res)


def _run_oracle(oracle, seed):
    ow = oracle.OracleWorld(P.asdict(), seed)
    pops, ress = [], []
    for k in range(STEPS):
        ow.step()
        if (k + 1) % EVERY == 0:
            pops.append(ow.population)
            ress.append(int(ow.res.sum()))
    bands = _bands(ow.res)
    ow.close()
    return np.array(pops), np.array(ress), bands


def _close(g, o, what):
    g, o = np.asarray(g, np.float64), np.asarray(o, np.float64)
    se = np.sqrt(g.var(axis=0, ddof=1) / len(g) + o.var(axis=0, ddof=1) / len(o))
    diff = np.abs(g.mean(axis=0) - o.mean(axis=0))
    assert np.all(diff <= 4 * se + 1.0), f"{what}: {diff} vs {4 * se + 1.0}"


def test_free_run_ensembles_agree(eco, oracle):
    gpu = [_run_gpu(eco, s) for s in SEEDS]
    ora = [_run_oracle(oracle, s) for s in SEEDS]
    _close([r[0] for r in gpu], [r[0] for r in ora], "population")
    _close([r[1] for r in gpu], [r[1] for r in ora], "resources")
    gb = np.array([r[2] for r in gpu])
    ob = np.array([r[2] for r in ora])
    se = np.sqrt(gb.var(axis=0, ddof=1) / len(gb) + ob.var(axis=0, ddof=1) / len(ob))
    assert np.all(np.abs(gb.mean(0) - ob.mean(0)) <= 4 * se + 0.01), (gb.mean(0), ob.mean(0))
    # the climate rises toward the bottom rows: so do the resources
    assert gb.mean(0)[-1] > gb.mean(0)[0] and ob.mean(0)[-1] > ob.mean(0)[0]
    # most seeds follow the oracle exactly for the first window
    same = sum(int(g[0][0] == o[0][0]) for g, o in zip(gpu, ora))
    assert same >= len(SEEDS) // 2
