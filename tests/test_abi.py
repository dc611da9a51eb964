"""CPU checks of the C ABI: the library builds, loads, exports every entry
point include/ecoevo.h declares, and validates parameters on the host."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2302_09334_gb300 import params as P
from paper_2302_09334_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def L():
    from paper_2302_09334_gb300 import build
    build.build()
    return _lib.lib()


def _declared():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(eco_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declarations_exported(L):
    declared = _declared()
    assert len(declared) >= 19
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = declared - exported
    assert not missing, missing
    for name in declared:
        assert hasattr(L, name)
    assert set(_lib.SIGNATURES) <= declared


def test_world_bytes_and_validation(L):
    def nbytes(p):
        c = _lib.to_c_params(p)
        return L.eco_world_bytes(ctypes.byref(c))

    small = nbytes(P.small_20x40())
    paper = nbytes(P.paper_200x400())
    large = nbytes(P.large_1000x2000())
    # the weight arena dominates: capacity x 23,360 floats
    assert paper > 8192 * 23360 * 4 and paper < 8192 * 23360 * 4 * 1.05
    assert large > 131072 * 23360 * 4 and small < paper < large
    bad = [P.small_20x40().replace(nbr_radius=4), P.small_20x40().replace(n_agents0=300),
           P.small_20x40().replace(class_edges=(3, 1, 5)), P.small_20x40().replace(H=0),
           P.small_20x40().replace(lat_mode=2), P.small_20x40().replace(capacity=-1)]
    for p in bad:
        assert nbytes(p) == 0, p
    c = _lib.to_c_params(P.small_20x40())
    c.abi_version = 7
    assert L.eco_world_bytes(ctypes.byref(c)) == 0


def test_strerror_and_kernel_names(L):
    assert L.eco_strerror(0) == b"ok"
    assert L.eco_strerror(_lib.ECO_ETIMEOUT) == b"device wait timed out"
    assert L.eco_kernels_per_step(None) == _lib.ECO_EINVAL
    names = [L.eco_kernel_name(k) for k in range(_lib.NKERNELS)]
    assert names[1] == b"observe_lstm" and names[8] == b"agents_fused"
    assert len(set(names)) == _lib.NKERNELS


def test_create_rejects_bad_arguments_without_gpu(L):
    # argument checks happen before any CUDA call
    h = ctypes.c_void_p()
    c = _lib.to_c_params(P.small_20x40())
    assert L.eco_world_create(ctypes.byref(c), 0, None, 0, None, ctypes.byref(h)) == _lib.ECO_EINVAL
    c.nbr_radius = 9
    assert L.eco_world_create(ctypes.byref(c), 0, None, 0, ctypes.c_void_p(1),
                              ctypes.byref(h)) == _lib.ECO_EINVAL
    c = _lib.to_c_params(P.small_20x40())
    assert L.eco_world_create(ctypes.byref(c), 0, ctypes.c_void_p(0x1001), 1 << 30,
                              ctypes.c_void_p(1), ctypes.byref(h)) == _lib.ECO_EINVAL
    assert L.eco_world_create(ctypes.byref(c), 0, ctypes.c_void_p(0x1000), 16,
                              ctypes.c_void_p(1), ctypes.byref(h)) == _lib.ECO_ENOMEM
    assert L.eco_batch_create(None, 0, ctypes.byref(h)) == _lib.ECO_EINVAL


def test_new_entry_points_validate_arguments_without_gpu(L):
    # every entry point checks its handle and pointers before any CUDA call
    null = None
    p = ctypes.c_void_p(0)
    assert L.eco_world_analysis_async(null, null) == _lib.ECO_EINVAL
    assert L.eco_world_lab_window(null) == _lib.ECO_EINVAL
    assert L.eco_world_lab_read(null, null, null) == _lib.ECO_EINVAL
    assert L.eco_world_counters_async(null, null) == _lib.ECO_EINVAL
    r = _lib.CEcoTuneResult()
    assert L.eco_batch_autotune(null, 4, ctypes.byref(r)) == _lib.ECO_EINVAL
    assert L.eco_world_autotune(null, 4, ctypes.byref(r)) == _lib.ECO_EINVAL
    assert L.eco_batch_set_config(null, 1, 4, 16) == _lib.ECO_EINVAL
    assert L.eco_world_set_config(null, 1, 4, 16) == _lib.ECO_EINVAL
    f = ctypes.c_int()
    assert L.eco_world_get_config(null, ctypes.byref(f), ctypes.byref(f),
                                  ctypes.byref(f)) == _lib.ECO_EINVAL
    assert L.eco_strerror(_lib.ECO_EBOUNDS) == b"device index out of range"
    # the paper controller's parameters are accepted, an unknown controller is not
    c = _lib.to_c_params(P.paper_natural())
    assert L.eco_world_bytes(ctypes.byref(c)) > 0
    c.controller = 2
    assert L.eco_world_bytes(ctypes.byref(c)) == 0
    # the paper controller's arena is an order of magnitude smaller (9.8 KB rows)
    lstm = _lib.to_c_params(P.paper_natural().replace(controller=0))
    paper = _lib.to_c_params(P.paper_natural())
    assert L.eco_world_bytes(ctypes.byref(lstm)) > 5 * L.eco_world_bytes(ctypes.byref(paper))
    assert p.value is None


def test_greediness_and_life_expectancy_host_functions():
    """The App. C ratios computed by the library's host functions (no GPU):
    G = C_r / T_r with NaN where T_r = 0; life expectancy pooled over
    analysis records, None when nobody died."""
    import numpy as np
    from paper_2302_09334_gb300.world import greediness, life_expectancy
    g = greediness([0, 2, 4, 5], [0, 1, 4, 0])
    assert np.isnan(g[0]) and g[1] == 0.5 and g[2] == 1.0 and g[3] == 0.0
    rec = lambda d, s: {"t": 0, "window": 50, "population": 0, "resources": 0, "deaths": d,
                        "death_age_sum": s, "movers": 0, "move_bins": np.zeros(17, np.int64)}
    assert life_expectancy([rec(2, 100), rec(0, 0), rec(3, 50)]) == 30.0
    assert life_expectancy([rec(0, 0)]) is None and life_expectancy([]) is None
    from paper_2302_09334_gb300._lib import ECO_EINVAL, lib
    assert lib().eco_greediness(None, None, -1, None) == ECO_EINVAL
    assert lib().eco_life_expectancy(None, 1, None) == ECO_EINVAL
