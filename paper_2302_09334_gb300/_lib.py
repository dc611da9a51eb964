"""ctypes declarations of the C ABI in include/ecoevo.h (marshalling only).

Loading fails loudly when libecoevo.so has not been built: there is no
fallback implementation of any part of the step.
"""
from __future__ import annotations

import ctypes
import os

from .params import EcoParams

ECO_ABI_V2 = 0x45434F02
CTRL_LSTM32, CTRL_PAPER = 0, 1
NPARAM_OF = {CTRL_LSTM32: 23333, CTRL_PAPER: 2445}
ECO_OK, ECO_EINVAL, ECO_ENOMEM, ECO_ECUDA, ECO_ETIMEOUT, ECO_ESTATE, ECO_EBOUNDS = \
    0, -1, -2, -3, -4, -5, -6
NCOUNTERS = 9
NKERNELS = 10
MOVE_BINS = 17
# EcoAnalysis: these int64 fields, then MOVE_BINS bin counts
ANALYSIS_KEYS = ("t", "window", "population", "resources", "deaths", "death_age_sum", "movers")
NANALYSIS = len(ANALYSIS_KEYS) + MOVE_BINS
(C_T, C_POP, C_BIRTHS, C_DEATHS, C_DROPPED, C_BIRTHS_LAST, C_DEATHS_LAST,
 C_DROPPED_LAST, C_AGENT_STEPS) = range(9)

# ECO_CHECKED=1 in the environment selects the range-checked build
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib",
                        "libecoevo_checked.so" if os.environ.get("ECO_CHECKED") == "1"
                        else "libecoevo.so")


class CEcoParams(ctypes.Structure):
    _fields_ = [
        ("abi_version", ctypes.c_uint32),
        ("H", ctypes.c_int32), ("W", ctypes.c_int32),
        ("capacity", ctypes.c_int32), ("n_agents0", ctypes.c_int32),
        ("border_walls", ctypes.c_int32),
        ("res_init_p", ctypes.c_double),
        ("nbr_shape", ctypes.c_int32), ("nbr_radius", ctypes.c_int32),
        ("class_edges", ctypes.c_int32 * 3),
        ("p_class", ctypes.c_double * 4),
        ("lat_mode", ctypes.c_int32),
        ("lat_top", ctypes.c_double), ("lat_bottom", ctypes.c_double),
        ("lat_alpha", ctypes.c_double),
        ("p_spont", ctypes.c_double),
        ("e0", ctypes.c_float), ("e_decay", ctypes.c_float),
        ("e_gain", ctypes.c_float), ("e_max", ctypes.c_float),
        ("e_repr", ctypes.c_float), ("t_repr", ctypes.c_int32),
        ("e_death", ctypes.c_float), ("t_death", ctypes.c_int32),
        ("max_age", ctypes.c_int32),
        ("wall_kills", ctypes.c_int32),
        ("w_init_std", ctypes.c_float), ("mut_std", ctypes.c_float),
        ("controller", ctypes.c_int32),
    ]


def to_c_params(p: EcoParams) -> CEcoParams:
    c = CEcoParams()
    c.abi_version = ECO_ABI_V2
    for name, ctype in CEcoParams._fields_[1:]:
        v = getattr(p, name)
        if name == "class_edges":
            c.class_edges = (ctypes.c_int32 * 3)(*[int(e) for e in v])
        elif name == "p_class":
            c.p_class = (ctypes.c_double * 4)(*[float(e) for e in v])
        elif ctype in (ctypes.c_float, ctypes.c_double):
            setattr(c, name, float(v))
        else:
            setattr(c, name, int(v))
    return c


_P = ctypes.c_void_p


class CEcoState(ctypes.Structure):
    _fields_ = [
        ("counters", ctypes.c_int64 * NCOUNTERS),
        ("res_host", _P), ("wall_host", _P), ("slot_map_host", _P),
        ("alive_host", _P), ("y_host", _P), ("x_host", _P), ("energy_host", _P),
        ("repr_ctr_host", _P), ("low_ctr_host", _P), ("age_host", _P),
        ("h_host", _P), ("c_host", _P), ("action_host", _P), ("logits_host", _P),
        ("weights_host", _P),
        ("weights_first", ctypes.c_int32), ("weights_count", ctypes.c_int32),
        ("prev_action_host", _P), ("ate_host", _P),
    ]


# name -> (restype, argtypes)
class CEcoTuneResult(ctypes.Structure):
    _fields_ = [("fused", ctypes.c_int32), ("spawn_ctas_per_sm", ctypes.c_int32),
                ("steps_per_graph", ctypes.c_int32), ("regrow_rows_per_cta", ctypes.c_int32),
                ("lstm_ctas_per_sm", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("steps_taken", ctypes.c_int64), ("ms_per_step_initial", ctypes.c_double),
                ("ms_per_step_best", ctypes.c_double)]


_I = ctypes.POINTER(ctypes.c_int)

SIGNATURES = {
    "eco_world_bytes": (ctypes.c_size_t, [ctypes.POINTER(CEcoParams)]),
    "eco_world_create": (ctypes.c_int, [ctypes.POINTER(CEcoParams), ctypes.c_uint64, _P,
                                        ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "eco_world_destroy": (None, [_P]),
    "eco_world_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "eco_world_step_forced": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "eco_world_read_state": (ctypes.c_int, [_P, ctypes.POINTER(CEcoState)]),
    "eco_world_load_state": (ctypes.c_int, [_P, ctypes.POINTER(CEcoState), ctypes.c_int]),
    "eco_world_sync": (ctypes.c_int, [_P]),
    "eco_world_counters_async": (ctypes.c_int, [_P, _P]),
    "eco_world_counter_log": (ctypes.c_int, [_P, _P, ctypes.c_int64]),
    "eco_world_analysis_async": (ctypes.c_int, [_P, _P]),
    "eco_world_lab_window": (ctypes.c_int, [_P]),
    "eco_world_lab_read": (ctypes.c_int, [_P, _P, _P]),
    "eco_world_selftest_timeout": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "eco_world_clear_status": (ctypes.c_int, [_P]),
    "eco_world_params": (_P, [_P]),
    "eco_world_stream": (_P, [_P]),
    "eco_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P)]),
    "eco_batch_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "eco_batch_sync": (ctypes.c_int, [_P]),
    "eco_batch_destroy": (None, [_P]),
    "eco_batch_set_config": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "eco_batch_get_config": (ctypes.c_int, [_P, _I, _I, _I]),
    "eco_batch_set_shape": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "eco_batch_get_shape": (ctypes.c_int, [_P, _I, _I]),
    "eco_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(CEcoTuneResult)]),
    "eco_world_set_config": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "eco_world_get_config": (ctypes.c_int, [_P, _I, _I, _I]),
    "eco_world_set_shape": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "eco_world_get_shape": (ctypes.c_int, [_P, _I, _I]),
    "eco_world_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(CEcoTuneResult)]),
    "eco_world_profile": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "eco_world_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_int64)]),
    "eco_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
    "eco_kernels_per_step": (ctypes.c_int, [_P]),
    "eco_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "eco_life_expectancy": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]),
    "eco_greediness": (ctypes.c_int, [_P, _P, ctypes.c_int64, _P]),
    "eco_moves_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P, _P]),
}

_lib = None


class EcoError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().eco_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})")


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"libecoevo.so is not built ({LIB_PATH}); run "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code: int, where: str) -> None:
    if code != ECO_OK:
        raise EcoError(code, where)
