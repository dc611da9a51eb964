"""ctypes view of the CPU oracle (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this module.  It shares nothing with the CUDA library: parameters come in as
a plain mapping of field names to numbers.
"""
import ctypes
import os

import numpy as np

from . import build as _build

NOBS, HID, NACT = 148, 32, 5
NPARAM = 23333
OFF_B, OFF_WO, OFF_BO = 23040, 23168, 23328
TAG_REGROW, TAG_PLACE, TAG_RES_INIT, TAG_INIT_W, TAG_MUT, TAG_ACT = 1, 2, 3, 4, 5, 6
CTRL_LSTM32, CTRL_PAPER = 0, 1
PC_VIEW, PC_NOBS, PC_HID, PC_EMB, PC_NPARAM = 15, 675, 4, 78, 2445
# logical parameter offsets of the paper controller (see the oracle header)
PC_OFF = {"W1": 0, "B1": 108, "W2": 112, "B2": 400, "WI": 408, "WH": 1656, "BL": 1720,
          "D1": 1736, "DB1": 2392, "D2": 2400, "DB2": 2440}

(F_RES, F_WALL, F_SLOT_MAP, F_ALIVE, F_Y, F_X, F_ENERGY, F_REPR_CTR, F_LOW_CTR,
 F_AGE, F_H, F_C, F_ACTION, F_LOGITS, F_ATE, F_WEIGHTS, F_COUNTERS, F_THR,
 F_BIRTH_PARENT, F_BIRTH_CHILD, F_MOVE_ACTION, F_PREV_ACTION, F_LAB_FLAGS, F_LAB_T,
 F_LAB_C, F_MAG_H, F_MAG_C, F_MAG_LOGITS) = range(28)
(C_T, C_POP, C_BIRTHS, C_DEATHS, C_DROPPED, C_BIRTHS_LAST, C_DEATHS_LAST,
 C_DROPPED_LAST, C_AGENT_STEPS) = range(9)
NCOUNTERS = 9


class OrParams(ctypes.Structure):
    _fields_ = [
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


def make_params(values) -> OrParams:
    """Fill OrParams from a mapping (or an object with attributes)."""
    get = values.get if hasattr(values, "get") else (lambda k: getattr(values, k))
    p = OrParams()
    for name, ctype in OrParams._fields_:
        v = get(name)
        if v is None and name == "controller":
            v = 0
        if name == "class_edges":
            p.class_edges = (ctypes.c_int32 * 3)(*[int(e) for e in v])
        elif name == "p_class":
            p.p_class = (ctypes.c_double * 4)(*[float(e) for e in v])
        elif ctype in (ctypes.c_float, ctypes.c_double):
            setattr(p, name, float(v))
        else:
            setattr(p, name, int(v))
    return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double)]
        L.or_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                ctypes.c_uint32, ctypes.c_uint32]
        L.or_normal.restype = ctypes.c_double
        L.or_fill_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_float, ctypes.c_void_p,
                                      ctypes.c_void_p]
        L.or_threshold_table.argtypes = [ctypes.POINTER(OrParams), u32p]
        L.or_regrow.argtypes = [ctypes.POINTER(OrParams), ctypes.c_uint64,
                                ctypes.c_uint32, u32p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p]
        L.or_observe.argtypes = [ctypes.POINTER(OrParams), ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                 ctypes.c_int32, ctypes.c_float, ctypes.c_void_p]
        L.or_lstm_step.argtypes = [ctypes.c_void_p] * 5
        L.or_lstm_step.restype = ctypes.c_int
        L.or_initial_layout.argtypes = [ctypes.POINTER(OrParams), ctypes.c_uint64,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.or_world_create.argtypes = [ctypes.POINTER(OrParams), ctypes.c_uint64,
                                      ctypes.POINTER(ctypes.c_void_p)]
        L.or_world_destroy.argtypes = [ctypes.c_void_p]
        L.or_world_step.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.or_world_field.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_world_field.restype = ctypes.c_void_p
        L.or_world_sync.argtypes = [ctypes.c_void_p]
        L.or_world_analysis.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.or_world_lab_window.argtypes = [ctypes.c_void_p]
        L.or_world_set_order.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        L.or_world_set_order.restype = ctypes.c_int
        L.or_fill_normals_n.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_float, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int]
        L.or_param_count.argtypes = [ctypes.c_int]
        L.or_param_count.restype = ctypes.c_int
        L.or_pc_observe.argtypes = [ctypes.POINTER(OrParams), ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_void_p]
        L.or_pc_forward.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.or_action_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
        L.or_action_uniform.restype = ctypes.c_double
        L.or_pc_sample.argtypes = [ctypes.c_void_p, ctypes.c_double]
        L.or_pc_sample.restype = ctypes.c_int
        L.or_lstm_mag.argtypes = [ctypes.c_void_p] * 9
        L.or_world_track_magnitudes.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_pc_mag.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int] + \
            [ctypes.c_void_p] * 7
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return list(o)


def box_muller(x1, x2):
    z0, z1 = ctypes.c_double(), ctypes.c_double()
    lib().or_box_muller(x1, x2, ctypes.byref(z0), ctypes.byref(z1))
    return z0.value, z1.value


def normal(seed, tag, t, ident, j):
    return lib().or_normal(seed, tag, t, ident, j)


def fill_normals(seed, tag, t, ident, scale, base=None) -> np.ndarray:
    """base + scale * N(0,1) over one parameter vector (float32)."""
    out = np.zeros(NPARAM, np.float32)
    b = None if base is None else np.ascontiguousarray(base, np.float32)
    lib().or_fill_normals(seed, tag, t, ident, scale, None if b is None else _ptr(b), _ptr(out))
    return out


def threshold_table(params) -> np.ndarray:
    p = make_params(params)
    thr = np.zeros((p.H, 4), np.uint32)
    lib().or_threshold_table(ctypes.byref(p),
                             thr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return thr


def regrow(params, seed, t, res_old, wall, thr=None) -> np.ndarray:
    p = make_params(params)
    if thr is None:
        thr = threshold_table(params)
    thr = np.ascontiguousarray(thr, np.uint32)
    res_old = np.ascontiguousarray(res_old, np.uint8)
    wall = np.ascontiguousarray(wall, np.uint8)
    out = np.zeros_like(res_old)
    lib().or_regrow(ctypes.byref(p), seed, t,
                    thr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                    _ptr(res_old), _ptr(wall), _ptr(out))
    return out


def observe(params, res, wall, slot_map, y, x, energy) -> np.ndarray:
    p = make_params(params)
    res = np.ascontiguousarray(res, np.uint8)
    wall = np.ascontiguousarray(wall, np.uint8)
    slot_map = np.ascontiguousarray(slot_map, np.int32)
    out = np.zeros(NOBS, np.float64)
    lib().or_observe(ctypes.byref(p), _ptr(res), _ptr(wall), _ptr(slot_map),
                     int(y), int(x), float(energy), _ptr(out))
    return out


def lstm_step(w, obs, h, c):
    """Returns (action, h', c', logits) without touching the inputs."""
    w = np.ascontiguousarray(w, np.float32)
    obs = np.ascontiguousarray(obs, np.float64)
    h2 = np.array(h, np.float64)
    c2 = np.array(c, np.float64)
    logits = np.zeros(NACT, np.float64)
    a = lib().or_lstm_step(_ptr(w), _ptr(obs), _ptr(h2), _ptr(c2), _ptr(logits))
    return a, h2, c2, logits


def lstm_mag(w, obs, h, c, eh=None, ec=None):
    """Error magnitudes (E_h', E_c', E_logits) of one LSTM step (test
    support, or_lstm_mag); eh, ec: magnitudes of the inputs (default 0)."""
    w = np.ascontiguousarray(w, np.float32)
    obs = np.ascontiguousarray(obs, np.float64)
    h = np.ascontiguousarray(h, np.float64)
    c = np.ascontiguousarray(c, np.float64)
    eh = np.zeros(HID) if eh is None else np.ascontiguousarray(eh, np.float64)
    ec = np.zeros(HID) if ec is None else np.ascontiguousarray(ec, np.float64)
    oh, oc, ol = np.zeros(HID), np.zeros(HID), np.zeros(NACT)
    lib().or_lstm_mag(_ptr(w), _ptr(obs), _ptr(h), _ptr(c), _ptr(eh), _ptr(ec), _ptr(oh),
                      _ptr(oc), _ptr(ol))
    return oh, oc, ol


def pc_mag(w, obs, prev_action, ate, h, c, eh=None, ec=None):
    """Error magnitudes (E_h', E_c', E_logits) of one paper-controller step
    (test support, or_pc_mag)."""
    w = np.ascontiguousarray(np.asarray(w, np.float32)[:PC_NPARAM])
    obs = np.ascontiguousarray(obs, np.float64).reshape(-1)
    h = np.ascontiguousarray(np.asarray(h, np.float64)[:PC_HID])
    c = np.ascontiguousarray(np.asarray(c, np.float64)[:PC_HID])
    eh = np.zeros(PC_HID) if eh is None else np.ascontiguousarray(eh, np.float64)[:PC_HID]
    ec = np.zeros(PC_HID) if ec is None else np.ascontiguousarray(ec, np.float64)[:PC_HID]
    oh, oc, ol = np.zeros(PC_HID), np.zeros(PC_HID), np.zeros(NACT)
    lib().or_pc_mag(_ptr(w), _ptr(obs), int(prev_action), int(ate), _ptr(h), _ptr(c),
                    _ptr(np.ascontiguousarray(eh)), _ptr(np.ascontiguousarray(ec)), _ptr(oh),
                    _ptr(oc), _ptr(ol))
    return oh, oc, ol


def param_count(controller: int) -> int:
    return int(lib().or_param_count(int(controller)))


def fill_normals_n(seed, tag, t, ident, scale, n, base=None) -> np.ndarray:
    """The first n values of fill_normals."""
    out = np.zeros(n, np.float32)
    b = None if base is None else np.ascontiguousarray(base, np.float32)
    lib().or_fill_normals_n(int(seed), tag, t, ident, float(scale),
                            None if b is None else _ptr(b), _ptr(out), int(n))
    return out


def pc_observe(params, res, wall, slot_map, y, x) -> np.ndarray:
    """The paper controller's 15x15x3 view, shape (15, 15, 3)."""
    p = make_params(params)
    res = np.ascontiguousarray(res, np.uint8)
    wall = np.ascontiguousarray(wall, np.uint8)
    slot_map = np.ascontiguousarray(slot_map, np.int32)
    out = np.zeros(PC_NOBS, np.float64)
    lib().or_pc_observe(ctypes.byref(p), _ptr(res), _ptr(wall), _ptr(slot_map),
                        int(y), int(x), _ptr(out))
    return out.reshape(PC_VIEW, PC_VIEW, 3)


def pc_forward(w, obs, prev_action, ate, h, c):
    """Returns (h', c', logits) of the paper controller (inputs untouched)."""
    w = np.ascontiguousarray(np.asarray(w, np.float32)[:PC_NPARAM])
    obs = np.ascontiguousarray(obs, np.float64).reshape(-1)
    h2 = np.array(h, np.float64)[:PC_HID].copy()
    c2 = np.array(c, np.float64)[:PC_HID].copy()
    logits = np.zeros(NACT, np.float64)
    lib().or_pc_forward(_ptr(w), _ptr(obs), int(prev_action), int(ate), _ptr(h2), _ptr(c2),
                        _ptr(logits))
    return h2, c2, logits


def action_uniform(seed, t, slot) -> float:
    return float(lib().or_action_uniform(int(seed), int(t), int(slot)))


def pc_sample(logits, u) -> int:
    lg = np.ascontiguousarray(logits, np.float64)
    return int(lib().or_pc_sample(_ptr(lg), float(u)))


def initial_layout(params, seed):
    """(res [H,W] u8, wall [H,W] u8, cells [n_agents0] int32) of a new world."""
    p = make_params(params)
    res = np.zeros((p.H, p.W), np.uint8)
    wall = np.zeros((p.H, p.W), np.uint8)
    cells = np.zeros(max(p.n_agents0, 1), np.int32)
    rc = lib().or_initial_layout(ctypes.byref(p), int(seed), _ptr(res), _ptr(wall), _ptr(cells))
    if rc != 0:
        raise ValueError(f"or_initial_layout failed ({rc})")
    return res, wall, cells[:p.n_agents0]


MOVE_BINS = 17
NANALYSIS = 7 + MOVE_BINS
ANALYSIS_KEYS = ("t", "window", "population", "resources", "deaths", "death_age_sum", "movers")


def analysis_record(a) -> dict:
    out = {k: int(a[i]) for i, k in enumerate(ANALYSIS_KEYS)}
    out["move_bins"] = np.asarray(a[len(ANALYSIS_KEYS):len(ANALYSIS_KEYS) + MOVE_BINS],
                                  np.int64).copy()
    return out


class OracleWorld:
    """One oracle world; the fields are numpy views into the C arrays."""

    def __init__(self, params, seed: int, magnitudes: bool = True):
        self.p = make_params(params)
        self.seed = int(seed)
        h = ctypes.c_void_p()
        rc = lib().or_world_create(ctypes.byref(self.p), self.seed, ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"or_world_create failed ({rc})")
        self._h = h
        if not magnitudes:   # test support only; the step itself is the same
            lib().or_world_track_magnitudes(h, 0)
        H, W, C = self.p.H, self.p.W, max(self.p.capacity, 1)
        f = self._field
        self.res = f(F_RES, np.uint8, (H, W))
        self.wall = f(F_WALL, np.uint8, (H, W))
        self.slot_map = f(F_SLOT_MAP, np.int32, (H, W))
        self.alive = f(F_ALIVE, np.uint8, (C,))
        self.y = f(F_Y, np.int32, (C,))
        self.x = f(F_X, np.int32, (C,))
        self.energy = f(F_ENERGY, np.float32, (C,))
        self.repr_ctr = f(F_REPR_CTR, np.int32, (C,))
        self.low_ctr = f(F_LOW_CTR, np.int32, (C,))
        self.age = f(F_AGE, np.int32, (C,))
        self.h = f(F_H, np.float64, (C, HID))
        self.c = f(F_C, np.float64, (C, HID))
        self.action = f(F_ACTION, np.int32, (C,))
        self.logits = f(F_LOGITS, np.float64, (C, NACT))
        self.ate = f(F_ATE, np.uint8, (C,))
        self.weights = f(F_WEIGHTS, np.float32, (C, NPARAM))
        self.counters = f(F_COUNTERS, np.int64, (NCOUNTERS,))
        self.thr = f(F_THR, np.uint32, (H, 4))
        self.birth_parent = f(F_BIRTH_PARENT, np.int32, (C,))
        self.birth_child = f(F_BIRTH_CHILD, np.int32, (C,))
        self.move_action = f(F_MOVE_ACTION, np.int32, (C,))
        self.prev_action = f(F_PREV_ACTION, np.int32, (C,))
        self.lab_flags = f(F_LAB_FLAGS, np.uint8, (C,))
        self.lab_t = f(F_LAB_T, np.int32, (C,))
        self.lab_c = f(F_LAB_C, np.int32, (C,))
        # test support: error magnitudes of h, c and the logits of the last
        # step (or_lstm_mag / or_pc_mag; 0 for state written from outside)
        self.mag_h = f(F_MAG_H, np.float64, (C, HID))
        self.mag_c = f(F_MAG_C, np.float64, (C, HID))
        self.mag_logits = f(F_MAG_LOGITS, np.float64, (C, NACT))

    def _field(self, fid, dtype, shape):
        addr = lib().or_world_field(self._h, fid)
        n = int(np.prod(shape))
        buf = (ctypes.c_char * (n * np.dtype(dtype).itemsize)).from_address(addr)
        return np.frombuffer(buf, dtype=dtype, count=n).reshape(shape)

    @property
    def t(self):
        return int(self.counters[C_T])

    @property
    def population(self):
        return int(self.counters[C_POP])

    def step(self, forced=None):
        if forced is None:
            rc = lib().or_world_step(self._h, None)
        else:
            fa = np.ascontiguousarray(forced, np.int32)
            assert fa.shape[0] >= self.p.capacity
            rc = lib().or_world_step(self._h, _ptr(fa))
        if rc != 0:
            raise RuntimeError(f"or_world_step failed ({rc})")

    def sync(self):
        """Rebuild slot_map/thresholds after fields were written directly
        (and start a new analysis window with fresh agent identities)."""
        if lib().or_world_sync(self._h) != 0:
            raise ValueError("inconsistent agent placement")

    def lab_window(self) -> None:
        """End a greediness window (or_world_lab_window)."""
        lib().or_world_lab_window(self._h)

    def set_order(self, perm) -> None:
        """Test hook (or_world_set_order): visit the slots in the order
        `perm` in the loops whose result must not depend on it; None
        restores ascending order."""
        if perm is None:
            rc = lib().or_world_set_order(self._h, None)
        else:
            a = np.ascontiguousarray(perm, dtype=np.int32)
            rc = lib().or_world_set_order(self._h, a.ctypes.data)
        if rc != 0:
            raise ValueError(f"or_world_set_order failed ({rc})")

    def analysis(self) -> dict:
        """App. C metrics of the window that ends now (or_world_analysis);
        a new window starts."""
        out = np.zeros(NANALYSIS, np.int64)
        lib().or_world_analysis(self._h, _ptr(out))
        return analysis_record(out)

    def close(self):
        if self._h:
            lib().or_world_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
