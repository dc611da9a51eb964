"""Python view of the C ABI: worlds and batches.

PyTorch provides the device memory (one uint8 arena per world, from its
caching allocator) and the CUDA stream; every part of the simulation step
runs in libecoevo's kernels.  Functions here only marshal arguments.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import check, lib, to_c_params
from .params import EcoParams

NPARAM = 23333
HID = 32
NACT = 5

# state field -> (dtype, per-slot width or "grid")
_GRID = {"res": np.uint8, "wall": np.uint8, "slot_map": np.int32}
_SLOT = {
    "alive": (np.uint8, 1), "y": (np.int32, 1), "x": (np.int32, 1),
    "energy": (np.float32, 1), "repr_ctr": (np.int32, 1), "low_ctr": (np.int32, 1),
    "age": (np.int32, 1), "h": (np.float32, HID), "c": (np.float32, HID),
    "action": (np.int32, 1), "logits": (np.float32, NACT),
    "prev_action": (np.int32, 1), "ate": (np.uint8, 1),
}
ALL_FIELDS = tuple(_GRID) + tuple(_SLOT)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _host_weights(count: int, nparam: int) -> np.ndarray:
    """Host array for weight rows: page-locked (a numpy view of a pinned
    torch tensor, which the array keeps alive) when large, so that the
    library's permutation kernel writes it directly."""
    if count * nparam * 4 < (1 << 20):
        return np.zeros((count, nparam), np.float32)
    import torch
    return torch.empty((count, nparam), dtype=torch.float32, pin_memory=True).numpy()


def analysis_record(a) -> dict:
    """EcoAnalysis as int64 values -> dict (move_bins: int64 array of 17)."""
    a = np.asarray(a, np.int64)
    out = {k: int(a[i]) for i, k in enumerate(_lib.ANALYSIS_KEYS)}
    n = len(_lib.ANALYSIS_KEYS)
    out["move_bins"] = a[n:n + _lib.MOVE_BINS].copy()
    return out


def greediness(seen_windows, meal_windows):
    """G = C_r / T_r per agent (App. C, eco_greediness); NaN where T_r = 0."""
    T = np.ascontiguousarray(seen_windows, np.int32)
    C = np.ascontiguousarray(meal_windows, np.int32)
    assert T.shape == C.shape
    out = np.empty(T.shape, np.float64)
    check(lib().eco_greediness(_ptr(T), _ptr(C), T.size, _ptr(out)), "eco_greediness")
    return out


def life_expectancy(records) -> float | None:
    """Mean age at death over consecutive analysis windows (App. C: the
    paper pools 500 steps; eco_life_expectancy); None when nobody died."""
    rec = np.zeros((len(records), _lib.NANALYSIS), np.int64)
    n = len(_lib.ANALYSIS_KEYS)
    for i, r in enumerate(records):
        rec[i, :n] = [r[k] for k in _lib.ANALYSIS_KEYS]
        rec[i, n:] = r["move_bins"]
    out = ctypes.c_double()
    check(lib().eco_life_expectancy(_ptr(rec) if len(records) else None, len(records),
                                    ctypes.byref(out)), "eco_life_expectancy")
    return None if np.isnan(out.value) else out.value


class _Configurable:
    """Launch configuration (results do not depend on it) and its tuner."""
    _prefix = ""

    def _fn(self, name):
        return getattr(lib(), f"eco_{self._prefix}_{name}")

    def get_config(self) -> dict:
        f, sp, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(self._fn("get_config")(self._h, ctypes.byref(f), ctypes.byref(sp), ctypes.byref(k)),
              f"eco_{self._prefix}_get_config")
        return {"fused": f.value, "spawn_ctas_per_sm": sp.value, "steps_per_graph": k.value}

    def set_config(self, fused=None, spawn_ctas_per_sm=None, steps_per_graph=None) -> None:
        c = self.get_config()
        c.update({k: v for k, v in (("fused", fused), ("spawn_ctas_per_sm", spawn_ctas_per_sm),
                                     ("steps_per_graph", steps_per_graph)) if v is not None})
        check(self._fn("set_config")(self._h, int(c["fused"]), int(c["spawn_ctas_per_sm"]),
                                     int(c["steps_per_graph"])), f"eco_{self._prefix}_set_config")

    def get_shape(self) -> dict:
        rk, lc = ctypes.c_int(), ctypes.c_int()
        check(self._fn("get_shape")(self._h, ctypes.byref(rk), ctypes.byref(lc)),
              f"eco_{self._prefix}_get_shape")
        return {"regrow_rows_per_cta": rk.value, "lstm_ctas_per_sm": lc.value}

    def set_shape(self, regrow_rows_per_cta=None, lstm_ctas_per_sm=None) -> None:
        """Kernel shapes (results unchanged): regrowth tiles stacked per CTA
        (0: chosen by size, or 1, 2, 4, 8) and controller CTAs per SM (1, 2);
        None keeps a shape as it is."""
        c = self.get_shape()
        rk = c["regrow_rows_per_cta"] if regrow_rows_per_cta is None else regrow_rows_per_cta
        lc = c["lstm_ctas_per_sm"] if lstm_ctas_per_sm is None else lstm_ctas_per_sm
        check(self._fn("set_shape")(self._h, int(rk), int(lc)), f"eco_{self._prefix}_set_shape")

    def autotune(self, trial_steps: int = 16) -> dict:
        """Time real steps under each candidate configuration and keep the
        fastest; the worlds advance by the returned steps_taken."""
        r = _lib.CEcoTuneResult()
        check(self._fn("autotune")(self._h, int(trial_steps), ctypes.byref(r)),
              f"eco_{self._prefix}_autotune")
        return {k: getattr(r, k) for k, _ in r._fields_ if k != "reserved"}


class World(_Configurable):
    """One simulated world resident on a CUDA device."""
    _prefix = "world"

    def __init__(self, params: EcoParams, seed: int = 0, device=None, stream=None):
        import torch
        self.p = params
        self.seed = int(seed)
        self.nparam = _lib.NPARAM_OF[int(getattr(params, "controller", 0))]
        self._c = to_c_params(params)
        L = lib()
        nbytes = L.eco_world_bytes(ctypes.byref(self._c))
        if nbytes == 0:
            raise ValueError(f"invalid world parameters: {params}")
        self.nbytes = nbytes
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        self._h = None
        self._counter_log = None
        with torch.cuda.device(dev):
            self.stream = stream if stream is not None else torch.cuda.Stream(dev)
            self.arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
            base = (self.arena.data_ptr() + 255) & ~255
            h = ctypes.c_void_p()
            check(L.eco_world_create(ctypes.byref(self._c), self.seed, ctypes.c_void_p(base),
                                     nbytes, ctypes.c_void_p(self.stream.cuda_stream),
                                     ctypes.byref(h)), "eco_world_create")
            self._h = h

    @property
    def handle(self):
        return self._h

    def step(self, n: int = 1) -> None:
        check(lib().eco_world_step(self._h, int(n)), "eco_world_step")

    def step_forced(self, actions) -> None:
        a = np.ascontiguousarray(actions, dtype=np.int32)
        if a.shape != (self.p.capacity,):
            raise ValueError("actions must have one entry per slot")
        check(lib().eco_world_step_forced(self._h, _ptr(a), 1), "eco_world_step_forced")

    def sync(self) -> None:
        check(lib().eco_world_sync(self._h), "eco_world_sync")

    def read_state(self, fields=ALL_FIELDS, weights=None) -> dict:
        """Copy state to host numpy arrays.  weights: None, or (first, count)
        slot range of logical parameter vectors."""
        st = _lib.CEcoState()
        out = {}
        H, W, C = self.p.H, self.p.W, self.p.capacity
        for f in fields:
            if f in _GRID:
                out[f] = np.zeros((H, W), _GRID[f])
            else:
                dt, width = _SLOT[f]
                out[f] = np.zeros((C, width) if width > 1 else (C,), dt)
            setattr(st, f + "_host", out[f].ctypes.data)
        if weights is not None:
            first, count = weights
            out["weights"] = _host_weights(count, self.nparam)
            st.weights_host = out["weights"].ctypes.data
            st.weights_first, st.weights_count = int(first), int(count)
        check(lib().eco_world_read_state(self._h, ctypes.byref(st)), "eco_world_read_state")
        out["counters"] = np.array(st.counters[:], np.int64)
        return out

    def load_state(self, state: dict, set_counters: bool = True, weights_first: int = 0) -> None:
        st = _lib.CEcoState()
        keep = []
        for f in ALL_FIELDS:
            if f == "slot_map" or f not in state:
                continue
            a = np.ascontiguousarray(state[f], dtype=(_GRID[f] if f in _GRID else _SLOT[f][0]))
            keep.append(a)
            setattr(st, f + "_host", a.ctypes.data)
        if "weights" in state:
            wts = np.ascontiguousarray(state["weights"], np.float32).reshape(-1, self.nparam)
            keep.append(wts)
            st.weights_host = wts.ctypes.data
            st.weights_first, st.weights_count = int(weights_first), wts.shape[0]
        if "counters" in state:
            for i, v in enumerate(state["counters"]):
                st.counters[i] = int(v)
        check(lib().eco_world_load_state(self._h, ctypes.byref(st), 1 if set_counters else 0),
              "eco_world_load_state")

    def counters(self) -> np.ndarray:
        return self.read_state(fields=())["counters"]

    def counters_async(self, out) -> None:
        """Enqueue a copy of the counters into `out`, a page-locked int64
        torch tensor of NCOUNTERS (9) elements on the host (valid after
        sync())."""
        assert out.is_pinned() and out.numel() >= _lib.NCOUNTERS and out.element_size() == 8
        check(lib().eco_world_counters_async(self._h, ctypes.c_void_p(out.data_ptr())),
              "eco_world_counters_async")

    def counter_log(self, log) -> None:
        """Have the step kernels write every step's counters to `log`, a
        page-locked int64 torch tensor of shape (rows, NCOUNTERS): step t
        (counted from 0) fills row t % rows when it ends, with no copy added
        to the step; rows are valid after sync().  None turns the log off.
        The world keeps a reference to `log` while the log is on."""
        if log is None:
            check(lib().eco_world_counter_log(self._h, None, 0), "eco_world_counter_log")
            self._counter_log = None
            return
        import torch
        assert (log.is_pinned() and log.dtype == torch.int64 and log.dim() == 2
                and log.shape[1] == _lib.NCOUNTERS and log.is_contiguous() and log.shape[0] > 0)
        check(lib().eco_world_counter_log(self._h, ctypes.c_void_p(log.data_ptr()),
                                          int(log.shape[0])), "eco_world_counter_log")
        self._counter_log = log

    def analysis_async(self, out) -> None:
        """Enqueue the App. C metrics of the window that ends now into `out`,
        a page-locked int64 torch tensor of at least 24 elements (valid after
        sync(); decode with analysis_record).  A new window starts."""
        assert out.is_pinned() and out.numel() >= _lib.NANALYSIS and out.element_size() == 8
        check(lib().eco_world_analysis_async(self._h, ctypes.c_void_p(out.data_ptr())),
              "eco_world_analysis_async")

    def lab_window(self) -> None:
        """End a greediness window (App. C; the paper's are 20 steps)."""
        check(lib().eco_world_lab_window(self._h), "eco_world_lab_window")

    def lab_read(self):
        """(T_r, C_r) per slot: windows with a resource in view, with a meal."""
        T = np.zeros(self.p.capacity, np.int32)
        C = np.zeros(self.p.capacity, np.int32)
        check(lib().eco_world_lab_read(self._h, _ptr(T), _ptr(C)), "eco_world_lab_read")
        return T, C

    def analysis(self) -> dict:
        """Synchronous analysis_async, decoded."""
        a = np.zeros(_lib.NANALYSIS, np.int64)
        check(lib().eco_world_analysis_async(self._h, _ptr(a)), "eco_world_analysis_async")
        self.sync()
        return analysis_record(a)

    def profile(self, enable: bool, max_steps: int = 1024) -> None:
        check(lib().eco_world_profile(self._h, 1 if enable else 0, int(max_steps)),
              "eco_world_profile")

    def profile_read(self) -> dict:
        ms = (ctypes.c_double * _lib.NKERNELS)()
        n = (ctypes.c_int64 * _lib.NKERNELS)()
        check(lib().eco_world_profile_read(self._h, ms, n), "eco_world_profile_read")
        return {lib().eco_kernel_name(k).decode(): (ms[k], n[k]) for k in range(_lib.NKERNELS)}

    def close(self) -> None:
        if self._h is not None:
            lib().eco_world_destroy(self._h)
            self._h = None
            self.arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch(_Configurable):
    """Independent worlds stepped together, one launch per kernel per step."""
    _prefix = "batch"

    def __init__(self, worlds):
        self.worlds = list(worlds)
        arr = (ctypes.c_void_p * len(self.worlds))(*[w.handle.value for w in self.worlds])
        h = ctypes.c_void_p()
        check(lib().eco_batch_create(arr, len(self.worlds), ctypes.byref(h)), "eco_batch_create")
        self._h = h

    def step(self, n: int = 1) -> None:
        check(lib().eco_batch_step(self._h, int(n)), "eco_batch_step")

    def sync(self) -> None:
        check(lib().eco_batch_sync(self._h), "eco_batch_sync")

    def close(self) -> None:
        if self._h is not None:
            lib().eco_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
