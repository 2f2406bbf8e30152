"""ctypes binding of libdash_gb300.so (include/dash.h): argument marshalling
only.  Every step of an update runs in the library's CUDA kernels; there is
no Python or CPU fallback, and loading fails loudly when the library is
missing."""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdash_gb300.so")

DASH_MODE_P, DASH_MODE_Q = 0, 1
PREC = {"fp64": 0, "fp32": 1, "f16x3": 2}
DTYPE = {"f64": 0, "f32": 1}
HOST, DEVICE = 0, 1

STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory or capacity", 3: "CUDA error",
          4: "invalid state", 5: "non-finite result", 6: "device wait timed out"}


class DashError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [("J", C.c_int32), ("R", C.c_int32), ("lambda_", C.c_double),
                ("mode", C.c_int32), ("precision", C.c_int32), ("input_dtype", C.c_int32),
                ("n_sweeps", C.c_int32), ("pinv_rtol", C.c_double),
                ("max_slices", C.c_int64), ("max_rows", C.c_int64),
                ("max_segments", C.c_int64), ("stream", C.c_void_p),
                ("max_staged_rows", C.c_int64)]


_lib = None

# (name, restype, argtypes): every entry point declared in include/dash.h
P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
PD = C.POINTER(C.c_double)
PI64 = C.POINTER(C.c_int64)
SIGNATURES = [
    ("dash_config_default", None, [C.POINTER(Config), I32, I32, D]),
    ("dash_init", C.c_int, [C.POINTER(Config), C.POINTER(P)]),
    ("dash_destroy", None, [P]),
    ("dash_last_error", C.c_char_p, [P]),
    ("dash_status_string", C.c_char_p, [C.c_int]),
    ("dash_set_factors", C.c_int, [P, PD, PD]),
    ("dash_set_state_p", C.c_int, [P, I64, PD, PD, PD, PD, PD, PD]),
    ("dash_get_state_p", C.c_int, [P, PD, PD, PD, PD, PD, PD]),
    ("dash_set_state_q", C.c_int, [P, I64, PD, PD, PD, PD, PD]),
    ("dash_get_state_q", C.c_int, [P, PD, PD, PD, PD, PD]),
    ("dash_num_slices", I64, [P]),
    ("dash_append_rows", C.c_int, [P, I64, P, I64, I64, I32]),
    ("dash_append_slices", C.c_int, [P, I64, PI64, C.POINTER(P), PI64, I32, PI64]),
    ("dash_append_batch", C.c_int, [P, I64, PI64, PI64, P, I32]),
    ("dash_update", C.c_int, [P]),
    ("dash_update_device", C.c_int, [P, I64, PI64, PI64, P]),
    ("dash_fit_initial", C.c_int, [P, I32]),
    ("dash_fit_initial_device", C.c_int, [P, I64, PI64, PI64, P, I32]),
    ("dash_factors", C.c_int, [P, PD, PD, I64, I64, PD]),
    ("dash_new_rows", C.c_int, [P, PD, PI64]),
    ("dash_fitness", C.c_int, [P, PD, PD]),
    ("dash_sync", C.c_int, [P]),
    ("dash_config_bytes", C.c_int, [C.POINTER(Config), PI64, PI64]),
    ("dash_device_bytes", I64, [P]),
    ("dash_query", C.c_int, [P, C.POINTER(C.c_int32)]),
    ("dash_last_update_ms", C.c_int, [P, C.POINTER(C.c_float)]),
    ("dash_launch_count", I64, [P]),
    ("dash_profile_enable", C.c_int, [P, I32]),
    ("dash_profile_kinds", I32, []),
    ("dash_profile_get", C.c_int, [P, I32, C.POINTER(C.c_char_p), PI64, PD]),
    ("dash_last_plan", C.c_int, [P, PI64, PI64, PI64, PI64, PI64]),
    ("dash_set_row_path", C.c_int, [P, I32]),
    ("dash_rows_error", C.c_int, [P, I64, PI64, PI64, P, P, PD, PD, PD]),
    ("dash_local_errors", C.c_int, [P, PD, PD, PD, I64]),
    ("dash_f_increment_noalloc", C.c_int, [P, P, I64, I32, I32, P, P, I64, P, P, P]),
    ("dash_counters", C.c_int, [P, PI64, PI64]),
    ("dash_fitness_lambda", C.c_int, [P, PD, PD]),
    ("dash_set_weighted_norm", C.c_int, [P, D]),
    ("dash_save", C.c_int, [P, C.c_char_p]),
    ("dash_load", C.c_int, [C.c_char_p, P, C.POINTER(P)]),
    ("dash_set_graph", C.c_int, [P, I32]),
    ("dash_measure_fp64_fma", C.c_int, [PD]),
    ("dash_set_wait_limit", C.c_int, [P, I64]),
    ("dash_inject_wait_fault", C.c_int, [P]),
    ("dash_graph_stats", C.c_int, [P, PI64, PI64]),
    ("dash_set_autotune", C.c_int, [P, I32]),
    ("dash_autotune_result", C.c_int, [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int32), C.POINTER(C.c_float)]),
]


def load(path: str = LIB_PATH):
    """Load the library (once).  Raises if it is missing: there is no
    fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -m paper_2305_18376_gb300.build` (needs nvcc)")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _pd(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(PD)


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64))


def _config(lib, J: int, R: int, lam: float, mode: str = "P", precision: str = "fp32",
            input_dtype: str = "f32", max_slices: int = 1 << 16, max_rows: int = 1 << 20,
            max_segments: int = 1 << 17, pinv_rtol: float = 0.0, stream=None,
            max_staged_rows: int = 0, n_sweeps: int = 1) -> Config:
    cfg = Config()
    lib.dash_config_default(C.byref(cfg), J, R, lam)
    cfg.n_sweeps = n_sweeps
    cfg.mode = DASH_MODE_P if mode == "P" else DASH_MODE_Q
    cfg.precision = PREC[precision]
    cfg.input_dtype = DTYPE[input_dtype]
    cfg.max_slices, cfg.max_rows, cfg.max_segments = max_slices, max_rows, max_segments
    cfg.pinv_rtol = pinv_rtol
    cfg.stream = stream
    cfg.max_staged_rows = max_staged_rows
    return cfg


def measure_fp64_fma() -> float:
    """FP64 FMAs per second of the current device (dash_measure_fp64_fma)."""
    lib = load()
    v = C.c_double()
    st = lib.dash_measure_fp64_fma(C.byref(v))
    if st != 0:
        raise DashError(st, "dash_measure_fp64_fma failed")
    return v.value


def config_bytes(J: int, R: int, lam: float, **kw) -> tuple:
    """(device bytes, pinned host bytes) that a DashModel with these
    arguments allocates, computed without allocating (dash_config_bytes)."""
    lib = load()
    cfg = _config(lib, J, R, lam, **kw)
    dev, host = C.c_int64(), C.c_int64()
    st = lib.dash_config_bytes(C.byref(cfg), C.byref(dev), C.byref(host))
    if st != 0:
        raise DashError(st, "dash_config_bytes rejected the configuration")
    return dev.value, host.value


class DashModel:
    """One streaming PARAFAC2 model behind the C ABI (dash_init ...)."""

    def __init__(self, J: int, R: int, lam: float, mode: str = "P", precision: str = "fp32",
                 input_dtype: str = "f32", max_slices: int = 1 << 16, max_rows: int = 1 << 20,
                 max_segments: int = 1 << 17, pinv_rtol: float = 0.0, stream=None,
                 max_staged_rows: int = 0, n_sweeps: int = 1, _handle=None):
        lib = load()
        if _handle is None:
            cfg = _config(lib, J, R, lam, mode, precision, input_dtype, max_slices, max_rows,
                          max_segments, pinv_rtol, stream, max_staged_rows, n_sweeps)
            h = P()
            st = lib.dash_init(C.byref(cfg), C.byref(h))
            if st != 0:
                raise DashError(st, "dash_init failed")
        else:
            h = _handle
        self._lib, self._h = lib, h
        self.J, self.R, self.lam, self.mode = J, R, lam, mode
        self.np_dtype = np.float64 if input_dtype == "f64" else np.float32

    @classmethod
    def load_file(cls, path: str, J: int, R: int, lam: float, mode: str = "P",
                  input_dtype: str = "f32", stream=None) -> "DashModel":
        """dash_load(): a model resumed from a dash_save() file (the shape
        arguments describe it to the binding; the file sizes the model)."""
        lib = load()
        h = P()
        st = lib.dash_load(os.fsencode(path), stream, C.byref(h))
        if st != 0:
            raise DashError(st, f"dash_load({path}) failed")
        return cls(J, R, lam, mode=mode, input_dtype=input_dtype, _handle=h)

    def save(self, path: str) -> None:
        self._ck(self._lib.dash_save(self._h, os.fsencode(path)))

    def fitness_lambda(self):
        """(λ-weighted fitness of every absorbed row, Σ λ^age ||x||²)."""
        f, x = C.c_double(), C.c_double()
        self._ck(self._lib.dash_fitness_lambda(self._h, C.byref(f), C.byref(x)))
        return f.value, x.value

    def set_wait_limit(self, cycles: int) -> None:
        self._ck(self._lib.dash_set_wait_limit(self._h, int(cycles)))

    def inject_wait_fault(self) -> None:
        self._ck(self._lib.dash_inject_wait_fault(self._h))

    def set_graph(self, on: bool) -> None:
        self._ck(self._lib.dash_set_graph(self._h, 1 if on else 0))

    def graph_stats(self):
        """(graph instantiations, in-place graph updates) since dash_init."""
        a, b = C.c_int64(), C.c_int64()
        self._ck(self._lib.dash_graph_stats(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def set_autotune(self, on: bool) -> None:
        self._ck(self._lib.dash_set_autotune(self._h, 1 if on else 0))

    def autotune_result(self) -> dict:
        """{candidates, chosen, resident, ring, ms} of the X·Q_V autotuning."""
        n, c, r, g = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        ms = (C.c_float * 8)()
        self._ck(self._lib.dash_autotune_result(self._h, C.byref(n), C.byref(c), C.byref(r), C.byref(g), ms))
        return {"candidates": n.value, "chosen": c.value, "resident": bool(r.value), "ring": g.value,
                "ms": [float(ms[i]) for i in range(n.value)]}

    def set_weighted_norm(self, xx: float) -> None:
        self._ck(self._lib.dash_set_weighted_norm(self._h, float(xx)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dash_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st: int):
        if st != 0:
            raise DashError(st, self._lib.dash_last_error(self._h).decode())

    # ---- factors / state ---------------------------------------------------
    @property
    def K(self) -> int:
        return int(self._lib.dash_num_slices(self._h))

    def set_factors(self, V, H=None):
        V = _f64(V, (self.J, self.R))
        Hh = None if H is None else _f64(H, (self.R, self.R))
        self._ck(self._lib.dash_set_factors(self._h, _pd(V), _pd(Hh)))

    def set_state_p(self, V, W, c, D, F, G):
        K = int(np.asarray(W).shape[0])
        R, J = self.R, self.J
        V, W, c = _f64(V, (J, R)), _f64(W, (K, R)), _f64(c, (K, R))
        D, F, G = _f64(D, (K, R, R)), _f64(F, (J, R)), _f64(G, (R, R))
        self._ck(self._lib.dash_set_state_p(self._h, K, _pd(V), _pd(W), _pd(c), _pd(D),
                                            _pd(F), _pd(G)))

    def get_state_p(self) -> dict:
        K, R, J = self.K, self.R, self.J
        out = dict(V=np.empty((J, R)), W=np.empty((K, R)), c=np.empty((K, R)),
                   D=np.empty((K, R, R)), F=np.empty((J, R)), G=np.empty((R, R)))
        self._ck(self._lib.dash_get_state_p(self._h, *(_pd(out[k]) for k in "VWcDFG")))
        return out

    def set_state_q(self, V, H, W, L, Y):
        """Load a mode-Q state: factors V, H, W, the triangular factors L_k of
        B_k and the projected data Y_k = T_k Z_k (K×R×J)."""
        K = int(np.asarray(W).shape[0])
        R, J = self.R, self.J
        V, H, W = _f64(V, (J, R)), _f64(H, (R, R)), _f64(W, (K, R))
        L, Y = _f64(L, (K, R, R)), _f64(Y, (K, R, J))
        self._ck(self._lib.dash_set_state_q(self._h, K, _pd(V), _pd(H), _pd(W), _pd(L), _pd(Y)))

    def get_state_q(self) -> dict:
        K, R, J = self.K, self.R, self.J
        out = dict(V=np.empty((J, R)), H=np.empty((R, R)), W=np.empty((K, R)),
                   L=np.empty((K, R, R)), Y=np.empty((K, R, J)))
        self._ck(self._lib.dash_get_state_q(self._h, *(_pd(out[k]) for k in "VHWLY")))
        return out

    def factors(self, k_first: int = 0, k_count: Optional[int] = None):
        """(V, W rows) in mode P; (V, W rows, H) in mode Q."""
        if k_count is None:
            k_count = self.K - k_first
        V = np.empty((self.J, self.R))
        W = np.empty((k_count, self.R))
        H = np.empty((self.R, self.R)) if self.mode == "Q" else None
        self._ck(self._lib.dash_factors(self._h, _pd(V), _pd(W), k_first, k_count, _pd(H)))
        return (V, W) if H is None else (V, W, H)

    def new_rows(self) -> np.ndarray:
        n = C.c_int64()
        self._ck(self._lib.dash_new_rows(self._h, None, C.byref(n)))
        out = np.empty((n.value, self.R))
        self._ck(self._lib.dash_new_rows(self._h, _pd(out), C.byref(n)))
        return out

    def fitness(self):
        f, x = C.c_double(), C.c_double()
        self._ck(self._lib.dash_fitness(self._h, C.byref(f), C.byref(x)))
        return f.value, x.value

    def last_plan(self) -> dict:
        """How the last batch was planned: tile rows/slices of the fused row
        kernel, tiles, chunked-path rows, general-kernel rows."""
        v = [C.c_int64() for _ in range(5)]
        self._ck(self._lib.dash_last_plan(self._h, *(C.byref(x) for x in v)))
        return dict(zip(("tile_rows", "tile_slices", "tiles", "chunk_rows", "general_rows"),
                        (x.value for x in v)))

    def rows_error(self, slice_ids, row_ptr, X, rows):
        """(Σ||x − x̂||², Σ||x||², Σ|x − x̂|) of the rows of X (a CUDA tensor of
        the input dtype) with factor rows `rows` (CUDA FP64, N×R) against the
        current factors; segments as in append_batch."""
        import torch
        ids, rp = _i64(slice_ids), _i64(row_ptr)
        xp, where, keep = self._ptr(X)
        if where != DEVICE or not (isinstance(rows, torch.Tensor) and rows.is_cuda):
            raise TypeError("rows_error needs CUDA tensors for X and rows")
        rows = rows.to(torch.float64).contiguous()
        e2, x2, ea = C.c_double(), C.c_double(), C.c_double()
        self._ck(self._lib.dash_rows_error(self._h, len(ids), ids.ctypes.data_as(PI64),
                                           rp.ctypes.data_as(PI64), xp, C.c_void_p(rows.data_ptr()),
                                           C.byref(e2), C.byref(x2), C.byref(ea)))
        return e2.value, x2.value, ea.value

    ROW_PATHS = {"auto": 0, "fused": 1, "split": 2, "split-warp": 3}

    def set_row_path(self, path: str) -> None:
        """Mode-P row pipeline for the next updates: "fused", "split" or
        "auto" (the library's choice)."""
        self._ck(self._lib.dash_set_row_path(self._h, self.ROW_PATHS[path]))

    def local_errors(self):
        """(te, direct batch fitness, se per slice (NaN without new rows)) of
        the last update: Definitions 1-2 from a second read of its rows."""
        te, fd = C.c_double(), C.c_double()
        se = np.empty(self.K)
        self._ck(self._lib.dash_local_errors(self._h, C.byref(te), C.byref(fd), _pd(se), se.size))
        return te.value, fd.value, se

    def last_update_ms(self) -> float:
        ms = C.c_float()
        self._ck(self._lib.dash_last_update_ms(self._h, C.byref(ms)))
        return ms.value

    def counters(self):
        """(wait timeouts, FP64 fallback solves) since the model was created."""
        a, b = C.c_int64(), C.c_int64()
        self._ck(self._lib.dash_counters(self._h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def launch_count(self) -> int:
        return int(self._lib.dash_launch_count(self._h))

    def profile(self, on: bool = True, phases: bool = False):
        """Per-launch event timing (on), plus in-kernel phase clocks (phases:
        extra work inside the kernels, for breakdowns rather than timing)."""
        self._ck(self._lib.dash_profile_enable(self._h, (2 if phases else 1) if on else 0))

    def profile_report(self) -> dict:
        """{kernel: (launches, total ms)} since profiling was enabled."""
        out = {}
        for i in range(self._lib.dash_profile_kinds()):
            name, n, ms = C.c_char_p(), C.c_int64(), C.c_double()
            self._ck(self._lib.dash_profile_get(self._h, i, C.byref(name), C.byref(n), C.byref(ms)))
            if n.value:
                out[name.value.decode()] = (n.value, ms.value)
        return out

    def sync(self):
        self._ck(self._lib.dash_sync(self._h))

    def device_bytes(self) -> int:
        """Device memory the model owns."""
        return int(self._lib.dash_device_bytes(self._h))

    def idle(self) -> bool:
        """True when all work the model has issued has finished (never waits)."""
        v = C.c_int32()
        self._ck(self._lib.dash_query(self._h, C.byref(v)))
        return bool(v.value)

    # ---- staging -------------------------------------------------------------
    def _ptr(self, X):
        """(pointer, where, keepalive) of a host numpy array or a CUDA tensor."""
        if hasattr(X, "is_cuda") and X.is_cuda:
            want = {np.float64: "float64", np.float32: "float32"}[self.np_dtype]
            if str(X.dtype).split(".")[-1] != want or not X.is_contiguous():
                raise TypeError(f"device X must be a contiguous {want} tensor")
            return C.c_void_p(X.data_ptr()), DEVICE, X
        if hasattr(X, "numpy"):
            X = X.numpy()
        X = np.ascontiguousarray(np.asarray(X, dtype=self.np_dtype))
        return C.c_void_p(X.ctypes.data), HOST, X

    def append_rows(self, k: int, X):
        ptr, where, keep = self._ptr(X)
        n = int(keep.shape[0])
        self._ck(self._lib.dash_append_rows(self._h, k, ptr, n, self.J, where))

    def append_slices(self, Xs: Sequence) -> int:
        ptrs, keeps, rows, where = [], [], [], HOST
        for X in Xs:
            p, where, keep = self._ptr(X)
            ptrs.append(p.value or 0)
            keeps.append(keep)
            rows.append(int(keep.shape[0]))
        L = len(rows)
        I = _i64(rows)
        arr = (C.c_void_p * max(L, 1))(*ptrs)
        first = C.c_int64()
        self._ck(self._lib.dash_append_slices(self._h, L, I.ctypes.data_as(PI64), arr, None,
                                              where, C.byref(first)))
        return first.value

    def append_batch(self, slice_ids, row_ptr, X):
        ids, rp = _i64(slice_ids), _i64(row_ptr)
        ptr, where, keep = self._ptr(X)
        self._ck(self._lib.dash_append_batch(self._h, len(ids), ids.ctypes.data_as(PI64),
                                             rp.ctypes.data_as(PI64), ptr, where))

    def update(self):
        self._ck(self._lib.dash_update(self._h))

    def update_device(self, slice_ids, row_ptr, X):
        ids, rp = _i64(slice_ids), _i64(row_ptr)
        ptr, where, keep = self._ptr(X)
        if where != DEVICE:
            raise TypeError("update_device needs a CUDA tensor")
        self._ck(self._lib.dash_update_device(self._h, len(ids), ids.ctypes.data_as(PI64),
                                              rp.ctypes.data_as(PI64), ptr))

    def fit_initial(self, n_iter: int):
        self._ck(self._lib.dash_fit_initial(self._h, n_iter))

    def fit_initial_device(self, slice_ids, row_ptr, X, n_iter: int):
        ids, rp = _i64(slice_ids), _i64(row_ptr)
        ptr, where, keep = self._ptr(X)
        if where != DEVICE:
            raise TypeError("fit_initial_device needs a CUDA tensor")
        self._ck(self._lib.dash_fit_initial_device(self._h, len(ids), ids.ctypes.data_as(PI64),
                                                   rp.ctypes.data_as(PI64), ptr, n_iter))
