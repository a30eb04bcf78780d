"""Thin ctypes binding of the C ABI in include/ptycho.h (argument marshalling only).

Every function of the ABI appears here under the same name; ``Reconstruction``
wraps them for convenience.  All computation runs in libptycho.so on the GPU:
there is no CPU or PyTorch fallback, and loading fails loudly when the library
has not been built (call ``paper_2311_11466_gb300.build.build()``).

Complex arrays cross the boundary as numpy complex64 (interleaved float32,
C order), positions as int32 [J, 2] (row, col), intensities as float32
[J, N, N] (host numpy, or a CUDA tensor's device pointer).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# PTYCHO_LIB=debug selects the checked build (libptycho_debug.so) for this process.
LIB_PATH = os.path.join(_PKG, "libptycho_debug.so" if os.environ.get("PTYCHO_LIB") == "debug"
                        else "libptycho.so")

PTYCHO_OK, PTYCHO_EINVAL, PTYCHO_ENOMEM, PTYCHO_ECUDA, PTYCHO_ETIMEOUT, PTYCHO_ESTATE = 0, -1, -2, -3, -4, -5
PTYCHO_PREC_FP32, PTYCHO_PREC_BF16X3 = 0, 1
PTYCHO_CONCUR_DETERMINISTIC, PTYCHO_CONCUR_ATOMIC = 0, 1
PTYCHO_DIVIDE_AUTO, PTYCHO_DIVIDE_CLUSTER, PTYCHO_DIVIDE_TWOPASS = 0, 1, 2
DIVIDE = {"auto": PTYCHO_DIVIDE_AUTO, "cluster": PTYCHO_DIVIDE_CLUSTER, "twopass": PTYCHO_DIVIDE_TWOPASS}
PTYCHO_LOAD_INTENSITY_DEVICE = 1

_STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ESTATE"}

# (a, b, c) of the named algorithms; DC is the paper's own definition
# (Introduction), the others are readings of the general update: expanding
# a P^b_C P^c_D x + (1 - a) x gives DR = (R_C R_D + I) / 2 for (1/2, 2, 2),
# RAAR(beta) = (beta/2)(R_C R_D + I) + (1 - beta) P_D for (1/2, 2 beta, 2),
# RRR(beta) = x + beta (P_C R_D x - P_D x) for (beta/2, 2, 2), SF = R_C P_D for
# (1, 2, 1) and AR = R_C R_D for (1, 2, 2).  Data, not code: every setting
# runs the same kernels.
PRESETS = {
    "DC": (1.0, 1.0, 1.0),
    "AR": (1.0, 2.0, 2.0),
    "DR": (0.5, 2.0, 2.0),
    "SF": (1.0, 2.0, 1.0),
    "RAAR": (0.5, 1.8, 2.0),   # beta = 0.9
    "RRR": (0.25, 2.0, 2.0),   # beta = 0.5
}


def raar(beta: float) -> tuple[float, float, float]:
    return (0.5, 2.0 * beta, 2.0)


def rrr(beta: float) -> tuple[float, float, float]:
    return (beta / 2.0, 2.0, 2.0)


class PtychoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class ptycho_opts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("precision", ctypes.c_int), ("concur", ctypes.c_int),
                ("alpha", ctypes.c_float), ("stream", ctypes.c_void_p), ("divide", ctypes.c_int)]


class ptycho_tuning_info(ctypes.Structure):
    _fields_ = [("tuned", ctypes.c_int32), ("gather_rows", ctypes.c_int32),
                ("gather_cols", ctypes.c_int32), ("probe_ppt", ctypes.c_int32),
                ("gather_ms", ctypes.c_float * 4), ("probe_ms", ctypes.c_float * 2),
                ("cluster_size", ctypes.c_int32), ("divide_ms", ctypes.c_float * 2)]


_lib = None

_P = ctypes.c_void_p
_SIGS = {
    "ptycho_default_opts": (None, [ctypes.POINTER(ptycho_opts)]),
    "ptycho_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(ptycho_opts)]),
    "ptycho_destroy": (None, [_P]),
    "ptycho_last_error": (ctypes.c_char_p, [_P]),
    "ptycho_load_scan": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_int32,
                                        ctypes.c_int32, _P, _P, ctypes.c_uint32]),
    "ptycho_iterate": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_int32]),
    "ptycho_sp_iterate": (ctypes.c_int, [_P, ctypes.c_float, _P, ctypes.c_int32]),
    "ptycho_check_bounded_wait": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint32]),
    "ptycho_get_object_probe": (ctypes.c_int, [_P, _P, _P]),
    "ptycho_set_object_probe": (ctypes.c_int, [_P, _P, _P]),
    "ptycho_get_exit_waves": (ctypes.c_int, [_P, _P]),
    "ptycho_set_exit_waves": (ctypes.c_int, [_P, _P]),
    "ptycho_errors": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "ptycho_iteration_count": (ctypes.c_int64, [_P]),
    "ptycho_model_error": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "ptycho_device_bytes": (ctypes.c_size_t, [_P]),
    "ptycho_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "ptycho_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int32)]),
    "ptycho_scan_bytes": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int]),
    "ptycho_divide_design": (ctypes.c_int, [_P]),
    "ptycho_set_probe_start": (ctypes.c_int, [_P, ctypes.c_int32]),
    "ptycho_set_tuning": (ctypes.c_int, [_P, ctypes.c_int]),
    "ptycho_tuning": (ctypes.c_int, [_P, ctypes.POINTER(ptycho_tuning_info)]),
    "ptycho_set_launch_shapes": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_int32]),
    "ptycho_debug_build": (ctypes.c_int, []),
    "ptycho_debug_flags": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_uint32)]),
    "ptycho_probe_update_noalloc": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                                   _P, _P]),
}


def lib() -> ctypes.CDLL:
    """Load libptycho.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run paper_2311_11466_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a) -> int:
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a.data_ptr())  # a torch tensor


def _check(rc: int, handle) -> None:
    if rc != PTYCHO_OK:
        msg = lib().ptycho_last_error(handle)
        raise PtychoError(rc, msg.decode() if msg else "")


def _c64(a, shape=None) -> np.ndarray:
    out = np.ascontiguousarray(a, dtype=np.complex64)
    if shape is not None and out.shape != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {out.shape}")
    return out


# --- the ABI, one function each -------------------------------------------

def ptycho_default_opts() -> ptycho_opts:
    o = ptycho_opts()
    lib().ptycho_default_opts(ctypes.byref(o))
    return o


def ptycho_create(opts: ptycho_opts | None = None) -> int:
    h = _P()
    rc = lib().ptycho_create(ctypes.byref(h), ctypes.byref(opts) if opts is not None else None)
    _check(rc, None)
    return h.value


def ptycho_destroy(h: int) -> None:
    lib().ptycho_destroy(h)


def ptycho_last_error(h: int | None) -> str:
    return lib().ptycho_last_error(h).decode()


def ptycho_load_scan(h, pos, intensity, obj0, probe0) -> None:
    pos = np.ascontiguousarray(pos, dtype=np.int32)
    J = pos.shape[0]
    flags = 0
    if isinstance(intensity, np.ndarray):
        inten = np.ascontiguousarray(intensity, dtype=np.float32)
        N = inten.shape[-1]
    else:  # a CUDA tensor: pass its device pointer (dense float32 only)
        if (str(getattr(intensity, "dtype", "")) != "torch.float32" or not intensity.is_contiguous()
                or not getattr(intensity, "is_cuda", False)):
            raise ValueError("a device intensity must be a contiguous float32 CUDA tensor")
        inten = intensity
        N = int(intensity.shape[-1])
        flags |= PTYCHO_LOAD_INTENSITY_DEVICE
    obj0 = _c64(obj0)
    probe0 = _c64(probe0, (N, N))
    if pos.ndim != 2 or pos.shape[1] != 2 or tuple(inten.shape) != (J, N, N):
        raise ValueError("pos must be [J, 2] and intensity [J, N, N]")
    rc = lib().ptycho_load_scan(h, J, N, _ptr(pos), _ptr(inten), obj0.shape[0], obj0.shape[1],
                                _ptr(obj0), _ptr(probe0), flags)
    _check(rc, h)


def ptycho_iterate(h, a: float, b: float, c: float, n_iter: int) -> None:
    _check(lib().ptycho_iterate(h, a, b, c, n_iter), h)


def ptycho_check_bounded_wait(device: int, timeout_ms: int) -> int:
    """Status code of a bounded wait that must expire (PTYCHO_ETIMEOUT expected)."""
    return int(lib().ptycho_check_bounded_wait(device, timeout_ms))


def ptycho_sp_iterate(h, lam: float, order, n_iter: int) -> None:
    o = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    _check(lib().ptycho_sp_iterate(h, lam, _ptr(o), n_iter), h)


def ptycho_get_object_probe(h, obj_out: np.ndarray | None, probe_out: np.ndarray | None) -> None:
    _check(lib().ptycho_get_object_probe(h, _ptr(obj_out), _ptr(probe_out)), h)


def ptycho_set_object_probe(h, obj: np.ndarray | None, probe: np.ndarray | None) -> None:
    _check(lib().ptycho_set_object_probe(h, _ptr(obj), _ptr(probe)), h)


def ptycho_get_exit_waves(h, x_out: np.ndarray) -> None:
    _check(lib().ptycho_get_exit_waves(h, _ptr(x_out)), h)


def ptycho_set_exit_waves(h, x: np.ndarray) -> None:
    _check(lib().ptycho_set_exit_waves(h, _ptr(x)), h)


def ptycho_errors(h, cap: int) -> np.ndarray:
    out = np.zeros(max(cap, 0), dtype=np.float64)
    n = ctypes.c_int32(0)
    _check(lib().ptycho_errors(h, _ptr(out), cap, ctypes.byref(n)), h)
    return out[:n.value]


def ptycho_iteration_count(h) -> int:
    return int(lib().ptycho_iteration_count(h))


def ptycho_model_error(h) -> float:
    v = ctypes.c_double(0.0)
    _check(lib().ptycho_model_error(h, ctypes.byref(v)), h)
    return v.value


def ptycho_device_bytes(h) -> int:
    return int(lib().ptycho_device_bytes(h))


def ptycho_profile_enable(h, enable: bool) -> None:
    _check(lib().ptycho_profile_enable(h, 1 if enable else 0), h)


def ptycho_profile_read(h) -> tuple[float, float, int]:
    d, c, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    _check(lib().ptycho_profile_read(h, ctypes.byref(d), ctypes.byref(c), ctypes.byref(n)), h)
    return d.value, c.value, n.value


def ptycho_scan_bytes(J: int, N: int, M_rows: int, M_cols: int, precision: int = 0) -> int:
    return int(lib().ptycho_scan_bytes(J, N, M_rows, M_cols, precision))


def ptycho_debug_build() -> bool:
    return bool(lib().ptycho_debug_build())


def ptycho_debug_flags(device: int = 0) -> int:
    """Synchronise the device and read-and-clear the checked build's bits."""
    f = ctypes.c_uint32(0)
    rc = lib().ptycho_debug_flags(device, ctypes.byref(f))
    if rc != PTYCHO_OK:
        raise PtychoError(rc, "ptycho_debug_flags")
    return int(f.value)


def ptycho_set_tuning(h, enable: bool) -> None:
    _check(lib().ptycho_set_tuning(h, 1 if enable else 0), h)


def ptycho_tuning(h) -> dict:
    t = ptycho_tuning_info()
    _check(lib().ptycho_tuning(h, ctypes.byref(t)), h)
    return {"tuned": bool(t.tuned), "gather_tile": (t.gather_rows, t.gather_cols),
            "probe_pixels_per_thread": t.probe_ppt,
            "gather_ms": {f"{r}x{c}": float(t.gather_ms[i])
                          for i, (r, c) in enumerate(((16, 32), (8, 32), (32, 32), (8, 64)))},
            "probe_ms": {"1": float(t.probe_ms[0]), "2": float(t.probe_ms[1])},
            "cluster_size": t.cluster_size,
            "divide128_ms": {"8x128": float(t.divide_ms[0]), "16x64": float(t.divide_ms[1])}}


def ptycho_set_launch_shapes(h, gather_rows: int, gather_cols: int, probe_ppt: int,
                             cluster_size: int = 0) -> None:
    _check(lib().ptycho_set_launch_shapes(h, gather_rows, gather_cols, probe_ppt, cluster_size), h)


def ptycho_set_probe_start(h, start: int) -> None:
    _check(lib().ptycho_set_probe_start(h, start), h)


def ptycho_divide_design(h) -> int:
    return int(lib().ptycho_divide_design(h))


def ptycho_probe_update_noalloc(y_dev: int, obj_dev: int, pos_dev: int, J: int, N: int,
                                M_rows: int, M_cols: int, alpha: float, probe_out_dev: int,
                                stream: int | None = None) -> int:
    """Probe update from device pointers with no device allocation; returns the
    status code (PTYCHO_OK on success) instead of raising."""
    return int(lib().ptycho_probe_update_noalloc(y_dev, obj_dev, pos_dev, J, N, M_rows, M_cols,
                                                 alpha, probe_out_dev, stream))


# --- convenience wrapper ---------------------------------------------------

class Reconstruction:
    """One blind reconstruction held on the GPU (a ptycho_ctx)."""

    def __init__(self, device: int = 0, precision: str = "fp32", concur: str = "deterministic",
                 alpha: float = 1e-6, stream: int | None = None, divide: str = "auto"):
        o = ptycho_default_opts()
        o.device = device
        o.precision = {"fp32": PTYCHO_PREC_FP32, "bf16x3": PTYCHO_PREC_BF16X3}[precision]
        o.concur = {"deterministic": PTYCHO_CONCUR_DETERMINISTIC, "atomic": PTYCHO_CONCUR_ATOMIC}[concur]
        o.alpha = alpha
        o.stream = stream
        o.divide = DIVIDE[divide]
        self.h = ptycho_create(o)
        self.J = self.N = 0
        self.M_shape = (0, 0)

    def close(self) -> None:
        if getattr(self, "h", None):
            ptycho_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def load_scan(self, pos, intensity, obj0, probe0) -> None:
        ptycho_load_scan(self.h, pos, intensity, obj0, probe0)
        self.J = int(np.asarray(pos).shape[0])
        self.N = int(np.asarray(probe0).shape[0])
        self.M_shape = tuple(np.asarray(obj0).shape)

    def iterate(self, a: float, b: float, c: float, n: int = 1) -> None:
        ptycho_iterate(self.h, a, b, c, n)

    def sp_iterate(self, lam: float = 1.0, n: int = 1, order=None) -> None:
        """n passes of sequential projections (order: a permutation, or ascending)."""
        ptycho_sp_iterate(self.h, lam, order, n)

    def run(self, name: str, n: int) -> None:
        self.iterate(*PRESETS[name], n)

    def object_probe(self) -> tuple[np.ndarray, np.ndarray]:
        O = np.empty(self.M_shape, dtype=np.complex64)
        P = np.empty((self.N, self.N), dtype=np.complex64)
        ptycho_get_object_probe(self.h, O, P)
        return O, P

    def set_object_probe(self, O=None, P=None) -> None:
        ptycho_set_object_probe(self.h, None if O is None else _c64(O, self.M_shape),
                                None if P is None else _c64(P, (self.N, self.N)))

    def exit_waves(self) -> np.ndarray:
        x = np.empty((self.J, self.N, self.N), dtype=np.complex64)
        ptycho_get_exit_waves(self.h, x)
        return x

    def set_exit_waves(self, x) -> None:
        ptycho_set_exit_waves(self.h, _c64(x, (self.J, self.N, self.N)))

    def errors(self) -> np.ndarray:
        return ptycho_errors(self.h, min(ptycho_iteration_count(self.h), 65536))

    def model_error(self) -> float:
        return ptycho_model_error(self.h)

    @property
    def iteration_count(self) -> int:
        return ptycho_iteration_count(self.h)

    def set_tuning(self, enable: bool) -> None:
        ptycho_set_tuning(self.h, enable)

    def tuning(self) -> dict:
        """The launch shapes the autotuner chose (and what it measured)."""
        return ptycho_tuning(self.h)

    def set_launch_shapes(self, gather_rows: int, gather_cols: int, probe_ppt: int,
                          cluster_size: int = 0) -> None:
        ptycho_set_launch_shapes(self.h, gather_rows, gather_cols, probe_ppt, cluster_size)

    def set_probe_start(self, start: int) -> None:
        """Hold the probe fixed in iterations k < start (k from 0 at the load)."""
        ptycho_set_probe_start(self.h, start)

    def divide_design(self) -> str:
        """'cluster' or 'twopass': the divide design of the loaded scan."""
        return {PTYCHO_DIVIDE_CLUSTER: "cluster", PTYCHO_DIVIDE_TWOPASS: "twopass"}.get(
            ptycho_divide_design(self.h), "")

    @property
    def device_bytes(self) -> int:
        return ptycho_device_bytes(self.h)
