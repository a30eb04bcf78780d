"""Thin ctypes binding of include/ptycho_serve.h (batching and serving), plus
the arrival-stream driver used by the serving benchmark and tests.

The scheduling itself (admission by HBM budget, rounds, retirement, graph
capture) runs in libptycho.so; this module only marshals arguments and, in
``run_stream``, submits requests at their arrival times and calls
``ptycho_server_step`` until every request is done.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import native
from .native import PtychoError, _P, _check, _ptr

PTYCHO_REQ_QUEUED, PTYCHO_REQ_ACTIVE, PTYCHO_REQ_DONE, PTYCHO_REQ_FAILED = 0, 1, 2, 3


class ptycho_scan_desc(ctypes.Structure):
    _fields_ = [("J", ctypes.c_int32), ("N", ctypes.c_int32), ("M_rows", ctypes.c_int32),
                ("M_cols", ctypes.c_int32), ("pos_rc", _P), ("intensity", _P), ("obj0", _P),
                ("probe0", _P)]


_SIGS = {
    "ptycho_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(native.ptycho_opts)]),
    "ptycho_batch_add": (ctypes.c_int, [_P, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "ptycho_batch_run": (ctypes.c_int, [_P, ctypes.c_int32]),
    "ptycho_batch_destroy": (None, [_P]),
    "ptycho_batch_set_mode": (ctypes.c_int, [_P, ctypes.c_int]),
    "ptycho_batch_info": (ctypes.c_int, [_P, ctypes.c_void_p]),
    "ptycho_server_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_size_t, ctypes.c_int32,
                                            ctypes.POINTER(native.ptycho_opts)]),
    "ptycho_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(ptycho_scan_desc), ctypes.c_float,
                                            ctypes.c_float, ctypes.c_float, ctypes.c_int32,
                                            ctypes.POINTER(ctypes.c_uint64)]),
    "ptycho_server_step": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32)]),
    "ptycho_server_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32), _P, _P,
                                          _P]),
    "ptycho_server_destroy": (None, [_P]),
}

_ready = False


def lib() -> ctypes.CDLL:
    global _ready
    L = native.lib()
    if not _ready:
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _ready = True
    return L


def _rc(rc: int, what: str) -> None:
    if rc != native.PTYCHO_OK:
        raise PtychoError(rc, what)


# --- the ABI, one function each -------------------------------------------

def ptycho_batch_create(opts: native.ptycho_opts | None = None) -> int:
    h = _P()
    _rc(lib().ptycho_batch_create(ctypes.byref(h), ctypes.byref(opts) if opts else None),
        "ptycho_batch_create")
    return h.value


def ptycho_batch_add(b: int, ctx: int, a: float, bb: float, c: float) -> None:
    _rc(lib().ptycho_batch_add(b, ctx, a, bb, c), "ptycho_batch_add")


def ptycho_batch_run(b: int, n_iter: int) -> None:
    _rc(lib().ptycho_batch_run(b, n_iter), "ptycho_batch_run")


PTYCHO_BATCH_AUTO, PTYCHO_BATCH_GROUPS, PTYCHO_BATCH_BRANCHES = 0, 1, 2


class ptycho_batch_info_t(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_int32), ("in_groups", ctypes.c_int32), ("used", ctypes.c_int32),
                ("groups_ms", ctypes.c_float), ("branches_ms", ctypes.c_float)]


def ptycho_batch_set_mode(b: int, mode: int) -> None:
    _rc(lib().ptycho_batch_set_mode(b, mode), "ptycho_batch_set_mode")


def ptycho_batch_info(b: int) -> dict:
    t = ptycho_batch_info_t()
    _rc(lib().ptycho_batch_info(b, ctypes.addressof(t)), "ptycho_batch_info")
    return {"groups": t.groups, "in_groups": t.in_groups,
            "used": {1: "groups", 2: "branches"}.get(t.used, ""),
            "groups_ms": float(t.groups_ms), "branches_ms": float(t.branches_ms)}


def ptycho_batch_destroy(b: int) -> None:
    lib().ptycho_batch_destroy(b)


def ptycho_server_create(budget_bytes: int, max_active: int,
                         opts: native.ptycho_opts | None = None) -> int:
    h = _P()
    _rc(lib().ptycho_server_create(ctypes.byref(h), budget_bytes, max_active,
                                   ctypes.byref(opts) if opts else None), "ptycho_server_create")
    return h.value


def ptycho_server_submit(s: int, pos, intensity, obj0, probe0, a: float, b: float, c: float,
                         n_iter: int) -> int:
    pos = np.ascontiguousarray(pos, dtype=np.int32)
    inten = np.ascontiguousarray(intensity, dtype=np.float32)
    obj0 = np.ascontiguousarray(obj0, dtype=np.complex64)
    probe0 = np.ascontiguousarray(probe0, dtype=np.complex64)
    d = ptycho_scan_desc(pos.shape[0], inten.shape[-1], obj0.shape[0], obj0.shape[1],
                         _ptr(pos), _ptr(inten), _ptr(obj0), _ptr(probe0))
    rid = ctypes.c_uint64(0)
    _rc(lib().ptycho_server_submit(s, ctypes.byref(d), a, b, c, n_iter, ctypes.byref(rid)),
        "ptycho_server_submit")
    return rid.value


def ptycho_server_step(s: int, iters_per_round: int) -> tuple[int, int]:
    na, nq = ctypes.c_int32(0), ctypes.c_int32(0)
    _rc(lib().ptycho_server_step(s, iters_per_round, ctypes.byref(na), ctypes.byref(nq)),
        "ptycho_server_step")
    return na.value, nq.value


def ptycho_server_poll(s: int, rid: int, obj_out=None, probe_out=None):
    st = ctypes.c_int32(0)
    times = np.zeros(4, dtype=np.float64)
    _rc(lib().ptycho_server_poll(s, rid, ctypes.byref(st), _ptr(obj_out), _ptr(probe_out),
                                 _ptr(times)), "ptycho_server_poll")
    return st.value, times


def ptycho_server_destroy(s: int) -> None:
    lib().ptycho_server_destroy(s)


# --- drivers ----------------------------------------------------------------

def run_batch(recons, settings, n_iter: int, device: int = 0, mode: int = PTYCHO_BATCH_AUTO) -> dict:
    """Advance several loaded Reconstructions together through one captured
    graph; returns what the batch did (ptycho_batch_info)."""
    o = native.ptycho_default_opts()
    o.device = device
    b = ptycho_batch_create(o)
    try:
        ptycho_batch_set_mode(b, mode)
        for r, abc in zip(recons, settings):
            ptycho_batch_add(b, r.h, *abc)
        ptycho_batch_run(b, n_iter)
        return ptycho_batch_info(b)
    finally:
        ptycho_batch_destroy(b)


def run_stream(scans, settings, n_iter: int, arrivals_s, budget_bytes: int, max_active: int,
               iters_per_round: int = 10, device: int = 0, keep_results: bool = False):
    """Submit scans[i] at arrivals_s[i] (seconds from start), serve all to
    completion, return per-request records and the wall time."""
    o = native.ptycho_default_opts()
    o.device = device
    s = ptycho_server_create(budget_bytes, max_active, o)
    order = np.argsort(arrivals_s, kind="stable")
    ids = [None] * len(scans)
    try:
        t0 = time.perf_counter()
        nxt = 0
        remaining = len(scans)
        done = set()
        records = [None] * len(scans)
        while remaining:
            now = time.perf_counter() - t0
            while nxt < len(order) and arrivals_s[order[nxt]] <= now:
                i = int(order[nxt])
                sc = scans[i]
                ids[i] = ptycho_server_submit(s, sc.pos, sc.intensity, sc.obj0, sc.probe0,
                                              *settings[i], n_iter)
                nxt += 1
            na, nq = ptycho_server_step(s, iters_per_round)
            if nxt - na - nq == len(done):   # nxt requests submitted so far
                # no request finished in this step: nothing to poll
                if na == 0 and nq == 0 and nxt < len(order):
                    time.sleep(max(0.0, min(0.01, arrivals_s[order[nxt]] - (time.perf_counter() - t0))))
                continue
            for i, rid in enumerate(ids):
                if rid is None or i in done:
                    continue
                O = P = None
                if keep_results:
                    O = np.empty(scans[i].M_shape, dtype=np.complex64)
                    P = np.empty((scans[i].N, scans[i].N), dtype=np.complex64)
                st, times = ptycho_server_poll(s, rid, O, P)
                if st in (PTYCHO_REQ_DONE, PTYCHO_REQ_FAILED):
                    done.add(i)
                    remaining -= 1
                    records[i] = {"state": st, "queue_s": times[0], "latency_s": times[1],
                                  "per100_s": times[2], "final_error": times[3], "O": O, "P": P}
            if na == 0 and nq == 0 and nxt < len(order):
                time.sleep(max(0.0, min(0.01, arrivals_s[order[nxt]] - (time.perf_counter() - t0))))
        wall = time.perf_counter() - t0
    finally:
        ptycho_server_destroy(s)
    return records, wall
