"""B300-native decentralized baseband processing (sm_103a CUDA behind a C ABI).

Thin Python binding of ``libdbp.so`` (declared in ``include/dbp.h``): the
functions here carry the C names and only marshal arguments.  Every step of
the computation runs in the library's CUDA kernels; there is no Python or CPU
fallback, and importing this package fails loudly when the library is absent.

Device buffers are passed as torch CUDA tensors (or raw integer addresses);
host buffers for the ``*_host`` variants as numpy arrays or CPU tensors.
Streams are ``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers or
None (the current torch stream is then used for device calls).
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdbp.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -m paper_1702_04458_b300.build` "
        "(there is no fallback implementation)")

_lib = ctypes.CDLL(LIB_PATH)

# ---------------------------------------------------------------------------
# Types mirrored from include/dbp.h
# ---------------------------------------------------------------------------
DBP_OK = 0
DBP_ERR_INVALID_ARG = 1
DBP_ERR_UNSUPPORTED = 2
DBP_ERR_NOMEM = 3
DBP_ERR_CUDA = 4
DBP_ERR_TIMEOUT = 5
DBP_ERR_UNIMPLEMENTED = 6
DBP_PENDING = 7
DBP_ERR_CANCELLED = 8

DBP_FP32, DBP_FP64, DBP_FP16, DBP_BF16 = 0, 1, 2, 3
DBP_REG_ZF, DBP_REG_MMSE, DBP_REG_BOX, DBP_REG_BPSK = 0, 1, 2, 3
DBP_FLAG_NORMALIZE = 1
DBP_MAP_AUTO, DBP_MAP_CTA, DBP_MAP_CLUSTER = 0, 1, 2
DBP_PATH_AUTO, DBP_PATH_GENERIC, DBP_PATH_TMA, DBP_PATH_MMA, DBP_PATH_BCAST, DBP_PATH_TC5 = 0, 1, 2, 3, 4, 5
DBP_PREFACTOR_AUTO, DBP_PREFACTOR_OFF, DBP_PREFACTOR_ON = 0, 1, 2

_STATUS = {0: "DBP_OK", 1: "DBP_ERR_INVALID_ARG", 2: "DBP_ERR_UNSUPPORTED", 3: "DBP_ERR_NOMEM",
           4: "DBP_ERR_CUDA", 5: "DBP_ERR_TIMEOUT", 6: "DBP_ERR_UNIMPLEMENTED", 7: "DBP_PENDING",
           8: "DBP_ERR_CANCELLED"}


class dbp_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_uint64)]


class dbp_frame_desc(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int32), ("C", ctypes.c_int32), ("U", ctypes.c_int32),
                ("W", ctypes.c_int32), ("N", ctypes.c_int32), ("qam_order", ctypes.c_int32),
                ("T_max", ctypes.c_int32), ("regularizer", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("rho", ctypes.c_double), ("gamma", ctypes.c_double), ("N0", ctypes.c_double),
                ("Es", ctypes.c_double), ("box_r", ctypes.c_double), ("eps", ctypes.c_double)]


class dbp_graph_item(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("desc", dbp_frame_desc),
                ("H", ctypes.c_void_p), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("labels", ctypes.c_void_p), ("beta_out", ctypes.c_void_p)]


class dbp_tuning(ctypes.Structure):
    _fields_ = [("mapping", ctypes.c_int32), ("cluster_size", ctypes.c_int32),
                ("warps_per_cta", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("prefactor", ctypes.c_int32)]


_P = ctypes.c_void_p
_H = ctypes.c_void_p
_S = ctypes.c_int

_lib.dbp_version.restype = ctypes.c_char_p
_lib.dbp_version.argtypes = []
_lib.dbp_create.restype = _S
_lib.dbp_create.argtypes = [ctypes.POINTER(_H), ctypes.POINTER(dbp_config)]
_lib.dbp_destroy.restype = _S
_lib.dbp_destroy.argtypes = [_H]
_lib.dbp_last_error.restype = ctypes.c_char_p
_lib.dbp_last_error.argtypes = [_H]
_lib.dbp_set_tuning.restype = _S
_lib.dbp_set_tuning.argtypes = [_H, ctypes.POINTER(dbp_tuning)]
for _name in ("dbp_uplink_admm", "dbp_uplink_cg", "dbp_uplink_admm_host", "dbp_uplink_cg_host"):
    getattr(_lib, _name).restype = _S
    getattr(_lib, _name).argtypes = [_H, ctypes.POINTER(dbp_frame_desc), _P, _P, _P, _P, _P]
for _name in ("dbp_downlink_admm", "dbp_downlink_admm_host"):
    getattr(_lib, _name).restype = _S
    getattr(_lib, _name).argtypes = [_H, ctypes.POINTER(dbp_frame_desc), _P, _P, _P, _P, _P]


class DbpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


def _ptr(x):
    """Address of a torch tensor, numpy array, ctypes object or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    return ctypes.addressof(x)


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(h, status: int):
    if status != DBP_OK:
        msg = _lib.dbp_last_error(h)
        raise DbpError(status, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# C entry points (same names)
# ---------------------------------------------------------------------------

def dbp_version() -> str:
    return _lib.dbp_version().decode()


def dbp_create(device: int = 0, hbm_budget_bytes: int = 0):
    h = _H()
    cfg = dbp_config(device, 0, hbm_budget_bytes)
    st = _lib.dbp_create(ctypes.byref(h), ctypes.byref(cfg))
    if st != DBP_OK:
        raise DbpError(st, "dbp_create failed (no usable CUDA device?)")
    return h


def dbp_destroy(h) -> None:
    _check(h, _lib.dbp_destroy(h))


def dbp_last_error(h) -> str:
    return _lib.dbp_last_error(h).decode()


def dbp_set_tuning(h, mapping: int = DBP_MAP_AUTO, cluster_size: int = 0, warps_per_cta: int = 0,
                   kernel: int = DBP_PATH_AUTO, prefactor: int = 0) -> None:
    t = dbp_tuning(mapping, cluster_size, warps_per_cta, kernel, prefactor)
    _check(h, _lib.dbp_set_tuning(h, ctypes.byref(t)))


def frame_desc(B, C, U, W, N, qam_order=0, T_max=3, regularizer=DBP_REG_MMSE,
               precision=DBP_FP32, flags=0, rho=1.0, gamma=1.0, N0=0.0, Es=1.0,
               box_r=0.0, eps=0.0) -> dbp_frame_desc:
    return dbp_frame_desc(B, C, U, W, N, qam_order, T_max, regularizer, precision, flags,
                          rho, gamma, N0, Es, box_r, eps)


_lib.dbp_device_status.restype = _S
_lib.dbp_device_status.argtypes = [_H]


def dbp_device_status(h) -> None:
    _check(h, _lib.dbp_device_status(h))


_lib.dbp_fp64_retries.restype = _S
_lib.dbp_fp64_retries.argtypes = [_H, ctypes.POINTER(ctypes.c_uint32)]


def dbp_fp64_retries(h) -> int:
    n = ctypes.c_uint32(0)
    _check(h, _lib.dbp_fp64_retries(h, ctypes.byref(n)))
    return int(n.value)


def dbp_uplink_admm(h, d, H, y, x_hat, labels=None, stream=None) -> None:
    _check(h, _lib.dbp_uplink_admm(h, ctypes.byref(d), _ptr(H), _ptr(y), _ptr(x_hat),
                                   _ptr(labels), _stream(stream)))


def dbp_uplink_cg(h, d, H, y, x_hat, labels=None, stream=None) -> None:
    _check(h, _lib.dbp_uplink_cg(h, ctypes.byref(d), _ptr(H), _ptr(y), _ptr(x_hat),
                                 _ptr(labels), _stream(stream)))


def dbp_downlink_admm(h, d, H, s, x, beta_out=None, stream=None) -> None:
    _check(h, _lib.dbp_downlink_admm(h, ctypes.byref(d), _ptr(H), _ptr(s), _ptr(x),
                                     _ptr(beta_out), _stream(stream)))


def dbp_uplink_admm_host(h, d, H, y, x_hat, labels=None, stream=0) -> None:
    _check(h, _lib.dbp_uplink_admm_host(h, ctypes.byref(d), _ptr(H), _ptr(y), _ptr(x_hat),
                                        _ptr(labels), _stream(stream)))


def dbp_uplink_cg_host(h, d, H, y, x_hat, labels=None, stream=0) -> None:
    _check(h, _lib.dbp_uplink_cg_host(h, ctypes.byref(d), _ptr(H), _ptr(y), _ptr(x_hat),
                                      _ptr(labels), _stream(stream)))


def dbp_downlink_admm_host(h, d, H, s, x, beta_out=None, stream=0) -> None:
    _check(h, _lib.dbp_downlink_admm_host(h, ctypes.byref(d), _ptr(H), _ptr(s), _ptr(x),
                                          _ptr(beta_out), _stream(stream)))


# Downlink with normalisation for callers that cannot allocate device memory
# (see dbp_downlink_admm_static in include/dbp.h).
DBP_STATIC_MAX_SUBCARRIERS = 16384
_lib.dbp_downlink_admm_static.restype = _S
_lib.dbp_downlink_admm_static.argtypes = [_H, ctypes.POINTER(dbp_frame_desc), _P, _P, _P, _P, _P]


def dbp_downlink_admm_static(h, d, H, s, x, beta_out=None, stream=None) -> None:
    _check(h, _lib.dbp_downlink_admm_static(h, ctypes.byref(d), _ptr(H), _ptr(s), _ptr(x),
                                            _ptr(beta_out), _stream(stream)))


# ---------------------------------------------------------------------------
# Request loop (serving)
# ---------------------------------------------------------------------------
DBP_KIND_UPLINK_ADMM, DBP_KIND_UPLINK_CG, DBP_KIND_DOWNLINK_ADMM = 0, 1, 2


class dbp_server_config(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_int32), ("reserved", ctypes.c_int32), ("hbm_bytes", ctypes.c_uint64)]


class dbp_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("flags", ctypes.c_uint32), ("desc", dbp_frame_desc),
                ("H", ctypes.c_void_p), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("labels", ctypes.c_void_p), ("beta_out", ctypes.c_void_p),
                ("channel_key", ctypes.c_uint64), ("coherence_epoch", ctypes.c_uint64),
                ("user_tag", ctypes.c_uint64)]


class dbp_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("resident_hit", ctypes.c_int32), ("user_tag", ctypes.c_uint64),
                ("submit_us", ctypes.c_double), ("start_us", ctypes.c_double), ("finish_us", ctypes.c_double)]


_lib.dbp_server_start.restype = _S
_lib.dbp_server_start.argtypes = [_H, ctypes.POINTER(dbp_server_config)]
_lib.dbp_server_stop.restype = _S
_lib.dbp_server_stop.argtypes = [_H]
_lib.dbp_submit.restype = _S
_lib.dbp_submit.argtypes = [_H, ctypes.POINTER(dbp_request), ctypes.POINTER(ctypes.c_uint64)]
_lib.dbp_poll.restype = _S
_lib.dbp_poll.argtypes = [_H, ctypes.c_uint64, ctypes.POINTER(dbp_result)]
_lib.dbp_wait.restype = _S
_lib.dbp_wait.argtypes = [_H, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(dbp_result)]


def dbp_server_start(h, streams: int = 4, hbm_bytes: int = 0) -> None:
    cfg = dbp_server_config(streams, 0, hbm_bytes)
    _check(h, _lib.dbp_server_start(h, ctypes.byref(cfg)))


def dbp_server_stop(h) -> None:
    _check(h, _lib.dbp_server_stop(h))


DBP_REQ_DEVICE_BUFFERS = 1


def request(kind, desc, H, inp, out, labels=None, beta_out=None, channel_key=0, coherence_epoch=0,
            user_tag=0, flags=0) -> dbp_request:
    """flags=DBP_REQ_DEVICE_BUFFERS: H, inp, out, labels, beta_out are device
    buffers (e.g. CUDA tensors) used in place; otherwise host buffers."""
    return dbp_request(kind, flags, desc, _ptr(H), _ptr(inp), _ptr(out), _ptr(labels), _ptr(beta_out),
                       channel_key, coherence_epoch, user_tag)


def dbp_submit(h, req: dbp_request) -> int:
    t = ctypes.c_uint64(0)
    _check(h, _lib.dbp_submit(h, ctypes.byref(req), ctypes.byref(t)))
    return int(t.value)


DBP_TEST_STARVE_COPY = 1
_lib.dbp_set_test_faults.restype = _S
_lib.dbp_set_test_faults.argtypes = [_H, ctypes.c_uint32]


def dbp_set_test_faults(h, flags: int) -> None:
    _check(h, _lib.dbp_set_test_faults(h, flags))


_lib.dbp_cancel.restype = _S
_lib.dbp_cancel.argtypes = [_H, ctypes.c_uint64]


def dbp_cancel(h, ticket: int) -> bool:
    """True if the queued frame was cancelled (its ticket then finishes with
    DBP_ERR_CANCELLED), False if it was already admitted and runs."""
    st = _lib.dbp_cancel(h, ticket)
    if st == DBP_PENDING:
        return False
    _check(h, st)
    return True


def dbp_poll(h, ticket: int):
    """None while pending, else the dbp_result (ticket released)."""
    r = dbp_result()
    st = _lib.dbp_poll(h, ticket, ctypes.byref(r))
    if st == DBP_PENDING:
        return None
    _check(h, st)
    return r


def dbp_wait(h, ticket: int, timeout_s: float = 60.0):
    """The dbp_result, or None if the frame is not done within timeout_s."""
    r = dbp_result()
    st = _lib.dbp_wait(h, ticket, timeout_s, ctypes.byref(r))
    if st == DBP_ERR_TIMEOUT:
        return None
    _check(h, st)
    return r


_lib.dbp_graph_create.restype = _S
_lib.dbp_graph_create.argtypes = [_H, ctypes.POINTER(dbp_graph_item), ctypes.c_int32, ctypes.c_int32,
                                  ctypes.POINTER(ctypes.c_void_p)]
_lib.dbp_graph_launch.restype = _S
_lib.dbp_graph_launch.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
_lib.dbp_graph_destroy.restype = _S
_lib.dbp_graph_destroy.argtypes = [ctypes.c_void_p]


_lib.dbp_uplink_llr.restype = _S
_lib.dbp_uplink_llr.argtypes = [_H, ctypes.POINTER(dbp_frame_desc), ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p]


def dbp_uplink_llr(h, d, H, x_hat, llr, stream=None) -> None:
    """Max-log LLRs [W][N][U][log2 M] (float32) of an uplink estimate."""
    _check(h, _lib.dbp_uplink_llr(h, ctypes.byref(d), _ptr(H), _ptr(x_hat), _ptr(llr), _stream(stream)))


_lib.dbp_autotune.restype = _S
_lib.dbp_autotune.argtypes = [_H, ctypes.c_int32, ctypes.POINTER(dbp_frame_desc), ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                              ctypes.POINTER(dbp_tuning)]
_lib.dbp_autotune_clear.restype = _S
_lib.dbp_autotune_clear.argtypes = [_H]
_lib.dbp_autotune_save.restype = _S
_lib.dbp_autotune_save.argtypes = [_H, ctypes.c_char_p]
_lib.dbp_autotune_load.restype = _S
_lib.dbp_autotune_load.argtypes = [_H, ctypes.c_char_p]


def dbp_autotune(h, kind, d, H, inp, out, labels=None, stream=None, reps: int = 0) -> dbp_tuning:
    """Time the launch choices for this frame shape; the fastest is used by
    later fully automatic calls and returned."""
    t = dbp_tuning()
    _check(h, _lib.dbp_autotune(h, kind, ctypes.byref(d), _ptr(H), _ptr(inp), _ptr(out), _ptr(labels),
                                _stream(stream), reps, ctypes.byref(t)))
    return t


_lib.dbp_plan.restype = _S
_lib.dbp_plan.argtypes = [_H, ctypes.c_int32, ctypes.POINTER(dbp_frame_desc), ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.c_void_p, ctypes.POINTER(dbp_tuning)]


def dbp_plan(h, kind, d, H, inp, out) -> dbp_tuning:
    """The launch choice a call of this kind would make for these buffers
    (kernel path, mapping, cluster size, warps per CTA, separate operator
    kernel), resolved without launching anything."""
    t = dbp_tuning()
    _check(h, _lib.dbp_plan(h, kind, ctypes.byref(d), _ptr(H), _ptr(inp), _ptr(out), ctypes.byref(t)))
    return t


def dbp_autotune_clear(h) -> None:
    _check(h, _lib.dbp_autotune_clear(h))


def dbp_autotune_save(h, path: str) -> None:
    _check(h, _lib.dbp_autotune_save(h, path.encode()))


def dbp_autotune_load(h, path: str) -> None:
    _check(h, _lib.dbp_autotune_load(h, path.encode()))


def graph_item(kind, desc, H, inp, out, labels=None, beta_out=None) -> dbp_graph_item:
    return dbp_graph_item(kind, 0, desc, _ptr(H), _ptr(inp), _ptr(out), _ptr(labels), _ptr(beta_out))


class DbpGraph:
    """A captured batch of frames (dbp_graph_create); launch() runs them all."""

    def __init__(self, h, items, branches: int = 0):
        arr = (dbp_graph_item * len(items))(*items)
        g = ctypes.c_void_p(None)
        _check(h, _lib.dbp_graph_create(h, arr, len(items), branches, ctypes.byref(g)))
        self._h, self._g = h, g

    def launch(self, stream=None) -> None:
        _check(self._h, _lib.dbp_graph_launch(self._g, _stream(stream)))

    def close(self) -> None:
        if self._g:
            _check(self._h, _lib.dbp_graph_destroy(self._g))
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dbp_graph_create(h, items, branches: int = 0) -> DbpGraph:
    return DbpGraph(h, items, branches)


def dbp_graph_launch(g: DbpGraph, stream=None) -> None:
    g.launch(stream)


def dbp_graph_destroy(g: DbpGraph) -> None:
    g.close()


__all__ = [n for n in dir() if n.startswith(("dbp_", "DBP_")) or n in ("frame_desc", "request", "graph_item",
                                                                      "DbpGraph", "DbpError", "LIB_PATH")]
