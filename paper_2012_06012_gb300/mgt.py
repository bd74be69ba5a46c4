"""Thin Python binding of libmgt.so (argument marshalling only).

Every function here forwards to the C ABI declared in include/mgt.h; the
transposition itself runs in the library's CUDA kernels.  PyTorch is used
for device memory and streams.  There is no fallback: if libmgt.so is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmgt.so")

MGT_OK, MGT_EINVAL, MGT_ENOMEM, MGT_EBADINPUT = 0, -1, -2, -3
MGT_ETIMEOUT, MGT_EAGAIN, MGT_ECUDA, MGT_EOVERFLOW, MGT_ENOTFOUND = -4, -5, -6, -7, -8
MGT_FLAG_VAR_WIDTH = 1

_lock = threading.Lock()
_lib = None


class MgtError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = _load().mgt_strerror(code).decode() if _lib is not None else str(code)
        if code == MGT_ECUDA and _lib is not None:
            msg += " [" + (_lib.mgt_last_error() or b"").decode() + "]"
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")
        self.code = code


class Desc(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64),
                ("n_cells", ctypes.c_int64), ("n_values", ctypes.c_int64),
                ("offset_bytes", ctypes.c_int32), ("payload_stride", ctypes.c_int32),
                ("n_parts", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("part_off", ctypes.POINTER(ctypes.c_int64))]


class XcsrIn(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("cell_ptr", ctypes.c_void_p), ("values", ctypes.c_void_p)]


class XcsrOut(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("cell_ptr", ctypes.c_void_p), ("values", ctypes.c_void_p),
                ("part_cells", ctypes.c_void_p), ("part_values", ctypes.c_void_p)]


class XcsrBuf(ctypes.Structure):
    _fields_ = [("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("cell_ptr", ctypes.c_void_p), ("values", ctypes.c_void_p)]


class TileCfg(ctypes.Structure):
    _fields_ = [("bucket_shift", ctypes.c_int32), ("scatter_tile", ctypes.c_int32),
                ("cluster", ctypes.c_int32), ("chunk_cap", ctypes.c_int32),
                ("copy_unroll", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]

    def as_dict(self):
        return {"bucket_shift": self.bucket_shift, "scatter_tile": self.scatter_tile,
                "cluster": self.cluster, "chunk_cap": self.chunk_cap,
                "copy_unroll": self.copy_unroll}


class ServerCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("max_queue", ctypes.c_int32),
                ("batch_max", ctypes.c_int32), ("fuse_max_cells", ctypes.c_int64),
                ("batch_window_us", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "submitted", "completed", "failed", "rejected", "launches", "fused_requests", "bytes",
        "peak_inflight_bytes", "peak_inflight_requests", "inflight_bytes", "queued")] + \
        [(n, ctypes.c_double) for n in ("p50_ms", "p99_ms", "mean_ms", "span_s")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


# names exported by libmgt.so and declared in include/mgt.h
EXPORTS = ["mgt_plan", "mgt_plan_tuned", "mgt_plan_config", "mgt_plan_destroy", "mgt_transpose",
           "mgt_transpose_profiled", "mgt_plan_phases", "mgt_plan_kernel_launches", "mgt_read_status", "mgt_batched_workspace", "mgt_transpose_batched",
           "mgt_minimal_bytes", "mgt_strerror", "mgt_version", "mgt_transpose_static",
           "mgt_static_status", "mgt_batch_create", "mgt_batch_launch",
           "mgt_batch_kernel_launches", "mgt_batch_status", "mgt_batch_destroy", "mgt_last_error",
           "mgt_autotune_candidates", "mgt_autotune_workspace", "mgt_autotune",
           "mgt_transpose_batched_profiled", "mgt_transpose_values", "mgt_transpose_host",
           "mgt_server_create", "mgt_submit", "mgt_poll", "mgt_server_drain", "mgt_server_get_stats",
           "mgt_server_reset_stats", "mgt_server_destroy", "mgt_probe_runs", "mgt_transpose_var", "mgt_probe_errors",
           "mgt_l2_fetch_granularity"]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libmgt.so not built ({LIB_PATH}); run __graft_entry__.build()")
            lib = ctypes.CDLL(LIB_PATH, mode=ctypes.RTLD_GLOBAL)
            vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
            P = ctypes.POINTER
            lib.mgt_plan.argtypes = [P(Desc), P(vp), P(sz)]
            lib.mgt_plan.restype = i32
            lib.mgt_plan_tuned.argtypes = [P(Desc), P(TileCfg), P(vp), P(sz)]
            lib.mgt_plan_tuned.restype = i32
            lib.mgt_plan_config.argtypes = [vp, P(TileCfg)]
            lib.mgt_plan_config.restype = i32
            lib.mgt_plan_destroy.argtypes = [vp]
            lib.mgt_plan_destroy.restype = None
            lib.mgt_transpose.argtypes = [vp, P(XcsrIn), P(XcsrOut), vp, sz, vp]
            lib.mgt_transpose.restype = i32
            lib.mgt_transpose_values.argtypes = [vp, P(XcsrIn), P(XcsrOut), vp, sz, vp]
            lib.mgt_transpose_values.restype = i32
            lib.mgt_transpose_host.argtypes = [vp, P(XcsrIn), P(XcsrOut), P(XcsrBuf), P(XcsrOut), vp, sz,
                                               vp, vp]
            lib.mgt_transpose_host.restype = i32
            lib.mgt_transpose_profiled.argtypes = [vp, P(XcsrIn), P(XcsrOut), vp, sz, vp, P(vp), i32]
            lib.mgt_transpose_profiled.restype = i32
            lib.mgt_plan_phases.argtypes = [vp, P(ctypes.c_char_p), i32]
            lib.mgt_plan_phases.restype = i32
            lib.mgt_plan_kernel_launches.argtypes = [vp]
            lib.mgt_plan_kernel_launches.restype = i32
            lib.mgt_read_status.argtypes = [vp, vp]
            lib.mgt_read_status.restype = i32
            lib.mgt_batched_workspace.argtypes = [i32, P(vp), P(sz)]
            lib.mgt_batched_workspace.restype = i32
            lib.mgt_transpose_batched.argtypes = [i32, P(vp), P(XcsrIn), P(XcsrOut), vp, sz, vp]
            lib.mgt_transpose_batched.restype = i32
            lib.mgt_transpose_batched_profiled.argtypes = [i32, P(vp), P(XcsrIn), P(XcsrOut), vp, sz, vp,
                                                           P(vp), i32]
            lib.mgt_transpose_batched_profiled.restype = i32
            lib.mgt_batch_create.argtypes = [i32, P(vp), P(XcsrIn), P(XcsrOut), vp, sz, P(vp)]
            lib.mgt_batch_create.restype = i32
            lib.mgt_batch_launch.argtypes = [vp, vp]
            lib.mgt_batch_launch.restype = i32
            lib.mgt_batch_kernel_launches.argtypes = [vp]
            lib.mgt_batch_kernel_launches.restype = i32
            lib.mgt_batch_status.argtypes = [vp, vp, P(i32)]
            lib.mgt_batch_status.restype = i32
            lib.mgt_batch_destroy.argtypes = [vp]
            lib.mgt_batch_destroy.restype = None
            lib.mgt_minimal_bytes.argtypes = [P(Desc)]
            lib.mgt_minimal_bytes.restype = i64
            lib.mgt_strerror.argtypes = [i32]
            lib.mgt_strerror.restype = ctypes.c_char_p
            lib.mgt_transpose_static.argtypes = [P(Desc), P(XcsrIn), P(XcsrOut), vp]
            lib.mgt_transpose_static.restype = i32
            lib.mgt_static_status.argtypes = [vp]
            lib.mgt_static_status.restype = i32
            lib.mgt_autotune_candidates.argtypes = [P(Desc), P(TileCfg), i32]
            lib.mgt_autotune_candidates.restype = i32
            lib.mgt_autotune_workspace.argtypes = [P(Desc), P(sz)]
            lib.mgt_autotune_workspace.restype = i32
            lib.mgt_autotune.argtypes = [P(Desc), P(XcsrIn), P(XcsrOut), vp, sz, vp, i32, P(TileCfg),
                                         P(ctypes.c_float)]
            lib.mgt_autotune.restype = i32
            lib.mgt_server_create.argtypes = [P(ServerCfg), P(vp)]
            lib.mgt_server_create.restype = i32
            lib.mgt_submit.argtypes = [vp, vp, P(XcsrIn), P(XcsrOut), P(ctypes.c_uint64)]
            lib.mgt_submit.restype = i32
            lib.mgt_poll.argtypes = [vp, ctypes.c_uint64, P(i32), P(i32), P(ctypes.c_double)]
            lib.mgt_poll.restype = i32
            lib.mgt_server_drain.argtypes = [vp]
            lib.mgt_server_drain.restype = i32
            lib.mgt_server_get_stats.argtypes = [vp, P(ServerStats)]
            lib.mgt_server_get_stats.restype = i32
            lib.mgt_server_reset_stats.argtypes = [vp]
            lib.mgt_server_reset_stats.restype = i32
            lib.mgt_server_destroy.argtypes = [vp]
            lib.mgt_server_destroy.restype = None
            lib.mgt_last_error.argtypes = []
            lib.mgt_last_error.restype = ctypes.c_char_p
            lib.mgt_transpose_var.argtypes = [vp, P(XcsrIn), vp, P(XcsrOut), vp, i64, vp, sz, vp,
                                              P(vp), i32]
            lib.mgt_transpose_var.restype = i32
            lib.mgt_probe_runs.argtypes = [i32, vp, vp, vp, i64, ctypes.c_int32, vp]
            lib.mgt_probe_runs.restype = i32
            lib.mgt_probe_errors.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
            lib.mgt_probe_errors.restype = i32
            lib.mgt_l2_fetch_granularity.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
            lib.mgt_l2_fetch_granularity.restype = i32
            lib.mgt_version.argtypes = []
            lib.mgt_version.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def lib():
    return _load()


def _check(rc: int, what: str):
    if rc != MGT_OK:
        raise MgtError(rc, what)


def make_desc(n_rows, n_cols, n_cells, n_values, offset_bytes, payload_stride, part_off=None,
              flags=0):
    """Returns (Desc, keepalive) -- keepalive holds the part_off array."""
    d = Desc()
    d.n_rows, d.n_cols, d.n_cells, d.n_values = int(n_rows), int(n_cols), int(n_cells), int(n_values)
    d.offset_bytes, d.payload_stride = int(offset_bytes), int(payload_stride)
    keep = None
    if part_off is None:
        d.n_parts = 1
        d.part_off = ctypes.POINTER(ctypes.c_int64)()
    else:
        keep = np.ascontiguousarray(part_off, dtype=np.int64)
        d.n_parts = int(keep.shape[0] - 1)
        d.part_off = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.flags = int(flags)
    return d, keep


class Plan:
    """Owns an mgt_plan_t (host metadata only)."""

    def __init__(self, n_rows, n_cols, n_cells, n_values, offset_bytes, payload_stride,
                 part_off=None, cfg: dict | None = None, var_width: bool = False):
        L = _load()
        self.var_width = bool(var_width)
        self.desc, self._keep = make_desc(n_rows, n_cols, n_cells, n_values, offset_bytes,
                                          1 if var_width else payload_stride, part_off,
                                          MGT_FLAG_VAR_WIDTH if var_width else 0)
        self.n_parts = self.desc.n_parts
        h = ctypes.c_void_p()
        ws = ctypes.c_size_t()
        if cfg:
            c = TileCfg()
            for k, v in cfg.items():
                setattr(c, k, int(v))
            rc = L.mgt_plan_tuned(ctypes.byref(self.desc), ctypes.byref(c), ctypes.byref(h),
                                  ctypes.byref(ws))
        else:
            rc = L.mgt_plan(ctypes.byref(self.desc), ctypes.byref(h), ctypes.byref(ws))
        _check(rc, "mgt_plan")
        self.handle = h
        self.workspace_bytes = int(ws.value)

    @property
    def config(self) -> dict:
        c = TileCfg()
        _check(_load().mgt_plan_config(self.handle, ctypes.byref(c)), "mgt_plan_config")
        return c.as_dict()

    @property
    def phases(self) -> list[str]:
        n = _load().mgt_plan_phases(self.handle, None, 0)
        arr = (ctypes.c_char_p * n)()
        _load().mgt_plan_phases(self.handle, arr, n)
        return [a.decode() for a in arr]

    @property
    def kernel_launches(self) -> int:
        return int(_load().mgt_plan_kernel_launches(self.handle))

    def minimal_bytes(self) -> int:
        return int(_load().mgt_minimal_bytes(ctypes.byref(self.desc)))

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.mgt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _nbytes(a) -> int:
    """Bytes of a numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        return int(a.nbytes)
    return int(a.numel() * a.element_size())


def _itemsize(a) -> int:
    return int(a.itemsize) if isinstance(a, np.ndarray) else int(a.element_size())


_IN_NAMES = ("row_ptr", "col_idx", "cell_ptr", "values")
_OUT_NAMES = _IN_NAMES + ("part_cells", "part_values")


def _expected(plan: "Plan"):
    """Byte sizes and element widths the C ABI reads or writes through each
    array of one transpose with ``plan``: (input sizes, output sizes, input
    widths, output widths).  A width of None accepts any element type; a raw
    byte buffer (element size 1) is accepted for every array."""
    d = plan.desc
    o, C, V, s, P = d.offset_bytes, d.n_cells, d.n_values, d.payload_stride, d.n_parts
    ins = ((d.n_rows + 1) * o, C * 4, (C + 1) * o, V * s)
    outs = ((d.n_cols + 1) * o, C * 4, (C + 1) * o, V * s, P * P * 8, P * P * 8)
    return ins, outs, (o, 4, o, None), (o, 4, o, None, 8, 8)


def check_arrays(plan: "Plan", inp=None, out=None, what: str = "", device: bool | None = None):
    """Refuses, before any call into the library, arrays whose byte size or
    element width does not match the plan: the library copies or writes
    exactly the plan's sizes through the raw pointers, so a short array (or
    one of the wrong offset width) would be read or written past its end.
    ``device``: True requires CUDA tensors, False host arrays, None either.
    The optional P x P outputs may be None or larger than P * P."""
    ins, outs, wi, wo = _expected(plan)
    for arrays, sizes, widths, names, side in ((inp, ins, wi, _IN_NAMES, "input"),
                                               (out, outs, wo, _OUT_NAMES, "output")):
        if arrays is None:
            continue
        for k, a in enumerate(arrays):
            if a is None or k >= len(sizes):
                continue
            name = f"{what}{side} {names[k]}"
            if device is not None and not isinstance(a, np.ndarray):
                if bool(a.is_cuda) != device:
                    raise ValueError(f"{name}: expected a {'CUDA' if device else 'host'} array")
            elif device and isinstance(a, np.ndarray):
                raise ValueError(f"{name}: expected a CUDA tensor, got a numpy array")
            nb, want = _nbytes(a), sizes[k]
            if (nb < want) if k >= 4 else (nb != want):
                raise ValueError(f"{name}: {nb} bytes, the plan needs {want}")
            w = widths[k]
            if w is not None and _itemsize(a) not in (1, w):
                raise ValueError(f"{name}: elements of {_itemsize(a)} bytes, the plan's are {w}")


def transpose(plan: Plan, inp, out, workspace, stream=None):
    """inp: (row_ptr, col_idx, cell_ptr, values) device tensors; out: a
    (row_ptr, col_idx, cell_ptr, values, part_cells, part_values) tuple
    (the last two may be None).  Enqueues on ``stream``."""
    check_arrays(plan, inp, out, device=True)
    xi = XcsrIn(*[_ptr(t) for t in inp])
    xo = XcsrOut(*[_ptr(t) for t in out])
    rc = _load().mgt_transpose(plan.handle, ctypes.byref(xi), ctypes.byref(xo), _ptr(workspace),
                               workspace.numel() * workspace.element_size(), _stream_handle(stream))
    _check(rc, "mgt_transpose")


def transpose_values(plan: Plan, inp, out, workspace, stream=None):
    """Re-transposes only the values (mgt_transpose_values): ``inp``/``out``
    as for transpose(), whose structure arrays must be those of the last
    full transpose made with this plan and workspace."""
    check_arrays(plan, inp, out, device=True)
    xi = XcsrIn(*[_ptr(t) for t in inp])
    xo = XcsrOut(*[_ptr(t) for t in out])
    rc = _load().mgt_transpose_values(plan.handle, ctypes.byref(xi), ctypes.byref(xo), _ptr(workspace),
                                      workspace.numel() * workspace.element_size(), _stream_handle(stream))
    _check(rc, "mgt_transpose_values")


def _hptr(a):
    """Host address of a contiguous numpy array or CPU torch tensor (None stays
    None).  No copy is made: the asynchronous copies read and write the
    caller's own memory, which must stay alive until the stream reaches them."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if not a.is_contiguous() or a.is_cuda:
        raise ValueError("host tensors must be contiguous CPU tensors")
    return ctypes.c_void_p(a.data_ptr())


def transpose_host(plan: Plan, host_in, host_out, dev_in, dev_out, workspace, stream=None,
                   copy_stream=None):
    """Transposes a matrix held in host memory (mgt_transpose_host): uploads
    ``host_in`` (row_ptr, col_idx, cell_ptr, values; numpy arrays or CPU
    tensors, pinned for asynchronous copies) into the device buffers
    ``dev_in``, transposes into ``dev_out`` (as for transpose()), and downloads
    the result into ``host_out`` (four arrays, or six with the P x P counts).
    ``copy_stream``: a second torch stream on which the copies that do not
    feed the next kernel overlap the kernels.  Every host and device array
    must have exactly the plan's size (ValueError otherwise, before any copy)."""
    check_arrays(plan, host_in, host_out, what="host ", device=False)
    check_arrays(plan, dev_in, dev_out, what="device ", device=True)
    hi = XcsrIn(*[_hptr(a) for a in host_in])
    ho = list(host_out) + [None] * (6 - len(host_out))
    ho = XcsrOut(*[_hptr(a) for a in ho])
    di = XcsrBuf(*[_ptr(t) for t in dev_in])
    do = XcsrOut(*[_ptr(t) for t in dev_out])
    cs = None if copy_stream is None else ctypes.c_void_p(copy_stream.cuda_stream)
    rc = _load().mgt_transpose_host(plan.handle, ctypes.byref(hi), ctypes.byref(ho), ctypes.byref(di),
                                    ctypes.byref(do), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(),
                                    _stream_handle(stream), cs)
    _check(rc, "mgt_transpose_host")


def transpose_profiled(plan: Plan, inp, out, workspace, events, stream=None):
    """As transpose(); ``events``: list of torch.cuda.Event (len >= phases + 1)
    recorded around the phases on the same stream."""
    check_arrays(plan, inp, out, device=True)
    xi = XcsrIn(*[_ptr(t) for t in inp])
    xo = XcsrOut(*[_ptr(t) for t in out])
    for e in events:
        if not e.cuda_event:  # torch creates the CUDA event on its first record
            e.record(stream)
    ev = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
    rc = _load().mgt_transpose_profiled(plan.handle, ctypes.byref(xi), ctypes.byref(xo),
                                        _ptr(workspace), workspace.numel() * workspace.element_size(),
                                        _stream_handle(stream), ev, len(events))
    _check(rc, "mgt_transpose_profiled")


def transpose_var(plan: Plan, inp, in_val_off, out, out_val_off, workspace, stream=None,
                  events=None):
    """Variable-width values (mgt_transpose_var): ``inp`` = (row_ptr, col_idx,
    cell_ptr, value bytes) device tensors, ``in_val_off`` the int64 byte
    offsets of the input values (n_values + 1); ``out`` as for transpose()
    (value bytes the same size as the input's) and ``out_val_off`` the int64
    output offsets.  ``events``: optional torch.cuda.Event list around the
    phases (as transpose_profiled)."""
    if not plan.var_width:
        raise ValueError("transpose_var needs a plan made with var_width=True")
    V = plan.desc.n_values
    n_bytes = _nbytes(inp[3]) if inp[3] is not None else 0
    for name, a in (("input value offsets", in_val_off), ("output value offsets", out_val_off)):
        if a is None or not a.is_cuda or a.element_size() != 8 or a.numel() != V + 1:
            raise ValueError(f"{name}: a CUDA int64 tensor of n_values + 1 entries")
    ins, outs, _, _ = _expected(plan)
    for k, (a, want) in enumerate(zip(inp[:3], ins[:3])):
        if a is None or not a.is_cuda or _nbytes(a) != want:
            raise ValueError(f"input {_IN_NAMES[k]}: {None if a is None else _nbytes(a)} bytes, the plan needs {want}")
    for k, (a, want) in enumerate(zip(out[:3], outs[:3])):
        if a is None or not a.is_cuda or _nbytes(a) != want:
            raise ValueError(f"output {_OUT_NAMES[k]}: {None if a is None else _nbytes(a)} bytes, the plan needs {want}")
    if n_bytes and (out[3] is None or _nbytes(out[3]) != n_bytes):
        raise ValueError("output value bytes must be as many as the input's")
    for k in (4, 5):
        if len(out) > k and out[k] is not None and _nbytes(out[k]) < outs[k]:
            raise ValueError(f"output {_OUT_NAMES[k]}: shorter than P * P")
    xi = XcsrIn(*[_ptr(t) for t in inp])
    xo = XcsrOut(*[_ptr(t) for t in (list(out) + [None] * (6 - len(out)))])
    ev, nev = None, 0
    if events is not None:
        for e in events:
            if not e.cuda_event:
                e.record(stream)
        ev = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
        nev = len(events)
    rc = _load().mgt_transpose_var(plan.handle, ctypes.byref(xi), _ptr(in_val_off), ctypes.byref(xo),
                                   _ptr(out_val_off), int(n_bytes), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(),
                                   _stream_handle(stream), ev, nev)
    _check(rc, "mgt_transpose_var")


def read_status(workspace, stream=None) -> int:
    return int(_load().mgt_read_status(_ptr(workspace), _stream_handle(stream)))


def batched_workspace(plans) -> int:
    arr = (ctypes.c_void_p * len(plans))(*[p.handle for p in plans])
    sz = ctypes.c_size_t()
    _check(_load().mgt_batched_workspace(len(plans), arr, ctypes.byref(sz)), "mgt_batched_workspace")
    return int(sz.value)


def transpose_batched(plans, inps, outs, workspace, stream=None):
    n = len(plans)
    for m in range(n):
        check_arrays(plans[m], inps[m], outs[m], what=f"member {m} ", device=True)
    arr = (ctypes.c_void_p * n)(*[p.handle for p in plans])
    xi = (XcsrIn * n)(*[XcsrIn(*[_ptr(t) for t in i]) for i in inps])
    xo = (XcsrOut * n)(*[XcsrOut(*[_ptr(t) for t in o]) for o in outs])
    rc = _load().mgt_transpose_batched(n, arr, xi, xo, _ptr(workspace),
                                       workspace.numel() * workspace.element_size(),
                                       _stream_handle(stream))
    _check(rc, "mgt_transpose_batched")


def autotune_candidates(x, with_parts=True) -> list[dict]:
    """Tile shapes the autotuner may try for matrix ``x`` (sizes only)."""
    po = x.part_off if (with_parts and x.part_off is not None and len(x.part_off) > 2) else None
    d, keep = make_desc(x.n_rows, x.n_cols, x.n_cells, x.n_values, x.offset_bytes, x.stride, po)
    arr = (TileCfg * 64)()
    n = _load().mgt_autotune_candidates(ctypes.byref(d), arr, 64)
    if n < 0:
        _check(n, "mgt_autotune_candidates")
    return [arr[i].as_dict() for i in range(min(n, 64))]


def autotune(x: "DeviceXCSR", reps: int = 2, out=None, workspace=None, stream=None,
             with_parts=True) -> tuple[dict, float]:
    """Times the candidate tile shapes on device matrix ``x`` (mgt_autotune);
    returns (shape dict for Plan(cfg=...), mean ms of the winner)."""
    po = x.part_off if (with_parts and x.part_off is not None and len(x.part_off) > 2) else None
    d, keep = make_desc(x.n_rows, x.n_cols, x.n_cells, x.n_values, x.offset_bytes, x.stride, po)
    if workspace is None:
        sz = ctypes.c_size_t()
        _check(_load().mgt_autotune_workspace(ctypes.byref(d), ctypes.byref(sz)), "mgt_autotune_workspace")
        workspace = alloc_workspace(int(sz.value))
    out = out or alloc_output(x, parts=po is not None)
    xi = XcsrIn(*[_ptr(t) for t in x.arrays()])
    xo = XcsrOut(*[_ptr(t) for t in out])
    best = TileCfg()
    ms = ctypes.c_float()
    rc = _load().mgt_autotune(ctypes.byref(d), ctypes.byref(xi), ctypes.byref(xo), _ptr(workspace),
                              workspace.numel() * workspace.element_size(), _stream_handle(stream),
                              int(reps), ctypes.byref(best), ctypes.byref(ms))
    _check(rc, "mgt_autotune")
    return best.as_dict(), float(ms.value)


class TuneCache:
    """Autotuned shapes per size class: (offset width, stride, P > 1, log2 of
    the rows, log2 of the cells per row).  The first matrix of a class is
    tuned on itself; later ones reuse its shape.  With a file (``path``, or
    the MGT_TUNE_CACHE environment variable) the shapes persist as JSON, so a
    later process does not tune the same classes again."""

    def __init__(self, reps: int = 2, path: str | None = None):
        self.reps = reps
        self.path = path if path is not None else os.environ.get("MGT_TUNE_CACHE")
        self.best: dict[tuple, dict] = {}
        if self.path and os.path.exists(self.path):
            import json
            with open(self.path) as f:
                for k, v in json.load(f).items():
                    self.best[tuple(json.loads(k))] = {n: int(x) for n, x in v.items()}

    def save(self):
        """Writes the cache file (atomically: a temporary file, then a rename)."""
        if not self.path:
            return
        import json
        tmp = self.path + ".tmp"
        with open(tmp, "w") as f:
            json.dump({json.dumps(list(k)): v for k, v in sorted(self.best.items())}, f, indent=1)
        os.replace(tmp, self.path)

    @staticmethod
    def key(x) -> tuple:
        import math
        parts = x.part_off is not None and len(x.part_off) > 2
        cpr = x.n_cells / max(1, x.n_rows)
        return (x.offset_bytes, x.stride, parts, int(math.log2(max(1, x.n_rows))),
                int(round(math.log2(max(1e-9, cpr)))) if cpr > 0 else -99)

    def cfg_for(self, x: "DeviceXCSR", stream=None) -> dict:
        k = self.key(x)
        if k not in self.best:
            self.best[k], _ = autotune(x, self.reps, stream=stream)
            self.save()
        return self.best[k]


class Batch:
    """A reusable batch of independent transposes: one launch per phase over
    all members, captured once into a CUDA graph (mgt_batch_create).  The
    tensors passed in stay bound to it; launch() recomputes every member
    from what its inputs then hold."""

    def __init__(self, plans, inps, outs, workspace):
        n = len(plans)
        for m in range(n):
            check_arrays(plans[m], inps[m], outs[m], what=f"member {m} ", device=True)
        arr = (ctypes.c_void_p * n)(*[p.handle for p in plans])
        xi = (XcsrIn * n)(*[XcsrIn(*[_ptr(t) for t in i]) for i in inps])
        xo = (XcsrOut * n)(*[XcsrOut(*[_ptr(t) for t in o]) for o in outs])
        h = ctypes.c_void_p()
        rc = _load().mgt_batch_create(n, arr, xi, xo, _ptr(workspace),
                                      workspace.numel() * workspace.element_size(), ctypes.byref(h))
        _check(rc, "mgt_batch_create")
        self.handle = h
        self.n = n
        self._keep = (plans, inps, outs, workspace)

    @property
    def kernel_launches(self) -> int:
        return int(_load().mgt_batch_kernel_launches(self.handle))

    def launch(self, stream=None):
        _check(_load().mgt_batch_launch(self.handle, _stream_handle(stream)), "mgt_batch_launch")

    def status(self, stream=None) -> list[int]:
        st = (ctypes.c_int32 * self.n)()
        _load().mgt_batch_status(self.handle, _stream_handle(stream), st)
        return [int(v) for v in st]

    def close(self):
        if getattr(self, "handle", None):
            _load().mgt_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The serving loop (mgt_server_*): submit() queues a transpose on
    caller-owned device tensors, which this object keeps alive until poll()
    reports the request done."""

    def __init__(self, hbm_budget_bytes=180 * 10**9, max_slots=64, n_streams=4, max_queue=4096,
                 batch_max=16, fuse_max_cells=1 << 22, batch_window_us=0):
        cfg = ServerCfg(int(hbm_budget_bytes), max_slots, n_streams, max_queue, batch_max,
                        int(fuse_max_cells), int(batch_window_us))
        h = ctypes.c_void_p()
        _check(_load().mgt_server_create(ctypes.byref(cfg), ctypes.byref(h)), "mgt_server_create")
        self.handle = h
        self._live: dict[int, tuple] = {}

    def submit(self, plan: Plan, inp, out) -> int:
        """Returns the ticket; raises MgtError (MGT_EAGAIN when the queue is full)."""
        check_arrays(plan, inp, out, device=True)
        xi = XcsrIn(*[_ptr(t) for t in inp])
        xo = XcsrOut(*[_ptr(t) for t in out])
        t = ctypes.c_uint64()
        _check(_load().mgt_submit(self.handle, plan.handle, ctypes.byref(xi), ctypes.byref(xo),
                                  ctypes.byref(t)), "mgt_submit")
        self._live[int(t.value)] = (plan, inp, out)
        return int(t.value)

    def poll(self, ticket: int):
        """(done, status, latency_ms); a finished ticket is released."""
        d, st, lat = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _check(_load().mgt_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(d), ctypes.byref(st),
                                ctypes.byref(lat)), "mgt_poll")
        if d.value:
            self._live.pop(ticket, None)
            return True, int(st.value), float(lat.value)
        return False, None, None

    def drain(self):
        _check(_load().mgt_server_drain(self.handle), "mgt_server_drain")

    def stats(self) -> dict:
        st = ServerStats()
        _check(_load().mgt_server_get_stats(self.handle, ctypes.byref(st)), "mgt_server_get_stats")
        return st.as_dict()

    def reset_stats(self):
        _check(_load().mgt_server_reset_stats(self.handle), "mgt_server_reset_stats")

    def close(self):
        if getattr(self, "handle", None):
            _load().mgt_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def transpose_batched_profiled(plans, inps, outs, workspace, events, stream=None):
    """As transpose_batched(); ``events``: torch.cuda.Event list (>= phases + 2):
    events[0] first, events[1] after zeroing, events[i + 2] after phase i."""
    n = len(plans)
    arr = (ctypes.c_void_p * n)(*[p.handle for p in plans])
    xi = (XcsrIn * n)(*[XcsrIn(*[_ptr(t) for t in i]) for i in inps])
    xo = (XcsrOut * n)(*[XcsrOut(*[_ptr(t) for t in o]) for o in outs])
    for e in events:
        if not e.cuda_event:
            e.record(stream)
    ev = (ctypes.c_void_p * len(events))(*[ctypes.c_void_p(e.cuda_event) for e in events])
    rc = _load().mgt_transpose_batched_profiled(n, arr, xi, xo, _ptr(workspace),
                                                workspace.numel() * workspace.element_size(),
                                                _stream_handle(stream), ev, len(events))
    _check(rc, "mgt_transpose_batched_profiled")


class _DescOnly:
    """A descriptor standing in for a plan in check_arrays."""

    def __init__(self, desc):
        self.desc = desc


def transpose_static(x, inp, out, stream=None):
    """The allocation-free entry point (scratch in the library's fixed device
    array).  ``x`` supplies the sizes (an XCSR-like object); inp/out as for
    transpose()."""
    part_off = x.part_off if (x.part_off is not None and len(x.part_off) > 2) else None
    desc, keep = make_desc(x.n_rows, x.n_cols, x.n_cells, x.n_values, x.offset_bytes, x.stride,
                           part_off)
    check_arrays(_DescOnly(desc), inp, out, device=True)
    xi = XcsrIn(*[_ptr(t) for t in inp])
    xo = XcsrOut(*[_ptr(t) for t in out])
    rc = _load().mgt_transpose_static(ctypes.byref(desc), ctypes.byref(xi), ctypes.byref(xo),
                                      _stream_handle(stream))
    del keep
    _check(rc, "mgt_transpose_static")


def static_status(stream=None) -> int:
    return int(_load().mgt_static_status(_stream_handle(stream)))


def probe_runs(mode: int, src, dst, perm, n_runs: int, run_bytes: int, stream=None):
    """Enqueues the memory-system probe (mgt_probe_runs): mode 0 gather, 1
    scatter, 2 random 4-byte writes, 3 sequential copy, 4 gather staged in
    shared memory with cp.async, 5 gather through TMA bulk copies, of
    ``n_runs`` runs of ``run_bytes`` bytes; ``perm`` a device uint32/int32
    permutation of [0, n_runs)."""
    need = n_runs * (4 if mode == 2 else run_bytes)
    if _nbytes(dst) < need or (mode != 2 and _nbytes(src) < n_runs * run_bytes):
        raise ValueError("probe buffers smaller than n_runs * run_bytes")
    if mode in (0, 1, 2, 4, 5) and (perm is None or perm.numel() < n_runs or perm.element_size() != 4):
        raise ValueError("probe permutation must hold n_runs 4-byte entries")
    _check(_load().mgt_probe_runs(int(mode), _ptr(src), _ptr(dst), _ptr(perm), int(n_runs),
                                  int(run_bytes), _stream_handle(stream)), "mgt_probe_runs")


def probe_errors() -> int:
    """Waits of probe mode 5 that ran out of polls (mgt_probe_errors)."""
    n = ctypes.c_uint32(0)
    _check(_load().mgt_probe_errors(ctypes.byref(n)), "mgt_probe_errors")
    return int(n.value)


def l2_fetch_granularity(set_bytes: int = -1) -> int:
    """The current context's L2 fetch granularity hint before the call
    (mgt_l2_fetch_granularity); ``set_bytes`` >= 0 sets a new one."""
    prev = ctypes.c_int32(0)
    _check(_load().mgt_l2_fetch_granularity(int(set_bytes), ctypes.byref(prev)), "mgt_l2_fetch_granularity")
    return int(prev.value)


def version() -> str:
    return _load().mgt_version().decode()


def strerror(code: int) -> str:
    return _load().mgt_strerror(code).decode()


# ------------------------------------------------------------ tensor helpers
@dataclasses.dataclass
class DeviceXCSR:
    """An XCSR matrix whose arrays live in GPU memory (torch tensors)."""
    n_rows: int
    n_cols: int
    offset_bytes: int
    stride: int
    row_ptr: object
    col_idx: object
    cell_ptr: object
    values: object   # uint8, n_values * stride bytes
    part_off: np.ndarray

    @property
    def n_cells(self) -> int:
        return int(self.col_idx.numel())

    @property
    def n_values(self) -> int:
        return int(self.values.numel() // self.stride)

    def arrays(self):
        return (self.row_ptr, self.col_idx, self.cell_ptr, self.values)


def to_device(x, device="cuda", pin=False):
    """Copies a host XCSR (numpy arrays) to the GPU."""
    import torch

    def t(a):
        h = torch.from_numpy(np.ascontiguousarray(a))
        if pin:
            h = h.pin_memory()
        return h.to(device, non_blocking=pin)

    return DeviceXCSR(x.n_rows, x.n_cols, x.offset_bytes, x.stride, t(x.row_ptr), t(x.col_idx),
                      t(x.cell_ptr), t(x.values), np.asarray(x.part_off, dtype=np.int64))


@dataclasses.dataclass
class DeviceVarXCSR:
    """A matrix with variable-width values in GPU memory (torch tensors):
    val_off holds the int64 byte offsets of the values, values the bytes."""
    n_rows: int
    n_cols: int
    offset_bytes: int
    row_ptr: object
    col_idx: object
    cell_ptr: object
    val_off: object
    values: object
    part_off: np.ndarray

    @property
    def n_cells(self) -> int:
        return int(self.col_idx.numel())

    @property
    def n_values(self) -> int:
        return int(self.val_off.numel() - 1)

    def arrays(self):
        return (self.row_ptr, self.col_idx, self.cell_ptr, self.values)


def to_device_var(x, device="cuda"):
    """Copies a host VarXCSR (numpy arrays) to the GPU."""
    import torch

    def t(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(device)

    return DeviceVarXCSR(x.n_rows, x.n_cols, x.offset_bytes, t(x.row_ptr), t(x.col_idx),
                         t(x.cell_ptr), t(x.val_off), t(x.values), np.asarray(x.part_off, np.int64))


def plan_for_var(x, cfg=None, with_parts=True) -> Plan:
    """Plan for a matrix with variable-width values (VarXCSR or DeviceVarXCSR)."""
    return Plan(x.n_rows, x.n_cols, x.n_cells, x.n_values, x.offset_bytes, 1,
                x.part_off if (with_parts and x.part_off is not None and len(x.part_off) > 2) else None,
                cfg, var_width=True)


def alloc_output_var(x, device="cuda", parts=True):
    """The transposed variable-width matrix's arrays: (row_ptr, col_idx,
    cell_ptr, value bytes, part_cells, part_values) and the value offsets."""
    import torch
    odt = torch.int32 if x.offset_bytes == 4 else torch.int64
    P = len(x.part_off) - 1 if x.part_off is not None else 1
    out = (torch.empty(x.n_cols + 1, dtype=odt, device=device),
           torch.empty(x.n_cells, dtype=torch.int32, device=device),
           torch.empty(x.n_cells + 1, dtype=odt, device=device),
           torch.empty(int(x.values.numel()) if hasattr(x.values, "numel") else len(x.values),
                       dtype=torch.uint8, device=device),
           torch.empty(P * P, dtype=torch.int64, device=device) if parts else None,
           torch.empty(P * P, dtype=torch.int64, device=device) if parts else None)
    return out, torch.empty(x.n_values + 1, dtype=torch.int64, device=device)


def plan_for(x, cfg=None, with_parts=True) -> Plan:
    return Plan(x.n_rows, x.n_cols, x.n_cells, x.n_values, x.offset_bytes, x.stride,
                x.part_off if (with_parts and x.part_off is not None and len(x.part_off) > 2) else None,
                cfg)


def alloc_output(x, device="cuda", parts=True):
    """Allocates the transposed matrix's arrays (same sizes; n_cols + 1 row pointers)."""
    import torch
    odt = torch.int32 if x.offset_bytes == 4 else torch.int64
    P = len(x.part_off) - 1 if x.part_off is not None else 1
    out = (torch.empty(x.n_cols + 1, dtype=odt, device=device),
           torch.empty(x.n_cells, dtype=torch.int32, device=device),
           torch.empty(x.n_cells + 1, dtype=odt, device=device),
           torch.empty(x.n_values * x.stride, dtype=torch.uint8, device=device),
           torch.empty(P * P, dtype=torch.int64, device=device) if parts else None,
           torch.empty(P * P, dtype=torch.int64, device=device) if parts else None)
    return out


def alloc_workspace(nbytes: int, device="cuda"):
    import torch
    return torch.empty(max(256, (nbytes + 255) // 256 * 256), dtype=torch.uint8, device=device)


def transpose_device(x: DeviceXCSR, plan: Plan | None = None, workspace=None, out=None,
                     stream=None, check=True):
    """Allocates what is missing, transposes, optionally checks the status.
    Returns (out tuple, plan, workspace)."""
    plan = plan or plan_for(x)
    workspace = workspace if workspace is not None else alloc_workspace(plan.workspace_bytes)
    out = out or alloc_output(x, parts=True)
    transpose(plan, x.arrays(), out, workspace, stream)
    if check:
        rc = read_status(workspace, stream)
        _check(rc, "device status")
    return out, plan, workspace
