"""ORACLE -- test infrastructure only.

A plain, slow, obviously correct CPU implementation of the transposition of a
multigraph / high-cardinality sparse matrix in XCSR (the paper's Sec. 2
definition M^T_ij = M_ji applied to cells that hold value lists).  Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's ``cpu_baseline`` /
reference leg may import it.  It shares no code with the CUDA path.

* ``transpose``  -- the counting transpose in ``xcsr_oracle.c`` (plain C, one
  thread): full output plus the P x P cell and value counts.
* ``degrees``    -- column degrees (row_ptr' is their exclusive prefix).
* ``rows``       -- selected output rows computed one by one from the
  definition, for checks at sizes where the full oracle is too slow.
* ``literal``    -- a second restatement that follows the paper's own steps
  (LocalTranspose, then the two view-swap exchanges, Sec. 3), in numpy.
* ``transpose_var`` -- the same transpose for values of individual byte
  widths (the paper's heterogeneous-datatype variant, Sec. 2, MPI_Alltoallw):
  the counting transpose of the cells, then every value moved with its own
  size, one at a time in output order.

Pins (tests/test_oracle_pins.py) tie it to facts other than itself: brute
force on tiny dense matrices, numpy's stable argsort and bincount, scipy's
CSR transpose for single-value cells, involution (12 chained transposes),
P-invariance, tuple-multiset preservation and closed forms of the workloads.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xcsr_oracle.c")
_lock = threading.Lock()
_libs: dict = {}

XO_OK, XO_EINVAL, XO_ENOMEM, XO_EBADINPUT = 0, -1, -2, -3


def lib_path(mutant: int = 0) -> str:
    return os.path.join(_HERE, "libxcsr_oracle.so" if mutant == 0 else f"libxcsr_oracle_m{mutant}.so")


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle with gcc.  ``mutant > 0`` plants one known mistake
    (used only by the pin-strength test)."""
    path = lib_path(mutant)
    with _lock:
        if (not force and os.path.exists(path)
                and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
            return path
        tmp = path + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared",
                               f"-DXO_MUTANT={int(mutant)}", "-o", tmp, _SRC])
        os.replace(tmp, path)
        return path


def _load(mutant: int = 0):
    if mutant not in _libs:
        lib = ctypes.CDLL(build(mutant))
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.xo_validate.argtypes = [i64, i64, i64, i64, i32, i32, vp, vp, vp, i64, vp]
        lib.xo_validate.restype = i32
        lib.xo_transpose.argtypes = [i64, i64, i64, i64, i32, i32, vp, vp, vp, vp, i64, vp,
                                     vp, vp, vp, vp, vp, vp, vp]
        lib.xo_transpose.restype = i32
        lib.xo_degrees.argtypes = [i64, vp, i64, vp]
        lib.xo_degrees.restype = i32
        lib.xo_rows.argtypes = [i64, i64, i32, i32, vp, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp]
        lib.xo_rows.restype = i32
        lib.xo_transpose_var.argtypes = [i64, i64, i64, i64, i32, vp, vp, vp, vp, vp,
                                         vp, vp, vp, vp, vp]
        lib.xo_transpose_var.restype = i32
        _libs[mutant] = lib
    return _libs[mutant]


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle rejected the input (code {code})")
        self.code = code


@dataclasses.dataclass
class Transposed:
    row_ptr: np.ndarray
    col_idx: np.ndarray
    cell_ptr: np.ndarray
    values: np.ndarray
    src: np.ndarray
    part_cells: np.ndarray
    part_values: np.ndarray


def _p(a):
    return a.ctypes.data if a is not None and a.size else None


def validate(x) -> int:
    return _load().xo_validate(x.n_rows, x.n_cols, x.n_cells, x.n_values, x.offset_bytes, x.stride,
                               _p(x.row_ptr), _p(x.col_idx), _p(x.cell_ptr), x.n_parts,
                               _p(x.part_off))


def transpose(x, part_off=None, mutant: int = 0) -> Transposed:
    """Transpose XCSR ``x`` (a ``synth.XCSR``-like object).  ``part_off``
    overrides the row blocks used for the P x P counts."""
    off = np.ascontiguousarray(x.part_off if part_off is None else part_off, dtype=np.int64)
    P = off.shape[0] - 1
    o = x.offset_bytes
    odt = np.int32 if o == 4 else np.int64
    C, V, N = x.n_cells, x.n_values, x.n_cols
    t_row = np.zeros(N + 1, dtype=odt)
    t_col = np.zeros(C, dtype=np.int32)
    t_cp = np.zeros(C + 1, dtype=odt)
    t_val = np.zeros(V * x.stride, dtype=np.uint8)
    src = np.zeros(C, dtype=np.int64)
    pc = np.zeros(P * P, dtype=np.int64)
    pv = np.zeros(P * P, dtype=np.int64)
    rc = _load(mutant).xo_transpose(x.n_rows, N, C, V, o, x.stride, _p(x.row_ptr), _p(x.col_idx),
                                    _p(x.cell_ptr), _p(x.values), P, _p(off), _p(t_row), _p(t_col),
                                    _p(t_cp), _p(t_val), _p(src), _p(pc), _p(pv))
    if rc != XO_OK:
        raise OracleError(rc)
    return Transposed(t_row, t_col, t_cp, t_val, src, pc.reshape(P, P), pv.reshape(P, P))


def as_xcsr(t: Transposed, x):
    """The transposed matrix as an XCSR of the same kind as ``x`` (for chains)."""
    import synth
    return synth.XCSR(x.n_cols, x.n_rows, x.offset_bytes, x.stride, t.row_ptr, t.col_idx,
                      t.cell_ptr, t.values, x.part_off.copy())


def degrees(x) -> np.ndarray:
    deg = np.zeros(x.n_cols, dtype=np.int64)
    rc = _load().xo_degrees(x.n_cells, _p(x.col_idx), x.n_cols, _p(deg))
    if rc != XO_OK:
        raise OracleError(rc)
    return deg


def rows(x, sel):
    """Output rows ``sel`` (strictly ascending column ids) from the definition.
    Returns (cnt[m], t_col, t_len, t_values) with the rows back to back."""
    sel = np.ascontiguousarray(sel, dtype=np.int64)
    m = sel.shape[0]
    cnt = np.zeros(m, dtype=np.int64)
    vcnt = np.zeros(m, dtype=np.int64)
    lib = _load()
    args = (x.n_rows, x.n_cells, x.offset_bytes, x.stride, _p(x.row_ptr), _p(x.col_idx),
            _p(x.cell_ptr), _p(x.values), m, _p(sel), _p(cnt), _p(vcnt))
    rc = lib.xo_rows(*args, None, None, None)
    if rc != XO_OK:
        raise OracleError(rc)
    t_col = np.zeros(int(cnt.sum()), dtype=np.int32)
    t_len = np.zeros(int(cnt.sum()), dtype=np.int64)
    t_val = np.zeros(int(vcnt.sum()) * x.stride, dtype=np.uint8)
    rc = lib.xo_rows(*args, _p(t_col), _p(t_len), _p(t_val))
    if rc != XO_OK:
        raise OracleError(rc)
    return cnt, t_col, t_len, t_val


@dataclasses.dataclass
class TransposedVar:
    row_ptr: np.ndarray
    col_idx: np.ndarray
    cell_ptr: np.ndarray
    val_off: np.ndarray
    values: np.ndarray


def transpose_var(x, mutant: int = 0) -> TransposedVar:
    """Transpose a matrix whose values have individual byte widths (a
    ``synth.VarXCSR``-like object: val_off[V+1] byte offsets, values bytes)."""
    o = x.offset_bytes
    odt = np.int32 if o == 4 else np.int64
    C, V, N = x.n_cells, x.n_values, x.n_cols
    B = int(x.val_off[-1]) if V >= 0 and x.val_off.shape[0] else 0
    t_row = np.zeros(N + 1, dtype=odt)
    t_col = np.zeros(C, dtype=np.int32)
    t_cp = np.zeros(C + 1, dtype=odt)
    t_vo = np.zeros(V + 1, dtype=np.int64)
    t_val = np.zeros(B, dtype=np.uint8)
    rc = _load(mutant).xo_transpose_var(x.n_rows, N, C, V, o, _p(x.row_ptr), _p(x.col_idx),
                                        _p(x.cell_ptr), _p(x.val_off), _p(x.values), _p(t_row),
                                        _p(t_col), _p(t_cp), _p(t_vo), _p(t_val))
    if rc != XO_OK:
        raise OracleError(rc)
    return TransposedVar(t_row, t_col, t_cp, t_vo, t_val)


def as_var_xcsr(t: TransposedVar, x):
    """The transposed variable-width matrix as a VarXCSR (for chains)."""
    import synth
    return synth.VarXCSR(x.n_cols, x.n_rows, x.offset_bytes, t.row_ptr, t.col_idx, t.cell_ptr,
                         t.val_off, t.values, x.part_off.copy())
