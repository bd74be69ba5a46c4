"""Seeded synthetic XCSR workloads (inputs only; no transposition arithmetic).

The five workloads follow the shapes of the paper's benchmark section (Sec. 4:
a heterogeneous multigraph with variable-length cell runs and a perfectly
balanced one) scaled to one GPU:

* ``tiny``           1,000 x 1,000, 4 equal row blocks, cells/row ~ Poisson(8),
                     run length 1 + Poisson(3), int64 counter payload, int32 offsets.
* ``balanced``       4,194,304 x 4,194,304, exactly 32 distinct uniform columns
                     per row, exactly 4 values per cell, 8-byte random payload,
                     64 equal row blocks, int64 offsets.
* ``heterogeneous``  8,388,608 x 8,388,608, cells/row LogNormal (arithmetic mean
                     20, sigma 1) capped at 4,096, Zipf(1.1) columns without
                     repeats (rank -> column through a seeded bijection), run
                     length Geometric(mean 5) clamped to [1, 64], 32-byte payload
                     of 8 fp32 in [0, 1), 256 row blocks sized by LogNormal(0, 1)
                     weights, int64 offsets.
* ``batched``        per matrix: rows log-uniform in [1e3, 2e6], square,
                     cells/row LogNormal (mean 16, sigma 1), uniform distinct
                     columns, run length Geometric(mean 4) in [1, 64], 16-byte
                     payload (4 x fp32), one partition, int32 offsets.

Every array is a pure function of (workload, seed, index); the C generator in
``synth.c`` is multi-threaded but thread-count independent.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

ROW_EXACT, ROW_POISSON, ROW_LOGNORMAL, ROW_UNIFORM = 0, 1, 2, 3
COL_UNIFORM, COL_ZIPF = 0, 1
LEN_EXACT, LEN_ONE_PLUS_POISSON, LEN_GEOMETRIC, LEN_UNIFORM = 0, 1, 2, 3
PAY_COUNTER, PAY_BITS, PAY_F32, PAY_ID = 0, 1, 2, 3


class _Spec(ctypes.Structure):
    _fields_ = [
        ("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64),
        ("row_dist", ctypes.c_int32), ("row_a", ctypes.c_double), ("row_b", ctypes.c_double),
        ("row_cap", ctypes.c_int64),
        ("col_dist", ctypes.c_int32), ("col_a", ctypes.c_double), ("col_perm", ctypes.c_int32),
        ("len_dist", ctypes.c_int32), ("len_a", ctypes.c_double),
        ("len_min", ctypes.c_int64), ("len_max", ctypes.c_int64),
        ("payload", ctypes.c_int32), ("stride", ctypes.c_int32), ("offset_bytes", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``libsynth.so`` beside it (gcc, no -march)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + ".tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.syn_row_ptr.argtypes = [ctypes.POINTER(_Spec), vp, i32]
        lib.syn_row_ptr.restype = i64
        lib.syn_cells.argtypes = [ctypes.POINTER(_Spec), vp, vp, vp, i32]
        lib.syn_cells.restype = i64
        lib.syn_values.argtypes = [ctypes.POINTER(_Spec), i64, vp, i32]
        lib.syn_values.restype = i32
        lib.syn_partitions.argtypes = [i32, i64, i64, ctypes.c_double, ctypes.c_uint64, vp]
        lib.syn_partitions.restype = i32
        lib.syn_loguniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, i64, i64]
        lib.syn_loguniform.restype = i64
        lib.syn_uniform01.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.syn_uniform01.restype = ctypes.c_double
        lib.syn_key.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.syn_key.restype = ctypes.c_uint64
        lib.syn_perm.argtypes = [ctypes.c_uint64, i64, i64]
        lib.syn_perm.restype = i64
        lib.syn_zipf_sample.argtypes = [ctypes.c_double, i64, ctypes.c_uint64, i64, vp]
        lib.syn_zipf_sample.restype = i64
        lib.syn_widths.argtypes = [ctypes.c_uint64, i64, vp, i32, vp, i32]
        lib.syn_widths.restype = i64
        lib.syn_bytes.argtypes = [ctypes.c_uint64, i64, vp, i32]
        lib.syn_bytes.restype = i32
        _lib = lib
    return _lib


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


@dataclasses.dataclass
class Spec:
    """Distribution parameters of one synthetic XCSR matrix."""
    n_rows: int
    n_cols: int
    row_dist: int = ROW_EXACT
    row_a: float = 0.0
    row_b: float = 0.0
    row_cap: int = 0
    col_dist: int = COL_UNIFORM
    col_a: float = 0.0
    col_perm: int = 1
    len_dist: int = LEN_EXACT
    len_a: float = 1.0
    len_min: int = 0
    len_max: int = -1
    payload: int = PAY_BITS
    stride: int = 8
    offset_bytes: int = 8
    seed: int = 0
    # partitions: (kind, count, sigma); kind 0 = equal blocks, 1 = LogNormal weights
    part_kind: int = 0
    n_parts: int = 1
    part_sigma: float = 1.0

    def c_struct(self) -> _Spec:
        return _Spec(self.n_rows, self.n_cols, self.row_dist, self.row_a, self.row_b, self.row_cap,
                     self.col_dist, self.col_a, self.col_perm, self.len_dist, self.len_a,
                     self.len_min, self.len_max, self.payload, self.stride, self.offset_bytes,
                     ctypes.c_uint64(self.seed & 0xFFFFFFFFFFFFFFFF).value)


@dataclasses.dataclass
class XCSR:
    """A row-major XCSR matrix in host memory (the paper's Sec. 2 format:
    CSR plus a per-cell count of values; here as prefix arrays).

    row_ptr[R+1], cell_ptr[C+1]: offset_bytes-wide ints; col_idx[C]: int32;
    values: V * stride opaque bytes; part_off[P+1]: int64 row-block bounds."""
    n_rows: int
    n_cols: int
    offset_bytes: int
    stride: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    cell_ptr: np.ndarray
    values: np.ndarray
    part_off: np.ndarray

    @property
    def n_cells(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def n_values(self) -> int:
        return int(self.values.shape[0] // self.stride) if self.stride else 0

    @property
    def n_parts(self) -> int:
        return int(self.part_off.shape[0] - 1)

    def minimal_bytes(self) -> int:
        """Input read once plus output written once (both XCSR, same sizes
        except that the output has n_cols + 1 row pointers)."""
        o, C, V, s = self.offset_bytes, self.n_cells, self.n_values, self.stride
        side = 4 * C + (C + 1) * o + V * s
        return (self.n_rows + 1) * o + side + (self.n_cols + 1) * o + side


def _off_dtype(o: int):
    return np.int32 if o == 4 else np.int64


def generate(spec: Spec, *, alloc=None, nthreads: int | None = None) -> XCSR:
    """Draw one matrix.  ``alloc(nbytes) -> writable uint8 numpy array`` lets a
    caller place the arrays (e.g. in pinned memory); default is numpy."""
    lib = _load()
    nt = nthreads or _threads()
    alloc = alloc or (lambda n: np.empty(n, dtype=np.uint8))
    cs = spec.c_struct()
    o = spec.offset_bytes
    odt = _off_dtype(o)
    row_ptr = alloc((spec.n_rows + 1) * o).view(odt)
    C = lib.syn_row_ptr(ctypes.byref(cs), row_ptr.ctypes.data, nt)
    if C < 0:
        raise ValueError(f"synth: row pass failed ({C})")
    col_idx = alloc(max(C, 0) * 4).view(np.int32)
    cell_ptr = alloc((C + 1) * o).view(odt)
    V = lib.syn_cells(ctypes.byref(cs), row_ptr.ctypes.data, col_idx.ctypes.data,
                      cell_ptr.ctypes.data, nt)
    if V < 0:
        raise ValueError(f"synth: cell pass failed ({V})")
    values = alloc(V * spec.stride)
    if lib.syn_values(ctypes.byref(cs), V, values.ctypes.data, nt) != 0:
        raise ValueError("synth: value pass failed")
    part_off = np.empty(spec.n_parts + 1, dtype=np.int64)
    if lib.syn_partitions(spec.part_kind, spec.n_parts, spec.n_rows, spec.part_sigma,
                          ctypes.c_uint64(spec.seed & 0xFFFFFFFFFFFFFFFF).value,
                          part_off.ctypes.data) != 0:
        raise ValueError("synth: partition pass failed")
    return XCSR(spec.n_rows, spec.n_cols, o, spec.stride, row_ptr, col_idx, cell_ptr, values,
                part_off)


# ---------------------------------------------------------------- workloads
def tiny(seed: int = 0, n: int = 1000, parts: int = 4) -> Spec:
    return Spec(n, n, ROW_POISSON, 8.0, 0.0, 0, COL_UNIFORM, 0.0, 0, LEN_ONE_PLUS_POISSON, 3.0,
                1, -1, PAY_COUNTER, 8, 4, seed, 0, parts)


def balanced(seed: int = 0, n: int = 4_194_304, parts: int = 64, cells: int = 32,
             vals: int = 4, stride: int = 8, offset_bytes: int = 8) -> Spec:
    return Spec(n, n, ROW_EXACT, float(cells), 0.0, 0, COL_UNIFORM, 0.0, 0, LEN_EXACT,
                float(vals), 0, -1, PAY_BITS, stride, offset_bytes, seed, 0, parts)


def heterogeneous(seed: int = 0, n: int = 8_388_608, parts: int = 256, perm: int = 1,
                  payload: int = PAY_F32) -> Spec:
    return Spec(n, n, ROW_LOGNORMAL, math.log(20.0) - 0.5, 1.0, 4096, COL_ZIPF, 1.1, perm,
                LEN_GEOMETRIC, 5.0, 1, 64, payload, 32, 8, seed, 1, parts, 1.0)


def paper_balanced(seed: int = 0, n: int = 1_048_576, parts: int = 16) -> Spec:
    """The paper's balanced benchmark shape (Sec. 5): 512 cells per row, each
    a list of 10 integer values (4-byte payload), 65,536 rows per row block."""
    return balanced(seed=seed, n=n, parts=parts, cells=512, vals=10, stride=4, offset_bytes=8)


def paper_heterogeneous(seed: int = 0, rows: int = 64, cols: int = 2_097_152,
                        lo: int = 300_000, hi: int = 1_000_000) -> Spec:
    """The paper's imbalanced benchmark shape (Sec. 5): every row holds
    between 300 thousand and 1 million uniformly distributed columns, each
    cell a list of 128-byte values, 5 per cell on average (geometric, capped
    at 64).  Few rows and many columns, one row block (rectangular)."""
    return Spec(rows, cols, ROW_UNIFORM, float(lo), float(hi), 0, COL_UNIFORM, 0.0, 0,
                LEN_GEOMETRIC, 5.0, 1, 64, PAY_BITS, 128, 8, seed, 0, 1)


def batched_member(seed: int, m: int, rows_lo: int = 1000, rows_hi: int = 2_000_000,
                   payload: int = PAY_F32) -> Spec:
    lib = _load()
    r = int(lib.syn_loguniform(seed & 0xFFFFFFFFFFFFFFFF, 1, m, rows_lo, rows_hi))
    mseed = int(lib.syn_key(seed & 0xFFFFFFFFFFFFFFFF, 7, m))
    return Spec(r, r, ROW_LOGNORMAL, math.log(16.0) - 0.5, 1.0, 0, COL_UNIFORM, 0.0, 0,
                LEN_GEOMETRIC, 4.0, 1, 64, payload, 16, 4, mseed, 0, 1)


def large_member(seed: int, m: int, n: int = 4_194_304) -> Spec:
    """The large requests of the serving mix: heterogeneous distributions."""
    lib = _load()
    mseed = int(lib.syn_key(seed & 0xFFFFFFFFFFFFFFFF, 8, m))
    s = heterogeneous(mseed, n=n, parts=1)
    return s


WORKLOADS = {
    "tiny": tiny,
    "balanced": balanced,
    "heterogeneous": heterogeneous,
    "paper_balanced": paper_balanced,
    "paper_heterogeneous": paper_heterogeneous,
}


def uniform01(seed: int, tag: int, idx: int) -> float:
    return float(_load().syn_uniform01(seed & 0xFFFFFFFFFFFFFFFF, tag, idx))


def zipf_sample(s: float, n: int, seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.int64)
    _load().syn_zipf_sample(s, n, seed & 0xFFFFFFFFFFFFFFFF, count, out.ctypes.data)
    return out


def perm(seed: int, n: int, x: int) -> int:
    return int(_load().syn_perm(seed & 0xFFFFFFFFFFFFFFFF, n, x))


def from_arrays(row_ptr, col_idx, cell_ptr, values, n_cols, stride, part_off=None,
                offset_bytes=None) -> XCSR:
    """Wrap hand-written arrays (small edge cases) as an XCSR."""
    o = offset_bytes or (4 if np.asarray(row_ptr).dtype == np.int32 else 8)
    odt = _off_dtype(o)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=odt)
    cell_ptr = np.ascontiguousarray(cell_ptr, dtype=odt)
    col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
    values = np.ascontiguousarray(values).view(np.uint8).reshape(-1)
    R = row_ptr.shape[0] - 1
    if part_off is None:
        part_off = np.array([0, R], dtype=np.int64)
    return XCSR(R, int(n_cols), o, int(stride), row_ptr, col_idx, cell_ptr, values,
                np.ascontiguousarray(part_off, dtype=np.int64))


# ------------------------------------------------ variable-width values
# The paper's heterogeneous-datatype variant (Sec. 2, one datatype per edge
# through MPI_Alltoallw): every value has a byte width of its own; value v
# occupies bytes [val_off[v], val_off[v + 1]) of ``values``.
TYPE_SIZES = (4, 8, 12, 16, 24, 32, 48, 64)  # int, double, vec3f, ... 16 doubles


@dataclasses.dataclass
class VarXCSR:
    """A row-major XCSR matrix whose values have individual byte widths:
    row_ptr[R+1], cell_ptr[C+1] (offset_bytes wide), col_idx[C] (int32),
    val_off[V+1] (int64 byte offsets), values (val_off[V] bytes),
    part_off[P+1]."""
    n_rows: int
    n_cols: int
    offset_bytes: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    cell_ptr: np.ndarray
    val_off: np.ndarray
    values: np.ndarray
    part_off: np.ndarray

    @property
    def n_cells(self) -> int:
        return int(self.col_idx.shape[0])

    @property
    def n_values(self) -> int:
        return int(self.val_off.shape[0] - 1)

    @property
    def n_bytes(self) -> int:
        return int(self.values.shape[0])

    @property
    def n_parts(self) -> int:
        return int(self.part_off.shape[0] - 1)

    def minimal_bytes(self) -> int:
        """Input read once plus output written once: the four XCSR arrays and
        the value offsets on each side."""
        o, C, V, B = self.offset_bytes, self.n_cells, self.n_values, self.n_bytes
        side = 4 * C + (C + 1) * o + 8 * (V + 1) + B
        return (self.n_rows + 1) * o + side + (self.n_cols + 1) * o + side


def generate_var(spec: Spec, sizes=TYPE_SIZES, *, alloc=None, nthreads: int | None = None) -> VarXCSR:
    """Draw the matrix structure of ``spec`` (rows, columns, run lengths and
    row blocks as generate() draws them) and give every value a width drawn
    uniformly from ``sizes`` (bytes, each >= 0) and random bytes."""
    lib = _load()
    nt = nthreads or _threads()
    alloc = alloc or (lambda n: np.empty(n, dtype=np.uint8))
    cs = spec.c_struct()
    o = spec.offset_bytes
    odt = _off_dtype(o)
    row_ptr = alloc((spec.n_rows + 1) * o).view(odt)
    C = lib.syn_row_ptr(ctypes.byref(cs), row_ptr.ctypes.data, nt)
    if C < 0:
        raise ValueError(f"synth: row pass failed ({C})")
    col_idx = alloc(max(C, 0) * 4).view(np.int32)
    cell_ptr = alloc((C + 1) * o).view(odt)
    V = lib.syn_cells(ctypes.byref(cs), row_ptr.ctypes.data, col_idx.ctypes.data,
                      cell_ptr.ctypes.data, nt)
    if V < 0:
        raise ValueError(f"synth: cell pass failed ({V})")
    sz = np.ascontiguousarray(sizes, dtype=np.int32)
    val_off = alloc((V + 1) * 8).view(np.int64)
    key = ctypes.c_uint64(spec.seed & 0xFFFFFFFFFFFFFFFF).value
    nb = lib.syn_widths(key, V, sz.ctypes.data, int(sz.shape[0]), val_off.ctypes.data, nt)
    if nb < 0:
        raise ValueError("synth: width pass failed")
    values = alloc(max(nb, 0))
    if lib.syn_bytes(key, nb, values.ctypes.data if nb else None, nt) != 0:
        raise ValueError("synth: byte pass failed")
    part_off = np.empty(spec.n_parts + 1, dtype=np.int64)
    if lib.syn_partitions(spec.part_kind, spec.n_parts, spec.n_rows, spec.part_sigma, key,
                          part_off.ctypes.data) != 0:
        raise ValueError("synth: partition pass failed")
    return VarXCSR(spec.n_rows, spec.n_cols, o, row_ptr, col_idx, cell_ptr, val_off, values, part_off)


def var_from_arrays(row_ptr, col_idx, cell_ptr, val_off, values, n_cols, part_off=None,
                    offset_bytes=None) -> VarXCSR:
    """Wrap hand-written arrays (small edge cases) as a VarXCSR."""
    o = offset_bytes or (4 if np.asarray(row_ptr).dtype == np.int32 else 8)
    odt = _off_dtype(o)
    row_ptr = np.ascontiguousarray(row_ptr, dtype=odt)
    R = row_ptr.shape[0] - 1
    if part_off is None:
        part_off = np.array([0, R], dtype=np.int64)
    return VarXCSR(R, int(n_cols), o, row_ptr, np.ascontiguousarray(col_idx, dtype=np.int32),
                   np.ascontiguousarray(cell_ptr, dtype=odt),
                   np.ascontiguousarray(val_off, dtype=np.int64),
                   np.ascontiguousarray(values).view(np.uint8).reshape(-1),
                   np.ascontiguousarray(part_off, dtype=np.int64))
