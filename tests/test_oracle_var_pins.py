"""Pins of the oracle's variable-width transpose (the paper's
heterogeneous-datatype variant, Sec. 2: one datatype per edge through
MPI_Alltoallw), to facts other than itself (no GPU needed).

Each pin is a function of a transpose routine ``T(x)``; the same pins run
against copies of the oracle with one planted mistake each (values sized by
their neighbour; values left at their input byte offsets), and every planted
mistake must fail at least one pin.
"""
from __future__ import annotations

import collections

import numpy as np
import pytest

import oracle
import synth
from helpers import (random_small, random_small_var, same_var, var_brute_force_dense,
                     var_cells_of)


def pin_var_brute_force_dense(T):
    """Dense transposition of an R x N array of lists of byte strings of
    mixed widths (zero and odd widths included)."""
    for seed, (R, N) in enumerate([(1, 1), (3, 5), (7, 2), (12, 12), (30, 17), (40, 40)]):
        for o in (4, 8):
            x = random_small_var(seed, R, N, offset_bytes=o)
            assert same_var(T(x), *var_brute_force_dense(x))


def pin_var_equal_widths_reduce_to_fixed(T):
    """All values of one width s: the result is the fixed-width transpose
    (the MPI_BYTE serialisation of Sec. 2, pinned on its own) with byte
    offsets s * p."""
    for seed, s in ((1, 4), (2, 8), (3, 12), (4, 32)):
        x = random_small(50 + seed, 60, 45, max_cells=8, max_len=5, stride=s, n_parts=1)
        V = x.n_values
        xv = synth.var_from_arrays(x.row_ptr, x.col_idx, x.cell_ptr,
                                   s * np.arange(V + 1, dtype=np.int64), x.values, x.n_cols)
        t, f = T(xv), oracle.transpose(x)
        assert np.array_equal(t.row_ptr, f.row_ptr)
        assert np.array_equal(t.col_idx, f.col_idx)
        assert np.array_equal(t.cell_ptr, f.cell_ptr)
        assert np.array_equal(t.val_off, s * np.arange(V + 1, dtype=np.int64))
        assert np.array_equal(t.values, f.values)


def pin_var_involution_chain(T):
    """Twelve chained transposes of a matrix with ascending columns per row
    give it back byte for byte (involution, Sec. 3; the paper chains 12)."""
    x = synth.generate_var(synth.heterogeneous(seed=6, n=300, parts=1))
    y = x
    for _ in range(12):
        y = oracle.as_var_xcsr(T(y), y)
    for a, b in ((y.row_ptr, x.row_ptr), (y.col_idx, x.col_idx), (y.cell_ptr, x.cell_ptr),
                 (y.val_off, x.val_off), (y.values, x.values)):
        assert np.array_equal(a, b)


def pin_var_tuple_multiset(T):
    """Every edge {i, j, e} becomes {j, i, e} (Sec. 2): the multiset of
    (row, column, list of value byte strings) maps to (column, row, same)."""
    x = random_small_var(9, 50, 50, max_cells=10, max_len=6, sorted_rows=False, dup_cols=True)
    t = oracle.as_var_xcsr(T(x), x)
    before = collections.Counter((j, i, run) for (i, j, run) in var_cells_of(x))
    after = collections.Counter(var_cells_of(t))
    assert before == after


def pin_var_sizes_follow_stable_argsort(T):
    """Output value sizes are the input sizes taken cell by cell in numpy's
    stable argsort order of the column ids, each cell's values in order."""
    x = random_small_var(12, 80, 33, max_cells=9, max_len=7, sorted_rows=False, dup_cols=True)
    t = T(x)
    order = np.argsort(x.col_idx, kind="stable")
    sizes = np.diff(x.val_off)
    want = [sizes[int(x.cell_ptr[k]):int(x.cell_ptr[k + 1])] for k in order]
    want = np.concatenate(want) if want else np.zeros(0, np.int64)
    assert np.array_equal(np.diff(t.val_off), want)
    assert t.val_off[-1] == x.val_off[-1]


def pin_var_edge_cases(T):
    """Empty matrix, only zero-width values, one long cell, empty rows and
    columns."""
    e = synth.var_from_arrays(np.zeros(4, np.int64), np.zeros(0, np.int32), np.zeros(1, np.int64),
                              np.zeros(1, np.int64), np.zeros(0, np.uint8), 3)
    t = T(e)
    assert np.array_equal(t.row_ptr, np.zeros(4, np.int64)) and t.val_off.tolist() == [0]
    z = synth.var_from_arrays([0, 2, 2], [1, 0], [0, 3, 5], np.zeros(6, np.int64),
                              np.zeros(0, np.uint8), 2)
    t = T(z)
    assert t.col_idx.tolist() == [0, 0] and t.cell_ptr.tolist() == [0, 2, 5]
    assert t.val_off.tolist() == [0] * 6
    vals = np.arange(1, 46, dtype=np.uint8)
    one = synth.var_from_arrays([0, 0, 1], [0], [0, 9], np.array([0, 1, 3, 6, 10, 15, 21, 28, 36, 45]),
                                vals, 4)
    t = T(one)
    assert t.row_ptr.tolist() == [0, 1, 1, 1, 1] and t.col_idx.tolist() == [1]
    assert t.val_off.tolist() == [0, 1, 3, 6, 10, 15, 21, 28, 36, 45]
    assert np.array_equal(t.values, vals)


VAR_PINS = [pin_var_brute_force_dense, pin_var_equal_widths_reduce_to_fixed,
            pin_var_involution_chain, pin_var_tuple_multiset, pin_var_sizes_follow_stable_argsort,
            pin_var_edge_cases]


@pytest.mark.parametrize("pin", VAR_PINS, ids=[p.__name__ for p in VAR_PINS])
def test_var_oracle_pin(pin):
    pin(oracle.transpose_var)


@pytest.mark.parametrize("mutant", [6, 7])
def test_var_pins_catch_planted_mistakes(mutant):
    """Each planted mistake (a value sized by its neighbour; values left at
    their input byte offsets) fails at least one pin."""

    def T(x):
        return oracle.transpose_var(x, mutant=mutant)

    failed = []
    for pin in VAR_PINS:
        try:
            pin(T)
        except (AssertionError, oracle.OracleError, ValueError, IndexError):
            failed.append(pin.__name__)
    assert failed, f"planted mistake {mutant} passed every pin"


def test_var_oracle_rejects_malformed():
    x = random_small_var(3, 10, 10)
    bad = synth.var_from_arrays(x.row_ptr, x.col_idx, x.cell_ptr, x.val_off[::-1].copy(),
                                x.values, x.n_cols)
    if x.n_values > 1 and x.val_off[-1] > 0:
        with pytest.raises(oracle.OracleError):
            oracle.transpose_var(bad)


def test_var_generator_widths():
    """Generated widths come from the requested set, independent of thread count."""
    sp = synth.heterogeneous(seed=4, n=3000, parts=1)
    a = synth.generate_var(sp, sizes=(4, 12, 64), nthreads=1)
    b = synth.generate_var(sp, sizes=(4, 12, 64), nthreads=7)
    assert set(np.unique(np.diff(a.val_off)).tolist()) <= {4, 12, 64}
    for f in ("row_ptr", "col_idx", "cell_ptr", "val_off", "values"):
        assert np.array_equal(getattr(a, f), getattr(b, f))
    assert a.n_bytes == int(a.val_off[-1])
