"""Pins of the CPU oracle to facts other than itself (no GPU needed).

Each pin is a function of a transpose routine ``T(x, part_off=None)`` so the
same pins run against the oracle and, in ``test_pins_catch_planted_mistakes``,
against copies of the oracle with one planted mistake each: every planted
mistake must fail at least one pin.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from oracle import literal
from helpers import (brute_force_dense, cells_of, parse_golden, random_small, same_xcsr,
                     sorted_rows_copy)

scipy_sparse = pytest.importorskip("scipy.sparse")


# ----------------------------------------------------------------------- pins
def pin_hand_example(T):
    """Hand-worked 4-vertex multigraph (tests/golden/hand_4x4.txt, derived
    from the definition of Sec. 2)."""
    x, (rp, ci, cp, vals) = parse_golden("hand_4x4.txt")
    t = T(x)
    assert same_xcsr(t.row_ptr, t.col_idx, t.cell_ptr, t.values, rp, ci, cp, vals)


def pin_brute_force_dense(T):
    """Dense transposition of an R x N array of value lists (Sec. 2: M^T_ij = M_ji)."""
    for seed, (R, N) in enumerate([(1, 1), (3, 5), (7, 2), (12, 12), (30, 17), (40, 40)]):
        for o in (4, 8):
            x = random_small(seed, R, N, offset_bytes=o, stride=4 * (1 + seed % 3))
            t = T(x)
            assert same_xcsr(t.row_ptr, t.col_idx, t.cell_ptr, t.values, *brute_force_dense(x))


def pin_stable_argsort_and_bincount(T):
    """Output order = numpy's stable argsort of the column ids; degrees =
    bincount (the counting-sort special case, Gustavson 1978)."""
    x = synth.generate(synth.tiny(seed=3, n=300))
    t = T(x)
    order = np.argsort(x.col_idx, kind="stable")
    assert np.array_equal(t.src, order)
    deg = np.bincount(x.col_idx, minlength=x.n_cols)
    assert np.array_equal(np.diff(t.row_ptr.astype(np.int64)), deg)
    rows_of = np.repeat(np.arange(x.n_rows), np.diff(x.row_ptr.astype(np.int64)))
    assert np.array_equal(t.col_idx, rows_of[order])


def pin_scipy_single_value(T):
    """One value per cell reduces XCSR to CSR (Sec. 3 remark on the
    single-value case): compare with scipy's CSR transpose."""
    rng = np.random.default_rng(11)
    R, N, nnz = 57, 41, 400
    dense = np.zeros((R, N), dtype=np.int64)
    flat = rng.choice(R * N, size=nnz, replace=False)
    dense.flat[flat] = rng.integers(1, 1 << 40, size=nnz)
    m = scipy_sparse.csr_matrix(dense)
    m.sort_indices()
    x = synth.from_arrays(m.indptr.astype(np.int64), m.indices, np.arange(m.nnz + 1),
                          m.data.astype(np.int64).view(np.uint8), N, 8)
    t = T(x)
    mt = scipy_sparse.csr_matrix(m.T)
    mt.sort_indices()
    assert np.array_equal(t.row_ptr, mt.indptr)
    assert np.array_equal(t.col_idx, mt.indices)
    assert np.array_equal(t.cell_ptr, np.arange(m.nnz + 1))
    assert np.array_equal(t.values.view(np.int64), mt.data.astype(np.int64))


def pin_involution_chain(T):
    """Twelve chained transposes give the input back (the paper's own
    benchmark chains 12 transposes, Sec. 4; involution, Sec. 3)."""
    x = synth.generate(synth.tiny(seed=5, n=200))
    y = x
    for _ in range(12):
        y = oracle.as_xcsr(T(y), y) if T is oracle.transpose else _wrap(T(y), y)
    assert same_xcsr(y.row_ptr, y.col_idx, y.cell_ptr, y.values,
                     x.row_ptr, x.col_idx, x.cell_ptr, x.values)


def _wrap(t, x):
    return synth.XCSR(x.n_cols, x.n_rows, x.offset_bytes, x.stride, t.row_ptr, t.col_idx,
                      t.cell_ptr, t.values, x.part_off.copy())


def pin_unsorted_rows_double_transpose(T):
    """With unsorted rows, T(T(M)) is M with each row sorted by column."""
    x = random_small(21, 25, 25, sorted_rows=False, max_cells=8)
    y = _wrap(T(_wrap(T(x), x)), x)
    z = sorted_rows_copy(x)
    assert same_xcsr(y.row_ptr, y.col_idx, y.cell_ptr, y.values,
                     z.row_ptr, z.col_idx, z.cell_ptr, z.values)


def pin_literal_and_partition_invariance(T):
    """LocalTranspose then ViewSwap (Sec. 3, Eqs. 3-4) for P ranks equals the
    transpose for every P, and the P x P counts are the metadata/value count
    matrices the view swap exchanges."""
    x = random_small(7, 24, 24, max_cells=7)
    ref = None
    for P in (1, 2, 3, 4, 24):
        off = np.asarray([(d * 24) // P for d in range(P + 1)], dtype=np.int64)
        t = T(x, off)
        lr, lc, lcp, lv, lpc, lpv = literal.transpose(x, off)
        assert same_xcsr(t.row_ptr, t.col_idx, t.cell_ptr, t.values, lr, lc, lcp, lv)
        assert np.array_equal(t.part_cells, lpc)
        assert np.array_equal(t.part_values, lpv)
        if ref is None:
            ref = t
        assert same_xcsr(t.row_ptr, t.col_idx, t.cell_ptr, t.values,
                         ref.row_ptr, ref.col_idx, ref.cell_ptr, ref.values)


def pin_tuple_multiset(T):
    """E* = {{j, i, e}} for all {i, j, e} in E (Sec. 2): the multiset of
    (row, column, run) tuples maps to (column, row, run)."""
    x = synth.generate(synth.heterogeneous(seed=2, n=2048, parts=8))
    t = _wrap(T(x), x)
    a = sorted((j, i, run) for (i, j, run) in cells_of(x))
    b = sorted(cells_of(t))
    assert a == b


def pin_degree_and_partition_sums(T):
    """Degree sums; P x P row sums are the source blocks' cells and values,
    column sums the destination blocks' (cover and disjointness, Sec. 2)."""
    x = synth.generate(synth.heterogeneous(seed=4, n=4096, parts=16))
    t = T(x)
    C, V = x.n_cells, x.n_values
    assert int(t.row_ptr[-1]) == C and int(t.cell_ptr[-1]) == V
    rp = x.row_ptr.astype(np.int64)
    cp = x.cell_ptr.astype(np.int64)
    off = x.part_off
    for s in range(x.n_parts):
        k0, k1 = rp[off[s]], rp[off[s + 1]]
        assert t.part_cells[s].sum() == k1 - k0
        assert t.part_values[s].sum() == cp[k1] - cp[k0]
    trp = t.row_ptr.astype(np.int64)
    tcp = t.cell_ptr.astype(np.int64)
    for d in range(x.n_parts):
        q0, q1 = trp[off[d]], trp[off[d + 1]]
        assert t.part_cells[:, d].sum() == q1 - q0
        assert t.part_values[:, d].sum() == tcp[q1] - tcp[q0]


def pin_closed_form_balanced(T):
    """Balanced workload: every run has 4 values, so cell_ptr'[q] = 4 q, and
    output rows list strictly ascending source rows."""
    x = synth.generate(synth.balanced(seed=1, n=4096, parts=8))
    t = T(x)
    assert np.array_equal(t.cell_ptr.astype(np.int64), 4 * np.arange(x.n_cells + 1))
    trp = t.row_ptr.astype(np.int64)
    for j in range(0, x.n_cols, 97):
        seg = t.col_idx[trp[j]:trp[j + 1]]
        assert np.all(np.diff(seg) > 0)


def pin_closed_form_counter_payload(T):
    """Tiny workload's payload is a counter: each id appears exactly once in
    the output and ids inside a run stay consecutive and ascending."""
    x = synth.generate(synth.tiny(seed=0))
    t = T(x)
    ids = t.values.view(np.int64)
    base = int(x.values.view(np.int64)[0])
    assert np.array_equal(np.sort(ids), base + np.arange(x.n_values))
    tcp = t.cell_ptr.astype(np.int64)
    for q in range(x.n_cells):
        run = ids[tcp[q]:tcp[q + 1]]
        assert np.all(np.diff(run) == 1)


def pin_edge_cases(T):
    """Empty matrix, empty rows/columns, zero-length runs, one hot column,
    duplicated columns inside a row (kept in input order)."""
    e = synth.from_arrays(np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(1, np.int64),
                          np.zeros(0, np.uint8), 9, 8)
    t = T(e)
    assert np.array_equal(t.row_ptr, np.zeros(10)) and t.col_idx.size == 0
    hot = synth.from_arrays(np.arange(0, 11, dtype=np.int64), np.full(10, 3, np.int32),
                            np.arange(0, 21, 2, dtype=np.int64),
                            np.arange(20, dtype=np.int64).view(np.uint8), 10, 8)
    t = T(hot)
    assert np.array_equal(t.col_idx, np.arange(10))
    assert np.array_equal(t.row_ptr, [0, 0, 0, 0, 10, 10, 10, 10, 10, 10, 10])
    assert np.array_equal(t.values.view(np.int64), np.arange(20))
    dup = synth.from_arrays(np.array([0, 3, 4], np.int64), np.array([2, 0, 2, 2], np.int32),
                            np.array([0, 1, 3, 3, 4], np.int64),
                            np.array([5, 6, 7, 8], np.int64).view(np.uint8), 3, 8)
    t = T(dup)
    assert np.array_equal(t.row_ptr, [0, 1, 1, 4])
    assert np.array_equal(t.col_idx, [0, 0, 0, 1])
    assert np.array_equal(t.cell_ptr, [0, 2, 3, 3, 4])
    assert np.array_equal(t.values.view(np.int64), [6, 7, 5, 8])


PINS = [pin_hand_example, pin_brute_force_dense, pin_stable_argsort_and_bincount,
        pin_scipy_single_value, pin_involution_chain, pin_unsorted_rows_double_transpose,
        pin_literal_and_partition_invariance, pin_tuple_multiset, pin_degree_and_partition_sums,
        pin_closed_form_balanced, pin_closed_form_counter_payload, pin_edge_cases]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_oracle_pin(pin):
    pin(oracle.transpose)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5])
def test_pins_catch_planted_mistakes(mutant):
    """Each planted mistake (reversed dealing, column kept instead of row,
    one run length off, two values swapped, destination block from the row)
    must fail at least one pin."""

    def T(x, part_off=None):
        return oracle.transpose(x, part_off, mutant=mutant)

    failed = []
    for pin in PINS:
        try:
            pin(T)
        except (AssertionError, oracle.OracleError, ValueError, IndexError):
            failed.append(pin.__name__)
    assert failed, f"planted mistake {mutant} passed every pin"


# ------------------------------------------------- other oracle entry points
def test_rows_against_brute_force():
    for seed in range(4):
        x = random_small(100 + seed, 30, 30, max_cells=6)
        rp, ci, cp, vals = brute_force_dense(x)
        sel = np.array([0, 3, 4, 17, 29], dtype=np.int64)
        cnt, t_col, t_len, t_val = oracle.rows(x, sel)
        pos, vpos = 0, 0
        for t, j in enumerate(sel):
            a, b = rp[j], rp[j + 1]
            assert cnt[t] == b - a
            assert np.array_equal(t_col[pos:pos + cnt[t]], ci[a:b])
            assert np.array_equal(t_len[pos:pos + cnt[t]], np.diff(cp[a:b + 1]))
            nb = (cp[b] - cp[a]) * x.stride
            assert np.array_equal(t_val[vpos:vpos + nb], vals[cp[a] * x.stride:cp[b] * x.stride])
            pos += cnt[t]
            vpos += nb


def test_degrees_against_bincount():
    x = synth.generate(synth.heterogeneous(seed=9, n=8192, parts=4))
    assert np.array_equal(oracle.degrees(x), np.bincount(x.col_idx, minlength=x.n_cols))


def test_validate_rejects_malformed():
    x = random_small(1, 10, 10)
    assert oracle.validate(x) == 0
    bad = synth.from_arrays(x.row_ptr.copy(), x.col_idx.copy(), x.cell_ptr.copy(), x.values, 10, 8)
    bad.col_idx[0] = 10
    assert oracle.validate(bad) == oracle.XO_EBADINPUT
    bad = synth.from_arrays(x.row_ptr.copy(), x.col_idx.copy(), x.cell_ptr.copy(), x.values, 10, 8)
    bad.row_ptr[3], bad.row_ptr[4] = bad.row_ptr[4] + 1, bad.row_ptr[3]
    assert oracle.validate(bad) == oracle.XO_EBADINPUT
    bad = synth.from_arrays(x.row_ptr, x.col_idx, x.cell_ptr, x.values, 10, 8,
                            part_off=np.array([0, 6, 5, 10]))
    assert oracle.validate(bad) == oracle.XO_EINVAL
    rect = random_small(2, 6, 9)
    rect.part_off = np.array([0, 3, 6], dtype=np.int64)
    assert oracle.validate(rect) == oracle.XO_EINVAL
    with pytest.raises(oracle.OracleError):
        oracle.transpose(rect)


def test_generator_shapes():
    """The synthetic workloads have the advertised structure."""
    b = synth.generate(synth.balanced(seed=0, n=8192, parts=8))
    assert b.n_cells == 32 * 8192 and b.n_values == 4 * b.n_cells
    for i in range(0, b.n_rows, 511):
        seg = b.col_idx[b.row_ptr[i]:b.row_ptr[i + 1]]
        assert len(seg) == 32 and np.all(np.diff(seg) > 0)
    h = synth.generate(synth.heterogeneous(seed=0, n=65536, parts=32))
    rl = np.diff(h.row_ptr)
    assert 17 < rl.mean() < 23 and rl.max() <= 4096
    ln = np.diff(h.cell_ptr)
    assert ln.min() >= 1 and ln.max() <= 64 and 4.6 < ln.mean() < 5.4
    assert np.all(np.diff(h.part_off) >= 0) and h.part_off[-1] == h.n_rows
    t = synth.generate(synth.tiny(seed=0))
    assert np.array_equal(t.part_off, [0, 250, 500, 750, 1000])
    # thread-count independence
    a = synth.generate(synth.heterogeneous(seed=3, n=20000, parts=4), nthreads=1)
    c = synth.generate(synth.heterogeneous(seed=3, n=20000, parts=4), nthreads=7)
    assert same_xcsr(a.row_ptr, a.col_idx, a.cell_ptr, a.values, c.row_ptr, c.col_idx,
                     c.cell_ptr, c.values)


def test_paper_benchmark_shapes():
    """The paper's Sec. 5 shapes: uniform row lengths in [lo, hi] with distinct
    ascending columns and 128-byte values of mean count 5; 512 cells of 10
    four-byte values; both independent of the thread count."""
    sp = synth.paper_heterogeneous(seed=2, rows=24, cols=40_000, lo=5_000, hi=15_000)
    h = synth.generate(sp)
    rl = np.diff(h.row_ptr)
    assert rl.min() >= 5_000 and rl.max() <= 15_000 and 8_500 < rl.mean() < 11_500
    for i in range(h.n_rows):
        seg = h.col_idx[h.row_ptr[i]:h.row_ptr[i + 1]]
        assert np.all(np.diff(seg) > 0) and seg[0] >= 0 and seg[-1] < h.n_cols
    ln = np.diff(h.cell_ptr)
    assert h.stride == 128 and ln.min() >= 1 and ln.max() <= 64 and 4.8 < ln.mean() < 5.2
    h1 = synth.generate(sp, nthreads=1)
    assert same_xcsr(h.row_ptr, h.col_idx, h.cell_ptr, h.values, h1.row_ptr, h1.col_idx,
                     h1.cell_ptr, h1.values)
    b = synth.generate(synth.paper_balanced(seed=0, n=1024, parts=4))
    assert b.n_cells == 512 * 1024 and b.n_values == 10 * b.n_cells and b.stride == 4
    assert np.array_equal(b.part_off, [0, 256, 512, 768, 1024])


def test_zipf_sampler_frequencies():
    """Rejection-inversion Zipf against the exact probability mass."""
    s, n = 1.1, 1000
    draws = synth.zipf_sample(s, n, 5, 400_000)
    assert draws.min() >= 1 and draws.max() <= n
    p = np.arange(1, n + 1, dtype=np.float64) ** -s
    p /= p.sum()
    freq = np.bincount(draws, minlength=n + 1)[1:] / draws.size
    for k in (1, 2, 3, 5, 10, 50):
        sd = np.sqrt(p[k - 1] * (1 - p[k - 1]) / draws.size)
        assert abs(freq[k - 1] - p[k - 1]) < 5 * sd + 1e-4


def test_perm_is_bijection():
    n = 5000
    img = np.array([synth.perm(9, n, i) for i in range(n)])
    assert np.array_equal(np.sort(img), np.arange(n))
