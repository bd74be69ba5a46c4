"""Parity at the benchmark's full sizes, in the benchmark's launch
configuration (default plan): the balanced multigraph (4,194,304 x
4,194,304, 128M cells, 512M values) and the heterogeneous matrix (8,388,608
x 8,388,608, ~168M cells, Zipf columns, 256 unequal row blocks).  The full
oracle is too slow here, so: row_ptr' against the oracle's column degrees
(every entry), sampled output rows against rows the oracle computes one by
one from the definition (random, first, last, the hottest columns and
empty ones), the P x P counts against their definition, and the sentinels."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def _part_counts(x):
    """P x P cells and values from the definition (row block of the cell's
    row, row block of its column)."""
    P = len(x.part_off) - 1
    rows = np.repeat(np.arange(x.n_rows, dtype=np.int64), np.diff(x.row_ptr.astype(np.int64)))
    s = np.searchsorted(x.part_off, rows, side="right") - 1
    d = np.searchsorted(x.part_off, x.col_idx.astype(np.int64), side="right") - 1
    lens = np.diff(x.cell_ptr.astype(np.int64))
    key = s * P + d
    cells = np.bincount(key, minlength=P * P).reshape(P, P)
    vals = np.bincount(key, weights=lens, minlength=P * P).astype(np.int64).reshape(P, P)
    return cells, vals


@pytest.mark.parametrize("workload", ["balanced", "heterogeneous"])
def test_full_size_sampled_parity(workload):
    from paper_2012_06012_gb300 import mgt
    spec = synth.balanced(seed=0) if workload == "balanced" else synth.heterogeneous(seed=0)
    x = synth.generate(spec)
    d = mgt.to_device(x)
    out, plan, ws = mgt.transpose_device(d)
    torch.cuda.synchronize()
    # every row pointer
    deg = oracle.degrees(x)
    want_rp = np.concatenate([[0], np.cumsum(deg)])
    got_rp = out[0].cpu().numpy().astype(np.int64)
    assert np.array_equal(got_rp, want_rp)
    got_cp = out[2].cpu().numpy().astype(np.int64)
    assert got_cp[0] == 0 and got_cp[-1] == x.n_values
    # sampled rows
    rng = np.random.default_rng(1)
    sel = set(rng.choice(x.n_cols, size=160, replace=False).tolist())
    sel |= {0, x.n_cols - 1}
    sel |= set(np.argsort(deg)[-4:].tolist())            # hottest columns
    empty = np.flatnonzero(deg == 0)
    sel |= set(empty[:4].tolist())
    sel = np.array(sorted(sel), dtype=np.int64)
    cnt, t_col, t_len, t_val = oracle.rows(x, sel)
    col_dev, val_dev = out[1], out[3]
    o = 0
    vo = 0
    for r, c in zip(sel, cnt):
        a, b = int(want_rp[r]), int(want_rp[r + 1])
        assert b - a == c
        assert np.array_equal(col_dev[a:b].cpu().numpy(), t_col[o:o + c])
        lens = np.diff(got_cp[a:b + 1])
        assert np.array_equal(lens, t_len[o:o + c])
        nb = int(lens.sum()) * x.stride
        v0 = int(got_cp[a]) * x.stride
        assert np.array_equal(val_dev[v0:v0 + nb].cpu().numpy(), t_val[vo:vo + nb])
        o += c
        vo += nb
    # P x P from the definition
    pc, pv = _part_counts(x)
    P = pc.shape[0]
    assert np.array_equal(out[4].cpu().numpy().reshape(P, P), pc)
    assert np.array_equal(out[5].cpu().numpy().reshape(P, P), pv)
