"""ORACLE (second restatement) -- test infrastructure only.

The distributed transpose of the paper's Sec. 3, simulated for P virtual ranks
in plain Python/numpy, step by step in the paper's order, for small inputs:

  0. every rank learns all ranks' row counts and turns them into row
     intervals [sum_{s<r} |V_s|, sum_{s<=r} |V_s|)            (Sec. 2, step 1)
  1. LocalTranspose (Eq. 3): rank s transposes its own row block M_s into
     M_s^T, whose rows are the global columns and whose cells name global
     rows; no communication                                     (Sec. 3)
  2. ViewSwap, step 1 (Eq. 4): a dense P x P transpose of the metadata
     counts tells each rank how many cells it receives from each sender;
     the metadata (row id, column id, number of values) of every cell is
     then sent to the rank that owns its row of M^T              (Sec. 3)
  3. ViewSwap, step 2: a dense P x P transpose of the value counts, then
     the values themselves                                       (Sec. 3)
  4. each receiver orders what it got by row, then by sender (row-column
     ordering), which is M_1^T // ... // M_P^T restricted to its rows
     (the composition argument at the end of Sec. 3).

Concatenating the receivers' blocks gives the global transpose.  The result
must equal the counting transpose of ``oracle.transpose`` for every P; that
equality is the paper's claim that LocalTranspose and ViewSwap compose to the
transpose (Sec. 3).  Nothing here is shared with ``xcsr_oracle.c``.
"""
from __future__ import annotations

import numpy as np


def _intervals(row_counts):
    """Row interval of each rank from the gathered row counts (Sec. 2)."""
    lo, out = 0, []
    for n in row_counts:
        out.append((lo, lo + n))
        lo += n
    return out


def _owner(intervals, j):
    for r, (a, b) in enumerate(intervals):
        if a <= j < b:
            return r
    raise ValueError(f"row {j} is not covered by any rank")


def transpose(x, part_off=None):
    """Returns (row_ptr', col_idx', cell_ptr', values', part_cells, part_values)
    with int64 offsets; ``x`` is a ``synth.XCSR``-like object."""
    off = np.asarray(x.part_off if part_off is None else part_off, dtype=np.int64)
    P = len(off) - 1
    s = x.stride
    row_ptr = np.asarray(x.row_ptr, dtype=np.int64)
    cell_ptr = np.asarray(x.cell_ptr, dtype=np.int64)
    col = np.asarray(x.col_idx, dtype=np.int64)
    vals = np.asarray(x.values, dtype=np.uint8)
    N = x.n_cols

    # 0. gather row counts, derive every rank's row interval
    src_iv = _intervals([int(off[r + 1] - off[r]) for r in range(P)])
    # receivers own rows of M^T; with one rank the output simply has N rows,
    # with several the matrix is square and the same intervals are reused
    dst_iv = src_iv if P > 1 else [(0, N)]

    # 1. LocalTranspose: rank r builds M_r^T as (row j, column i, value run)
    #    triples ordered by j, then by position in the rank's input
    local_T = []
    for r in range(P):
        a, b = src_iv[r]
        triples = []
        for i in range(a, b):
            for k in range(int(row_ptr[i]), int(row_ptr[i + 1])):
                run = bytes(vals[int(cell_ptr[k]) * s:int(cell_ptr[k + 1]) * s])
                triples.append((int(col[k]), i, run))
        triples.sort(key=lambda t: t[0])  # Python's sort is stable
        local_T.append(triples)

    # 2a. dense transpose of the metadata counts: send[r][d] -> recv[d][r]
    send_cells = np.zeros((P, P), dtype=np.int64)
    send_vals = np.zeros((P, P), dtype=np.int64)
    for r in range(P):
        for (j, i, run) in local_T[r]:
            d = _owner(dst_iv, j)
            send_cells[r, d] += 1
            send_vals[r, d] += len(run) // s
    recv_cells = send_cells.T.copy()
    # 2b. sparse transpose of the metadata (row id, column id, #values)
    meta_in = [[[] for _ in range(P)] for _ in range(P)]  # meta_in[d][r]
    for r in range(P):
        for (j, i, run) in local_T[r]:
            meta_in[_owner(dst_iv, j)][r].append((j, i, len(run) // s))
    # 3a. dense transpose of the value counts; 3b. sparse transpose of values
    recv_vals = send_vals.T.copy()
    vals_in = [[bytearray() for _ in range(P)] for _ in range(P)]
    for r in range(P):
        for (j, i, run) in local_T[r]:
            vals_in[_owner(dst_iv, j)][r] += run
    for d in range(P):
        for r in range(P):
            assert len(meta_in[d][r]) == recv_cells[d, r]
            assert len(vals_in[d][r]) == recv_vals[d, r] * s

    # 4. row-column ordering on each receiver: for every row it owns, the
    #    cells of sender 0, then sender 1, ...; value runs follow the metadata
    out_rows, out_cols, out_lens, out_vals = [], [], [], []
    for d in range(P):
        a, b = dst_iv[d]
        per_row = {j: [] for j in range(a, b)}
        for r in range(P):
            pos = 0
            buf = vals_in[d][r]
            for (j, i, n) in meta_in[d][r]:
                per_row[j].append((i, bytes(buf[pos * s:(pos + n) * s])))
                pos += n
        for j in range(a, b):
            out_rows.append(len(per_row[j]))
            for (i, run) in per_row[j]:
                out_cols.append(i)
                out_lens.append(len(run) // s)
                out_vals.append(run)

    t_row_ptr = np.concatenate([[0], np.cumsum(out_rows, dtype=np.int64)]).astype(np.int64)
    t_cell_ptr = np.concatenate([[0], np.cumsum(out_lens, dtype=np.int64)]).astype(np.int64)
    t_col = np.asarray(out_cols, dtype=np.int32)
    t_vals = np.frombuffer(b"".join(out_vals), dtype=np.uint8).copy()
    return t_row_ptr, t_col, t_cell_ptr, t_vals, send_cells, send_vals
