"""Shared test helpers: small hand-built XCSR matrices, brute-force dense
transposition and comparisons.  Test infrastructure only."""
from __future__ import annotations

import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def random_small(seed: int, R: int, N: int, *, max_cells: int = 6, max_len: int = 4,
                 stride: int = 8, offset_bytes: int = 8, sorted_rows: bool = True,
                 dup_cols: bool = False, n_parts: int = 1, p_zero_len: float = 0.2):
    """A tiny random XCSR matrix drawn with numpy (independent of synth.c's
    distributions; used for brute-force pins).  Values are random bytes."""
    rng = np.random.default_rng(seed)
    rows, lens = [], []
    for i in range(R):
        n = int(rng.integers(0, min(max_cells, N if not dup_cols else max_cells) + 1))
        if dup_cols:
            cols = rng.integers(0, N, size=n)
        else:
            cols = rng.choice(N, size=n, replace=False)
        if sorted_rows:
            cols = np.sort(cols, kind="stable")
        rows.append(cols.astype(np.int32))
        for _ in range(n):
            lens.append(0 if rng.random() < p_zero_len else int(rng.integers(1, max_len + 1)))
    row_ptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int64)
    col_idx = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
    cell_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64) if lens else np.zeros(1, np.int64)
    V = int(cell_ptr[-1])
    values = rng.integers(0, 256, size=V * stride, dtype=np.uint8)
    odt = np.int32 if offset_bytes == 4 else np.int64
    if n_parts > 1:
        assert R == N
        cuts = np.sort(rng.choice(np.arange(0, R + 1), size=n_parts - 1, replace=True))
        part_off = np.concatenate([[0], cuts, [R]]).astype(np.int64)
    else:
        part_off = np.array([0, R], dtype=np.int64)
    return synth.from_arrays(row_ptr.astype(odt), col_idx, cell_ptr.astype(odt), values, N,
                             stride, part_off, offset_bytes)


def cells_of(x):
    """List of (row, col, run bytes) in row-major order."""
    out = []
    s = x.stride
    for i in range(x.n_rows):
        for k in range(int(x.row_ptr[i]), int(x.row_ptr[i + 1])):
            a, b = int(x.cell_ptr[k]), int(x.cell_ptr[k + 1])
            out.append((i, int(x.col_idx[k]), bytes(x.values[a * s:b * s])))
    return out


def brute_force_dense(x):
    """Transpose through a dense R x N array of value lists (distinct columns
    per row required): M^T[j][i] = M[i][j], then re-encode row-major."""
    dense = [[None] * x.n_cols for _ in range(x.n_rows)]
    for (i, j, run) in cells_of(x):
        assert dense[i][j] is None, "dense pin needs distinct columns per row"
        dense[i][j] = run
    t_row, t_col, t_len, t_vals = [0], [], [], []
    for j in range(x.n_cols):
        for i in range(x.n_rows):
            if dense[i][j] is not None:
                t_col.append(i)
                t_len.append(len(dense[i][j]) // x.stride)
                t_vals.append(dense[i][j])
        t_row.append(len(t_col))
    t_cell = np.concatenate([[0], np.cumsum(t_len)]).astype(np.int64) if t_len else np.zeros(1, np.int64)
    return (np.asarray(t_row, np.int64), np.asarray(t_col, np.int32), t_cell,
            np.frombuffer(b"".join(t_vals), np.uint8))


def parse_golden(name: str):
    """Parse a hand-worked fixture: returns (input XCSR, expected arrays)."""
    meta, ins, outs = {}, {}, {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("in ") or line.startswith("out "):
                head, _, body = line.partition("|")
                kind, r = head.split()
                cells = []
                for tok in body.split():
                    c, _, v = tok.partition(":")
                    vs = [int(t) for t in v.strip("[]").split(",") if t]
                    cells.append((int(c), vs))
                (ins if kind == "in" else outs)[int(r)] = cells
            else:
                k, v = line.split()
                meta[k] = int(v)

    def encode(rows, n):
        rp, ci, cp, vals = [0], [], [0], []
        for r in range(n):
            for (c, vs) in rows.get(r, []):
                ci.append(c)
                vals.extend(vs)
                cp.append(cp[-1] + len(vs))
            rp.append(len(ci))
        return (np.asarray(rp, np.int64), np.asarray(ci, np.int32), np.asarray(cp, np.int64),
                np.asarray(vals, np.int64).view(np.uint8))

    R, N = meta["n_rows"], meta["n_cols"]
    rp, ci, cp, vals = encode(ins, R)
    x = synth.from_arrays(rp, ci, cp, vals, N, 8)
    return x, encode(outs, N)


def sorted_rows_copy(x):
    """x with each row's cells stably sorted by column (runs move along)."""
    rp, ci, cp, vals, s = x.row_ptr, x.col_idx, x.cell_ptr, x.values, x.stride
    order = []
    for i in range(x.n_rows):
        a, b = int(rp[i]), int(rp[i + 1])
        order.extend((a + np.argsort(ci[a:b], kind="stable")).tolist())
    order = np.asarray(order, dtype=np.int64)
    new_ci = ci[order] if len(order) else ci.copy()
    lens = (cp[1:] - cp[:-1])[order] if len(order) else np.zeros(0, np.int64)
    new_cp = np.concatenate([[0], np.cumsum(lens)]).astype(cp.dtype)
    chunks = [vals[int(cp[k]) * s:int(cp[k + 1]) * s] for k in order]
    new_vals = np.concatenate(chunks) if chunks else vals[:0].copy()
    return synth.from_arrays(rp.copy(), new_ci, new_cp, new_vals, x.n_cols, s, x.part_off.copy(),
                             x.offset_bytes)


def same_xcsr(a_row, a_col, a_cp, a_val, b_row, b_col, b_cp, b_val):
    return (np.array_equal(np.asarray(a_row, np.int64), np.asarray(b_row, np.int64))
            and np.array_equal(np.asarray(a_col, np.int32), np.asarray(b_col, np.int32))
            and np.array_equal(np.asarray(a_cp, np.int64), np.asarray(b_cp, np.int64))
            and np.array_equal(np.asarray(a_val, np.uint8).reshape(-1),
                               np.asarray(b_val, np.uint8).reshape(-1)))


# ------------------------------------------------------------ GPU helpers
def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def gpu_transpose(x, cfg=None, with_parts=True):
    """Transposes host XCSR ``x`` through the C ABI on cuda:0; returns
    (row_ptr, col_idx, cell_ptr, values, part_cells, part_values, status, plan)
    as numpy arrays."""
    import torch
    from paper_2012_06012_gb300 import mgt
    d = mgt.to_device(x)
    plan = mgt.plan_for(d, cfg=cfg, with_parts=with_parts)
    ws = mgt.alloc_workspace(plan.workspace_bytes)
    out = mgt.alloc_output(d, parts=True)
    if not with_parts or plan.n_parts == 1 and len(x.part_off) > 2:
        out = out[:4] + (None, None)
    mgt.transpose(plan, d.arrays(), out, ws)
    status = mgt.read_status(ws)
    torch.cuda.synchronize()
    res = [None if t is None else t.cpu().numpy() for t in out]
    return (*res, status, plan)


def assert_same_as_oracle(x, got, ref, check_parts=True):
    row_ptr, col_idx, cell_ptr, values, pc, pv, status, plan = got
    assert status == 0, f"device status {status} (tiles {plan.config})"
    assert np.array_equal(row_ptr, ref.row_ptr), f"row_ptr differs (tiles {plan.config})"
    assert np.array_equal(col_idx, ref.col_idx), f"col_idx differs (tiles {plan.config})"
    assert np.array_equal(cell_ptr, ref.cell_ptr), f"cell_ptr differs (tiles {plan.config})"
    assert np.array_equal(values, ref.values), f"values differ (tiles {plan.config})"
    if check_parts and pc is not None:
        P = ref.part_cells.shape[0]
        assert np.array_equal(pc.reshape(P, P), ref.part_cells), "P x P cells differ"
        assert np.array_equal(pv.reshape(P, P), ref.part_values), "P x P values differ"


# ------------------------------------------------ variable-width values
def random_small_var(seed: int, R: int, N: int, *, max_cells: int = 6, max_len: int = 4,
                     widths=(0, 1, 3, 4, 5, 8, 12, 16, 33), offset_bytes: int = 8,
                     sorted_rows: bool = True, dup_cols: bool = False, n_parts: int = 1):
    """A tiny random matrix whose values have individual byte widths drawn
    from ``widths`` (numpy; independent of synth.c)."""
    x = random_small(seed, R, N, max_cells=max_cells, max_len=max_len, stride=4,
                     offset_bytes=offset_bytes, sorted_rows=sorted_rows, dup_cols=dup_cols,
                     n_parts=n_parts)
    rng = np.random.default_rng(seed + 7919)
    V = x.n_values
    w = rng.choice(np.asarray(widths, dtype=np.int64), size=V) if V else np.zeros(0, np.int64)
    val_off = np.concatenate([[0], np.cumsum(w)]).astype(np.int64)
    values = rng.integers(0, 256, size=int(val_off[-1]), dtype=np.uint8)
    return synth.var_from_arrays(x.row_ptr, x.col_idx, x.cell_ptr, val_off, values, N,
                                 x.part_off, offset_bytes)


def var_cells_of(x):
    """List of (row, col, tuple of value byte strings) in row-major order."""
    out = []
    vo, vals = x.val_off, x.values
    for i in range(x.n_rows):
        for k in range(int(x.row_ptr[i]), int(x.row_ptr[i + 1])):
            run = tuple(bytes(vals[int(vo[v]):int(vo[v + 1])])
                        for v in range(int(x.cell_ptr[k]), int(x.cell_ptr[k + 1])))
            out.append((i, int(x.col_idx[k]), run))
    return out


def var_brute_force_dense(x):
    """Dense transposition of an R x N array of lists of byte strings
    (distinct columns per row), re-encoded: (row_ptr, col, cell_ptr,
    val_off, values)."""
    dense = [[None] * x.n_cols for _ in range(x.n_rows)]
    for (i, j, run) in var_cells_of(x):
        assert dense[i][j] is None, "dense pin needs distinct columns per row"
        dense[i][j] = run
    t_row, t_col, t_cell, sizes, chunks = [0], [], [0], [], []
    for j in range(x.n_cols):
        for i in range(x.n_rows):
            if dense[i][j] is not None:
                t_col.append(i)
                t_cell.append(t_cell[-1] + len(dense[i][j]))
                for b in dense[i][j]:
                    sizes.append(len(b))
                    chunks.append(b)
        t_row.append(len(t_col))
    t_vo = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64) if sizes else np.zeros(1, np.int64)
    return (np.asarray(t_row, np.int64), np.asarray(t_col, np.int32),
            np.asarray(t_cell, np.int64), t_vo, np.frombuffer(b"".join(chunks), np.uint8))


def same_var(t, rp, ci, cp, vo, vals) -> bool:
    return (np.array_equal(np.asarray(t.row_ptr, np.int64), np.asarray(rp, np.int64))
            and np.array_equal(np.asarray(t.col_idx, np.int32), np.asarray(ci, np.int32))
            and np.array_equal(np.asarray(t.cell_ptr, np.int64), np.asarray(cp, np.int64))
            and np.array_equal(np.asarray(t.val_off, np.int64), np.asarray(vo, np.int64))
            and np.array_equal(np.asarray(t.values, np.uint8).reshape(-1),
                               np.asarray(vals, np.uint8).reshape(-1)))
