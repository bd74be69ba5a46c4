"""Variable-width values (the paper's heterogeneous-datatype variant, Sec. 2:
one datatype per edge through MPI_Alltoallw) through the C ABI's
mgt_transpose_var, against the oracle's variable-width transpose bit for bit:
mixed widths that take the 16-, 8-, 4- and 1-byte copy paths, zero-width
values, unsorted rows with duplicate columns, both offset widths, several
tile shapes, row blocks with their P x P counts, malformed value offsets and
a transpose of the transpose."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from helpers import gpu_available, random_small_var

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

CFGS = [None,
        {"cluster": 1, "chunk_cap": 512, "scatter_tile": 1024, "copy_unroll": 1},
        {"cluster": 2, "chunk_cap": 1024, "bucket_shift": 5, "copy_unroll": 4},
        {"cluster": 8, "chunk_cap": 512, "bucket_shift": 3}]
CFG_IDS = ["default", "cs1-small", "cs2", "cs8-small"]


def gpu_transpose_var(x, cfg=None):
    import torch
    from paper_2012_06012_gb300 import mgt
    d = mgt.to_device_var(x)
    plan = mgt.plan_for_var(d, cfg)
    ws = mgt.alloc_workspace(plan.workspace_bytes)
    out, ovo = mgt.alloc_output_var(d, parts=True)
    for t in out + (ovo,):
        if t is not None:
            t.fill_(0x5A if t.dtype == torch.uint8 else -3)
    mgt.transpose_var(plan, d.arrays(), d.val_off, out, ovo, ws)
    st = mgt.read_status(ws)
    torch.cuda.synchronize()
    return [None if t is None else t.cpu().numpy() for t in out], ovo.cpu().numpy(), st, plan


def part_counts(x):
    """P x P counts from the fixed-width oracle on the same cells (the
    counts do not depend on the value widths)."""
    fx = synth.from_arrays(x.row_ptr, x.col_idx, x.cell_ptr,
                           np.zeros(int(x.cell_ptr[-1]) * 4, np.uint8), x.n_cols, 4, x.part_off,
                           x.offset_bytes)
    r = oracle.transpose(fx)
    return r.part_cells, r.part_values


def assert_var_equal(x, got, check_parts=True):
    out, ovo, st, plan = got
    assert st == 0, f"device status {st} (tiles {plan.config})"
    ref = oracle.transpose_var(x)
    assert np.array_equal(out[0], ref.row_ptr), "row_ptr'"
    assert np.array_equal(out[1], ref.col_idx), "col_idx'"
    assert np.array_equal(out[2], ref.cell_ptr), "cell_ptr'"
    assert np.array_equal(ovo, ref.val_off), "val_off'"
    assert np.array_equal(out[3], ref.values), "values'"
    if check_parts:
        pc, pv = part_counts(x)
        P = pc.shape[0]
        assert np.array_equal(out[4].reshape(P, P), pc)
        assert np.array_equal(out[5].reshape(P, P), pv)


WIDTHS = {
    "types": synth.TYPE_SIZES,            # 4..64, multiples of 4
    "x16": (16, 32, 48, 64),              # 16-byte copies
    "x8": (8, 24, 40),                    # 8-byte copies
    "odd": (0, 1, 2, 3, 5, 7, 13, 31),    # byte copies, zero widths
    "zero": (0,),                         # values without bytes
}


@pytest.mark.parametrize("widths", list(WIDTHS), ids=list(WIDTHS))
@pytest.mark.parametrize("offset_bytes", [4, 8])
def test_var_heterogeneous_widths(widths, offset_bytes):
    sp = synth.heterogeneous(seed=51, n=20_011, parts=7)
    sp.offset_bytes = offset_bytes
    x = synth.generate_var(sp, sizes=WIDTHS[widths])
    assert_var_equal(x, gpu_transpose_var(x))


@pytest.mark.parametrize("cfg", CFGS, ids=CFG_IDS)
def test_var_tile_shapes(cfg):
    x = synth.generate_var(synth.heterogeneous(seed=52, n=30_000, parts=16))
    assert_var_equal(x, gpu_transpose_var(x, cfg))


@pytest.mark.parametrize("seed", range(4))
def test_var_random_small_unsorted_duplicates(seed):
    x = random_small_var(200 + seed, 300, 300, max_cells=12, max_len=7, sorted_rows=False,
                         dup_cols=True, n_parts=3, offset_bytes=4 + 4 * (seed % 2))
    assert_var_equal(x, gpu_transpose_var(x))


def test_var_rectangular():
    x = random_small_var(210, 300, 257, max_cells=12, max_len=7, sorted_rows=False, dup_cols=True)
    assert_var_equal(x, gpu_transpose_var(x))


def test_var_edge_cases():
    empty = synth.var_from_arrays(np.zeros(6, np.int64), np.zeros(0, np.int32),
                                  np.zeros(1, np.int64), np.zeros(1, np.int64),
                                  np.zeros(0, np.uint8), 4)
    assert_var_equal(empty, gpu_transpose_var(empty), check_parts=False)
    no_values = synth.var_from_arrays([0, 2, 3], [0, 1, 1], [0, 0, 0, 0], np.zeros(1, np.int64),
                                      np.zeros(0, np.uint8), 2)
    assert_var_equal(no_values, gpu_transpose_var(no_values), check_parts=False)
    one_long = synth.var_from_arrays([0, 0, 1], [0], [0, 9],
                                     np.array([0, 1, 3, 6, 10, 15, 21, 28, 36, 45]),
                                     np.arange(1, 46, dtype=np.uint8), 3)
    assert_var_equal(one_long, gpu_transpose_var(one_long), check_parts=False)


def test_var_transpose_twice_is_identity():
    import torch
    from paper_2012_06012_gb300 import mgt
    x = synth.generate_var(synth.heterogeneous(seed=53, n=12_000, parts=1))
    out, ovo, st, _ = gpu_transpose_var(x)
    assert st == 0
    t = synth.var_from_arrays(out[0], out[1], out[2], ovo, out[3], x.n_rows,
                              offset_bytes=x.offset_bytes)
    back, bvo, st2, _ = gpu_transpose_var(t)
    assert st2 == 0
    for a, b in ((back[0], x.row_ptr), (back[1], x.col_idx), (back[2], x.cell_ptr), (bvo, x.val_off),
                 (back[3], x.values)):
        assert np.array_equal(a, b)
    del torch, mgt


def test_var_malformed_offsets_flagged():
    """Value offsets that decrease inside a run, or do not end at the byte
    count, are reported as MGT_EBADINPUT; nothing outside the buffers is
    touched and the next transpose on the same context is correct."""
    from paper_2012_06012_gb300 import mgt
    x = synth.generate_var(synth.heterogeneous(seed=54, n=5_000, parts=1))
    bad = synth.var_from_arrays(x.row_ptr, x.col_idx, x.cell_ptr, x.val_off.copy(), x.values,
                                x.n_cols)
    mid = len(bad.val_off) // 2
    bad.val_off[mid] = bad.val_off[mid + 1] + 8  # decreases after mid
    assert gpu_transpose_var(bad)[2] == mgt.MGT_EBADINPUT
    short = synth.var_from_arrays(x.row_ptr, x.col_idx, x.cell_ptr, x.val_off.copy(), x.values,
                                  x.n_cols)
    short.val_off[-1] -= 4  # ends before the byte count
    assert gpu_transpose_var(short)[2] == mgt.MGT_EBADINPUT
    assert_var_equal(x, gpu_transpose_var(x), check_parts=False)


def test_var_plan_refused_elsewhere():
    """A variable-width plan is refused by the fixed-width calls, and a
    fixed-width plan by mgt_transpose_var."""
    import torch
    from paper_2012_06012_gb300 import mgt
    x = synth.generate_var(synth.heterogeneous(seed=55, n=2_000, parts=1))
    d = mgt.to_device_var(x)
    plan = mgt.plan_for_var(d)
    ws = mgt.alloc_workspace(plan.workspace_bytes)
    out, ovo = mgt.alloc_output_var(d, parts=False)
    L = mgt.lib()
    import ctypes
    xi = mgt.XcsrIn(*[mgt._ptr(t) for t in d.arrays()])
    xo = mgt.XcsrOut(*[mgt._ptr(t) for t in out])
    assert L.mgt_transpose(plan.handle, ctypes.byref(xi), ctypes.byref(xo), mgt._ptr(ws), ws.numel(),
                           None) == mgt.MGT_EINVAL
    fixed = mgt.Plan(x.n_rows, x.n_cols, x.n_cells, x.n_values, x.offset_bytes, 4)
    assert L.mgt_transpose_var(fixed.handle, ctypes.byref(xi), mgt._ptr(d.val_off), ctypes.byref(xo),
                               mgt._ptr(ovo), int(d.values.numel()), mgt._ptr(ws), ws.numel(), None,
                               None, 0) == mgt.MGT_EINVAL
    torch.cuda.synchronize()
