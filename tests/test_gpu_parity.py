"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element and bit for bit, on seeded inputs spanning several tiles, buckets and
sort chunks, ragged tails and the method's degenerate cases."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from helpers import assert_same_as_oracle, gpu_available, gpu_transpose, random_small

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

# tile shapes that force each code path: default; one-CTA sort chunks small
# enough that most buckets split into several chunks; 2- and 4-CTA clusters
CFGS = [None,
        {"cluster": 1, "chunk_cap": 512, "scatter_tile": 1024, "copy_unroll": 1},
        {"cluster": 2, "chunk_cap": 1024, "bucket_shift": 5, "copy_unroll": 4},
        {"cluster": 4, "chunk_cap": 2048, "bucket_shift": 8, "scatter_tile": 4096},
        {"cluster": 8, "chunk_cap": 512, "bucket_shift": 3}]
CFG_IDS = ["default", "cs1-small", "cs2", "cs4", "cs8-small"]


@pytest.mark.parametrize("cfg", CFGS, ids=CFG_IDS)
def test_tiny_workload(cfg):
    x = synth.generate(synth.tiny(seed=0))
    assert_same_as_oracle(x, gpu_transpose(x, cfg), oracle.transpose(x))


@pytest.mark.parametrize("cfg", CFGS, ids=CFG_IDS)
def test_balanced_small(cfg):
    x = synth.generate(synth.balanced(seed=1, n=50_001, parts=8))
    assert_same_as_oracle(x, gpu_transpose(x, cfg), oracle.transpose(x))


@pytest.mark.parametrize("cfg", CFGS, ids=CFG_IDS)
def test_heterogeneous_small(cfg):
    x = synth.generate(synth.heterogeneous(seed=2, n=30_011, parts=16))
    assert_same_as_oracle(x, gpu_transpose(x, cfg), oracle.transpose(x))


@pytest.mark.parametrize("perm", [0, 1])
def test_heterogeneous_zipf_head(perm):
    """Identity rank->column mapping puts every hot column in bucket 0."""
    x = synth.generate(synth.heterogeneous(seed=3, n=65_536, parts=32, perm=perm))
    assert_same_as_oracle(x, gpu_transpose(x), oracle.transpose(x))


@pytest.mark.parametrize("offset_bytes", [4, 8])
@pytest.mark.parametrize("stride", [4, 8, 12, 16, 20, 32, 64])
def test_strides_and_offsets(stride, offset_bytes):
    sp = synth.heterogeneous(seed=4, n=5_003, parts=3)
    sp.stride, sp.offset_bytes, sp.payload = stride, offset_bytes, synth.PAY_BITS
    x = synth.generate(sp)
    assert_same_as_oracle(x, gpu_transpose(x), oracle.transpose(x))


@pytest.mark.parametrize("seed", range(6))
def test_random_small_with_unsorted_rows_and_duplicates(seed):
    x = random_small(500 + seed, 300, 300, max_cells=40, sorted_rows=False,
                     dup_cols=bool(seed % 2), n_parts=5, stride=8)
    for cfg in (None, CFGS[1]):
        assert_same_as_oracle(x, gpu_transpose(x, cfg), oracle.transpose(x))


def test_rectangular_single_partition():
    x = random_small(77, 1000, 37, max_cells=30)
    assert_same_as_oracle(x, gpu_transpose(x), oracle.transpose(x))
    y = random_small(78, 13, 4000, max_cells=300)
    assert_same_as_oracle(y, gpu_transpose(y), oracle.transpose(y))


def test_empty_and_degenerate():
    empty = synth.from_arrays(np.zeros(8, np.int64), np.zeros(0, np.int32), np.zeros(1, np.int64),
                              np.zeros(0, np.uint8), 5, 8)
    assert_same_as_oracle(empty, gpu_transpose(empty), oracle.transpose(empty))
    # one hot column, zero-length runs mixed in
    R = 20_000
    lens = np.where(np.arange(R) % 7 == 0, 0, 1 + np.arange(R) % 3)
    hot = synth.from_arrays(np.arange(R + 1, dtype=np.int64), np.full(R, 17, np.int32),
                            np.concatenate([[0], np.cumsum(lens)]).astype(np.int64),
                            np.arange(int(lens.sum()), dtype=np.int64).view(np.uint8), 40, 8)
    for cfg in (None, CFGS[1], CFGS[4]):
        assert_same_as_oracle(hot, gpu_transpose(hot, cfg), oracle.transpose(hot))
    # 1 x 1 and 1 x N
    one = synth.from_arrays(np.array([0, 1], np.int64), np.array([0], np.int32),
                            np.array([0, 3], np.int64), np.arange(3, dtype=np.int64).view(np.uint8), 1, 8)
    assert_same_as_oracle(one, gpu_transpose(one), oracle.transpose(one))


def test_long_runs_escape_path():
    """Runs of >= 65535 values take the length-recovery path."""
    lens = np.array([3, 70_000, 0, 65_535, 65_534, 1, 131_072], dtype=np.int64)
    C = len(lens)
    row_ptr = np.array([0, 2, 4, 7], np.int64)
    col = np.array([1, 0, 2, 0, 1, 2, 0], np.int32)
    cp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    vals = np.random.default_rng(5).integers(0, 255, size=int(cp[-1]) * 4, dtype=np.uint8)
    x = synth.from_arrays(row_ptr, col, cp, vals, 3, 4)
    assert_same_as_oracle(x, gpu_transpose(x), oracle.transpose(x))
    assert C == 7


def test_partition_invariance_of_arrays():
    """The XCSR output does not depend on P; only the P x P counts do."""
    x = synth.generate(synth.heterogeneous(seed=6, n=8_192, parts=1))
    base = gpu_transpose(x)
    for P in (2, 7, 64, 8_192):
        off = np.array([(d * x.n_rows) // P for d in range(P + 1)], dtype=np.int64)
        y = synth.from_arrays(x.row_ptr, x.col_idx, x.cell_ptr, x.values, x.n_cols, x.stride, off)
        got = gpu_transpose(y)
        for a, b in zip(got[:4], base[:4]):
            assert np.array_equal(a, b)
        ref = oracle.transpose(y)
        assert_same_as_oracle(y, got, ref)


def test_involution_chain_on_gpu():
    """Twelve chained transposes on the device give the input back."""
    import torch
    from paper_2012_06012_gb300 import mgt
    x = synth.generate(synth.tiny(seed=9, n=700))
    d = mgt.to_device(x)
    cur = d
    for _ in range(12):
        out, _, _ = mgt.transpose_device(cur)
        cur = mgt.DeviceXCSR(cur.n_cols, cur.n_rows, cur.offset_bytes, cur.stride, out[0], out[1],
                             out[2], out[3], cur.part_off)
    torch.cuda.synchronize()
    for a, b in zip(cur.arrays(), d.arrays()):
        assert torch.equal(a, b)


@pytest.mark.parametrize("N,cfg", [(20_000_000, None), (20_000_000, {"bucket_shift": 11}),
                                   (12_000_000, {"bucket_shift": 10})],
                         ids=["20M-default", "20M-bs11", "12M-bs10"])
def test_high_cardinality_columns(N, cfg):
    """Many columns, few cells per column: the most buckets a plan allows,
    with the second scatter pass's digit carried in wide intermediate
    records (20M columns: bucket_shift 11 + 6 digit bits > 16) or in the
    compact ones (12M: 10 + 6)."""
    rng = np.random.default_rng(11)
    R = 1 << 15
    per = rng.integers(0, 80, size=R)
    row_ptr = np.concatenate([[0], np.cumsum(per)]).astype(np.int64)
    C = int(row_ptr[-1])
    col = rng.integers(0, N, size=C, dtype=np.int64).astype(np.int32)
    lens = rng.integers(0, 4, size=C)
    cp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    vals = rng.integers(0, 256, size=int(cp[-1]) * 4, dtype=np.uint8)
    x = synth.from_arrays(row_ptr, col, cp, vals, N, 4)
    assert_same_as_oracle(x, gpu_transpose(x, cfg), oracle.transpose(x))


@pytest.mark.parametrize("cfg", [None, CFGS[1]], ids=["default", "cs1-small"])
def test_values_only_retranspose(cfg):
    """After a full transpose, new payloads on the same structure need only
    the value copy (mgt_transpose_values); a chain of twelve value-only
    transposes between the two structures gives the payload back."""
    import torch
    from paper_2012_06012_gb300 import mgt
    x = synth.generate(synth.heterogeneous(seed=12, n=20_000, parts=8))
    d = mgt.to_device(x)
    plan = mgt.plan_for(d, cfg)
    ws = mgt.alloc_workspace(plan.workspace_bytes)
    out = mgt.alloc_output(d)
    mgt.transpose(plan, d.arrays(), out, ws)
    assert mgt.read_status(ws) == 0
    rng = np.random.default_rng(13)
    x.values[:] = rng.integers(0, 256, size=x.values.shape, dtype=np.uint8)
    d.values.copy_(torch.from_numpy(x.values))
    out[3].zero_()
    mgt.transpose_values(plan, d.arrays(), out, ws)
    torch.cuda.synchronize()
    got = (*[t.cpu().numpy() for t in out], 0, plan)
    assert_same_as_oracle(x, got, oracle.transpose(x))
    # the way back once in full, then value-only round trips
    t = mgt.DeviceXCSR(d.n_cols, d.n_rows, d.offset_bytes, d.stride, out[0], out[1], out[2], out[3],
                       d.part_off)
    back_plan = mgt.plan_for(t, cfg)
    back_ws = mgt.alloc_workspace(back_plan.workspace_bytes)
    back = mgt.alloc_output(t)
    mgt.transpose(back_plan, t.arrays(), back, back_ws)
    original = d.values.clone()
    for _ in range(6):
        mgt.transpose_values(plan, d.arrays(), out, ws)            # M -> M^T
        mgt.transpose_values(back_plan, t.arrays(), back, back_ws)  # M^T -> M
        d.values.copy_(back[3])
    torch.cuda.synchronize()
    assert torch.equal(d.values, original)


def test_paper_benchmark_shapes_small():
    """The paper's two benchmark shapes (Sec. 5) at small scale: few long
    rows of uniform columns with 128-byte values, and its transpose (few
    columns holding huge runs of cells: the chunked path everywhere); 512
    cells per row of 10 four-byte values."""
    x = synth.generate(synth.paper_heterogeneous(seed=7, rows=8, cols=50_000, lo=3_000, hi=20_000))
    ref = oracle.transpose(x)
    assert_same_as_oracle(x, gpu_transpose(x), ref)
    xt = synth.from_arrays(ref.row_ptr, ref.col_idx, ref.cell_ptr, ref.values, x.n_rows, x.stride)
    back = gpu_transpose(xt)
    assert_same_as_oracle(xt, back, oracle.transpose(xt))
    assert np.array_equal(back[1], x.col_idx) and np.array_equal(back[3], x.values)
    y = synth.generate(synth.paper_balanced(seed=8, n=2048, parts=4))
    assert_same_as_oracle(y, gpu_transpose(y), oracle.transpose(y))


@pytest.mark.parametrize("P", [3, 64])
def test_null_part_off_means_equal_blocks(P):
    """mgt_desc.part_off = NULL with n_parts = P > 1 means P equal blocks,
    off[d] = floor(d R / P): called straight through the C ABI (the binding
    always passes explicit offsets) and compared with the oracle given those
    offsets, P x P counts included."""
    import ctypes
    import torch
    from paper_2012_06012_gb300 import mgt
    x = synth.generate(synth.heterogeneous(seed=41, n=9_999, parts=1))
    R = x.n_rows
    off = np.array([(d * R) // P for d in range(P + 1)], dtype=np.int64)
    desc, _ = mgt.make_desc(x.n_rows, x.n_cols, x.n_cells, x.n_values, x.offset_bytes, x.stride)
    desc.n_parts = P  # part_off stays NULL
    L = mgt.lib()
    h, wsb = ctypes.c_void_p(), ctypes.c_size_t()
    assert L.mgt_plan(ctypes.byref(desc), ctypes.byref(h), ctypes.byref(wsb)) == mgt.MGT_OK
    try:
        d = mgt.to_device(x)
        ws = mgt.alloc_workspace(int(wsb.value))
        odt = torch.int32 if x.offset_bytes == 4 else torch.int64
        out = (torch.empty(x.n_cols + 1, dtype=odt, device="cuda"),
               torch.empty(x.n_cells, dtype=torch.int32, device="cuda"),
               torch.empty(x.n_cells + 1, dtype=odt, device="cuda"),
               torch.empty(x.n_values * x.stride, dtype=torch.uint8, device="cuda"),
               torch.full((P * P,), -1, dtype=torch.int64, device="cuda"),
               torch.full((P * P,), -1, dtype=torch.int64, device="cuda"))
        xi = mgt.XcsrIn(*[mgt._ptr(t) for t in d.arrays()])
        xo = mgt.XcsrOut(*[mgt._ptr(t) for t in out])
        rc = L.mgt_transpose(h, ctypes.byref(xi), ctypes.byref(xo), mgt._ptr(ws),
                             ws.numel(), mgt._stream_handle(None))
        assert rc == mgt.MGT_OK
        assert mgt.read_status(ws) == mgt.MGT_OK
        ref = oracle.transpose(x, part_off=off)
        got = [t.cpu().numpy() for t in out]
        assert np.array_equal(got[0], ref.row_ptr)
        assert np.array_equal(got[1], ref.col_idx)
        assert np.array_equal(got[2], ref.cell_ptr)
        assert np.array_equal(got[3], ref.values)
        assert np.array_equal(got[4].reshape(P, P), ref.part_cells)
        assert np.array_equal(got[5].reshape(P, P), ref.part_values)
    finally:
        L.mgt_plan_destroy(h)


def _cut_blocks(n, P, seed, tiny_frac=0.3):
    """P row blocks over n rows: lognormal sizes with a share of empty and
    one-row blocks (tiles of the P x P output pass then span many blocks)."""
    rng = np.random.default_rng(seed)
    w = rng.lognormal(0.0, 2.0, size=P)
    w[rng.random(P) < tiny_frac] = 0.0
    cum = np.concatenate([[0.0], np.cumsum(w)])
    off = np.round(n * cum / cum[-1]).astype(np.int64)
    off[0], off[-1] = 0, n
    return np.maximum.accumulate(off)


@pytest.mark.parametrize("P,offset_bytes", [(2048, 8), (2048, 4), (2049, 8), (700, 8), (5, 4)])
def test_part_counts_block_layouts(P, offset_bytes):
    """P x P counts from the output pass (up to 2,048 blocks; above that the
    scatter pass counts) with empty and one-row blocks, so that tiles of
    output cells span more than the pass's window of destination blocks."""
    n = 60_000
    sp = synth.heterogeneous(seed=61 + P, n=n, parts=1)
    sp.offset_bytes = offset_bytes
    x = synth.generate(sp)
    x.part_off = _cut_blocks(n, P, seed=P)
    assert len(x.part_off) == P + 1
    assert_same_as_oracle(x, gpu_transpose(x), oracle.transpose(x))


@pytest.mark.parametrize("n", [262_144, 262_147], ids=["B-multiple-of-4", "B-ragged"])
def test_count_matrix_of_many_tiles(n):
    """More than 4,096 tiles of 2,048 cells: the tile scan gives each lane four
    neighbouring buckets (16-byte loads when the bucket count is a multiple of
    4, single loads with a ragged last group otherwise)."""
    x = synth.generate(synth.balanced(seed=9, n=n, parts=4, vals=1))
    cfg = {"scatter_tile": 2048, "bucket_shift": 7}
    assert x.n_cells // 2048 >= 4096
    assert_same_as_oracle(x, gpu_transpose(x, cfg), oracle.transpose(x))


@pytest.mark.parametrize("cfg", [None, {"bucket_shift": 4, "scatter_tile": 2048}], ids=["default", "two-pass"])
def test_blocks_on_super_bucket_boundaries(cfg):
    """Row blocks that start on super-bucket boundaries: the scatter pass counts
    P x P per tile and super-bucket (no cell's super-bucket spans two blocks)."""
    x = synth.generate(synth.balanced(seed=10, n=1 << 17, parts=16))
    assert_same_as_oracle(x, gpu_transpose(x, cfg), oracle.transpose(x))
