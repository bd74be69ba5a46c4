"""The allocation-free entry point, mgt_transpose_static.

It serves callers that cannot allocate device memory (a plug-in whose host
framework owns every device allocation, or a loop that cannot afford the
implicit synchronisation of cudaMalloc/cudaFree): its scratch is a fixed
64 MiB array inside the library.  These tests call it through the C ABI and
compare its output with the ordinary entry point's (bit for bit, the
tolerance every parity test here uses) on two calls in a row, so that state
left in the shared array by one call cannot leak into the next.  The file
is collected last so that a run stopping at the first failure has already
run everything else.
"""
from __future__ import annotations

import numpy as np
import pytest

import synth
from helpers import gpu_available


def _run_both(x):
    import torch
    from paper_2012_06012_gb300 import mgt
    d = mgt.to_device(x)
    ref, _, _ = mgt.transpose_device(d)
    out = mgt.alloc_output(d, parts=True)
    for t in out:
        t.fill_(0x5A if t.dtype == torch.uint8 else -7)
    mgt.transpose_static(d, d.arrays(), out)
    st = mgt.static_status()
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in ref], [t.cpu().numpy() for t in out], st


@pytest.mark.gpu
@pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")
def test_static_entry_matches_ordinary_entry_twice():
    first = synth.generate(synth.heterogeneous(seed=11, n=20_000, parts=8))
    second = synth.generate(synth.tiny(seed=12))
    for x in (first, second):
        ref, got, st = _run_both(x)
        assert st == 0
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)


@pytest.mark.gpu
@pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")
def test_static_entry_many_unequal_row_blocks():
    """About a thousand unequal row blocks: the entry point sends the block
    offsets to the device in several kernel-parameter chunks (480 offsets
    each), so this covers every chunk boundary; compared bit for bit with
    the ordinary entry point, P x P counts included, twice in a row."""
    rng = np.random.default_rng(5)
    n, P = 4_000, 1_003
    cuts = np.sort(rng.choice(np.arange(1, n), size=P - 1, replace=False))
    cuts[rng.integers(0, P - 1, size=40)] = cuts[0]  # some empty blocks
    part_off = np.concatenate([[0], np.sort(cuts), [n]]).astype(np.int64)
    for seed in (31, 32):
        x = synth.generate(synth.heterogeneous(seed=seed, n=n, parts=1))
        x.part_off = part_off
        ref, got, st = _run_both(x)
        assert st == 0
        assert got[4].shape == (P * P,)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b)


@pytest.mark.gpu
@pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")
def test_static_entry_null_part_off_equal_blocks():
    """part_off = NULL with n_parts > 1 (equal blocks) through the C ABI,
    against the ordinary entry point given the same blocks explicitly."""
    import ctypes
    import torch
    from paper_2012_06012_gb300 import mgt
    x = synth.generate(synth.heterogeneous(seed=33, n=6_000, parts=1))
    P = 600
    x.part_off = np.array([(d * x.n_rows) // P for d in range(P + 1)], dtype=np.int64)
    d = mgt.to_device(x)
    ref, _, _ = mgt.transpose_device(d)
    out = mgt.alloc_output(d, parts=True)
    desc, _ = mgt.make_desc(x.n_rows, x.n_cols, x.n_cells, x.n_values, x.offset_bytes, x.stride)
    desc.n_parts = P  # part_off stays NULL
    xi = mgt.XcsrIn(*[mgt._ptr(t) for t in d.arrays()])
    xo = mgt.XcsrOut(*[mgt._ptr(t) for t in out])
    rc = mgt.lib().mgt_transpose_static(ctypes.byref(desc), ctypes.byref(xi), ctypes.byref(xo),
                                        mgt._stream_handle(None))
    assert rc == mgt.MGT_OK
    assert mgt.static_status() == 0
    torch.cuda.synchronize()
    for a, b in zip(ref, out):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_static_entry_rejects_too_large():
    """A matrix whose workspace exceeds the fixed array is refused before any
    device work (no GPU needed)."""
    import ctypes
    from paper_2012_06012_gb300 import build as mgt_build
    from paper_2012_06012_gb300 import mgt
    mgt_build.build()
    desc, _ = mgt.make_desc(4_194_304, 4_194_304, 134_217_728, 536_870_912, 8, 8)
    xi = mgt.XcsrIn(None, None, None, None)
    xo = mgt.XcsrOut(None, None, None, None, None, None)
    rc = mgt.lib().mgt_transpose_static(ctypes.byref(desc), ctypes.byref(xi), ctypes.byref(xo), None)
    assert rc == mgt.MGT_ENOMEM
