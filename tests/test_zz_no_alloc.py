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
