"""Guard words around every output array and the workspace: a transpose
writes exactly inside its buffers (no byte before or after any of them
changes) on the shapes that exercise each kernel path, and its result still
equals the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from helpers import assert_same_as_oracle, gpu_available, random_small

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

GUARD = 4096
PATTERN = 0xA5


def _guarded(nbytes, dtype):
    """(whole buffer, view of nbytes in its middle as dtype)."""
    import torch
    buf = torch.full((2 * GUARD + nbytes,), PATTERN, dtype=torch.uint8, device="cuda")
    return buf, buf[GUARD:GUARD + nbytes].view(dtype)


def _guards_intact(buf, nbytes):
    import torch
    head = buf[:GUARD]
    tail = buf[GUARD + nbytes:]
    return bool(torch.all(head == PATTERN)) and bool(torch.all(tail == PATTERN))


CASES = {
    "tiny": (lambda: synth.generate(synth.tiny(seed=0)), None),
    "heterogeneous-chunked": (lambda: synth.generate(synth.heterogeneous(seed=2, n=30_011, parts=16)),
                              {"cluster": 1, "chunk_cap": 512, "scatter_tile": 1024}),
    "zipf-head-cs8": (lambda: synth.generate(synth.heterogeneous(seed=3, n=65_536, parts=32, perm=0)),
                      {"cluster": 8, "chunk_cap": 512, "bucket_shift": 3}),
    "unsorted-duplicates": (lambda: random_small(61, 300, 300, max_cells=40, sorted_rows=False,
                                                 dup_cols=True, n_parts=5, stride=12), None),
    "long-runs": (lambda: synth.from_arrays(
        np.array([0, 2, 4, 7], np.int64), np.array([1, 0, 2, 0, 1, 2, 0], np.int32),
        np.concatenate([[0], np.cumsum([3, 70_000, 0, 65_535, 65_534, 1, 131_072])]).astype(np.int64),
        np.random.default_rng(5).integers(0, 255, size=332_145 * 4, dtype=np.uint8), 3, 4), None),
}


@pytest.mark.parametrize("case", list(CASES))
def test_writes_stay_inside_buffers(case):
    import torch
    from paper_2012_06012_gb300 import mgt
    make, cfg = CASES[case]
    x = make()
    d = mgt.to_device(x)
    plan = mgt.plan_for(d, cfg)
    odt = torch.int32 if x.offset_bytes == 4 else torch.int64
    o = x.offset_bytes
    C, V = len(x.col_idx), len(x.values) // x.stride
    P = len(x.part_off) - 1
    sizes = [((x.n_cols + 1) * o, odt), (C * 4, torch.int32), ((C + 1) * o, odt),
             (V * x.stride, torch.uint8), (P * P * 8, torch.int64), (P * P * 8, torch.int64)]
    bufs, views = zip(*[_guarded(n, t) for n, t in sizes])
    wbuf, ws = _guarded(plan.workspace_bytes, torch.uint8)
    mgt.transpose(plan, d.arrays(), tuple(views), ws)
    status = mgt.read_status(ws)
    torch.cuda.synchronize()
    got = (*[v.cpu().numpy() for v in views], status, plan)
    assert_same_as_oracle(x, got, oracle.transpose(x))
    for (n, _), b in zip(sizes, bufs):
        assert _guards_intact(b, n)
    assert _guards_intact(wbuf, plan.workspace_bytes)
