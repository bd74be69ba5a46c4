"""The transpose of matrices held in host memory (mgt_transpose_host): host
to device copies, the transpose and the device to host copies in one call,
with and without a second stream for the overlapped copies, pinned and
pageable host arrays, and two alternating buffer sets as a pipelined caller
uses them.  Every output equals the oracle bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from helpers import assert_same_as_oracle, gpu_available, random_small

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def _host_out(x, pinned):
    import torch
    odt = np.int32 if x.offset_bytes == 4 else np.int64
    P = len(x.part_off) - 1
    shapes = [(x.n_cols + 1, odt), (len(x.col_idx), np.int32), (len(x.col_idx) + 1, odt),
              (len(x.values), np.uint8), (P * P, np.int64), (P * P, np.int64)]
    if pinned:
        tdt = {np.int32: torch.int32, np.int64: torch.int64, np.uint8: torch.uint8}
        ts = [torch.empty(n, dtype=tdt[d], pin_memory=True) for n, d in shapes]
        return ts, [t.numpy() for t in ts]
    arrs = [np.empty(n, dtype=d) for n, d in shapes]
    return arrs, arrs


def _host_in(x, pinned):
    import torch
    arrs = [x.row_ptr, x.col_idx, x.cell_ptr, x.values]
    if not pinned:
        return [np.ascontiguousarray(a) for a in arrs]
    return [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in arrs]


def _device_set(x):
    import torch
    from paper_2012_06012_gb300 import mgt
    d = mgt.DeviceXCSR(x.n_rows, x.n_cols, x.offset_bytes, x.stride,
                       *[torch.empty(a.shape, dtype=torch.from_numpy(a[:0]).dtype, device="cuda")
                         for a in (x.row_ptr, x.col_idx, x.cell_ptr, x.values)], x.part_off)
    return d, mgt.alloc_output(d, parts=True)


def _check(x, host_np, plan, ws):
    from paper_2012_06012_gb300 import mgt
    got = (*host_np, mgt.read_status(ws), plan)
    assert_same_as_oracle(x, got, oracle.transpose(x))


CASES = {
    "heterogeneous": lambda: synth.generate(synth.heterogeneous(seed=21, n=20_000, parts=8)),
    "balanced": lambda: synth.generate(synth.balanced(seed=22, n=8_192, parts=4)),
    "random-unsorted": lambda: random_small(23, 400, 400, max_cells=30, sorted_rows=False,
                                            n_parts=5, stride=12),
    "empty": lambda: synth.from_arrays(np.zeros(8, np.int64), np.zeros(0, np.int32),
                                       np.zeros(1, np.int64), np.zeros(0, np.uint8), 5, 8),
}


@pytest.mark.parametrize("overlap", [False, True], ids=["one-stream", "copy-stream"])
@pytest.mark.parametrize("pinned", [True, False], ids=["pinned", "pageable"])
@pytest.mark.parametrize("case", list(CASES))
def test_host_transpose_matches_oracle(case, pinned, overlap):
    import torch
    from paper_2012_06012_gb300 import mgt
    x = CASES[case]()
    d, out = _device_set(x)
    plan = mgt.plan_for(d)
    ws = mgt.alloc_workspace(plan.workspace_bytes)
    h_in = _host_in(x, pinned)
    h_out, h_np = _host_out(x, pinned)
    cs = torch.cuda.Stream() if overlap else None
    mgt.transpose_host(plan, h_in, h_out, d.arrays(), out, ws, copy_stream=cs)
    torch.cuda.current_stream().synchronize()
    _check(x, h_np, plan, ws)


def test_two_alternating_buffer_sets():
    """A pipelined caller: two device buffer sets and stream pairs take the
    calls in turn, each call's downloads overlapping the next one's uploads;
    different matrices of the same shape go through the same plan."""
    import torch
    from paper_2012_06012_gb300 import mgt
    xs = [synth.generate(synth.balanced(seed=30 + k, n=16_384, parts=8)) for k in range(4)]
    lanes = []
    for _ in range(2):
        d, out = _device_set(xs[0])
        lanes.append((d, out, torch.cuda.Stream(), torch.cuda.Stream()))
    plan = mgt.plan_for(lanes[0][0])
    wss = [mgt.alloc_workspace(plan.workspace_bytes) for _ in lanes]
    results = []
    for k, x in enumerate(xs):
        d, out, st, cs = lanes[k % 2]
        h_out, h_np = _host_out(x, True)
        mgt.transpose_host(plan, _host_in(x, True), h_out, d.arrays(), out, wss[k % 2], stream=st,
                           copy_stream=cs)
        results.append((x, h_np, h_out))
    torch.cuda.synchronize()
    for k, (x, h_np, _) in enumerate(results):
        assert_same_as_oracle(x, (*h_np, 0, plan), oracle.transpose(x))
    assert all(mgt.read_status(w) == 0 for w in wss)
