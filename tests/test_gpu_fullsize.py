"""Parity at the benchmark's full sizes, element by element and bit for bit,
in the launch configurations the benchmark times:

* the balanced multigraph (4,194,304 x 4,194,304, 128M cells, 512M values,
  64 row blocks) and the heterogeneous matrix (8,388,608 x 8,388,608, ~168M
  cells, Zipf columns, 256 unequal row blocks), each with the default plan:
  every entry of row_ptr', col_idx', cell_ptr', values' and the P x P counts
  against the oracle's full transpose (the GPU's output is downloaded and
  compared in chunks; the oracle's output is held whole in host memory,
  about 60 GB for the heterogeneous matrix);
* the largest members of the batched workload (rows >= 1M, autotuned plans)
  transposed inside one batch, replayed from its CUDA graph, next to small
  members;
* a large request of the serving workload (4,194,304 rows, heterogeneous
  distributions) served in a mix with small requests;
* the heterogeneous matrix with values of individual byte widths (the
  variable-width workload), against the oracle's variable-width transpose.

These need a GPU machine with enough host memory; they skip when it has less."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

CHUNK = 1 << 28  # bytes per device-to-host comparison chunk


def _host_mem_gb() -> float:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) / 2**20
    except OSError:
        pass
    return 0.0


def _need_host_gb(gb: float):
    if _host_mem_gb() < gb:
        pytest.skip(f"needs about {gb:.0f} GB of free host memory")


def assert_equal_chunked(dev: torch.Tensor, ref: np.ndarray, what: str):
    """Every element of device tensor ``dev`` equals host array ``ref``
    (compared as raw bytes, in chunks of CHUNK bytes)."""
    a = dev.reshape(-1).view(torch.uint8)
    b = np.ascontiguousarray(ref).reshape(-1).view(np.uint8)
    assert a.numel() == b.shape[0], f"{what}: {a.numel()} bytes vs {b.shape[0]}"
    for lo in range(0, b.shape[0], CHUNK):
        hi = min(b.shape[0], lo + CHUNK)
        got = a[lo:hi].cpu().numpy()
        if not np.array_equal(got, b[lo:hi]):
            bad = lo + int(np.flatnonzero(got != b[lo:hi])[0])
            raise AssertionError(f"{what}: first difference at byte {bad} "
                                 f"(element {bad // ref.dtype.itemsize})")


def assert_output_equals_oracle(out, ref, P=None):
    assert_equal_chunked(out[0], ref.row_ptr, "row_ptr'")
    assert_equal_chunked(out[1], ref.col_idx, "col_idx'")
    assert_equal_chunked(out[2], ref.cell_ptr, "cell_ptr'")
    assert_equal_chunked(out[3], ref.values, "values'")
    if P is not None and out[4] is not None:
        assert np.array_equal(out[4].cpu().numpy().reshape(P, P), ref.part_cells), "P x P cells"
        assert np.array_equal(out[5].cpu().numpy().reshape(P, P), ref.part_values), "P x P values"


@pytest.mark.parametrize("workload,host_gb", [("balanced", 30), ("heterogeneous", 90)])
def test_full_size_parity(workload, host_gb):
    """The bench's matrices, every output element against the oracle's full
    transpose, with the default plan and with the plan the bench times (the
    library's autotuner run on the same matrix, as bench.py does)."""
    _need_host_gb(host_gb)
    from paper_2012_06012_gb300 import mgt
    spec = synth.balanced(seed=0) if workload == "balanced" else synth.heterogeneous(seed=0)
    x = synth.generate(spec)
    d = mgt.to_device(x)
    ref = oracle.transpose(x)
    del x
    P = ref.part_cells.shape[0]
    out, plan, ws = mgt.transpose_device(d)
    torch.cuda.synchronize()
    assert_output_equals_oracle(out, ref, P=P)
    del out, ws
    cfg, _ = mgt.autotune(d, reps=1)
    if cfg != plan.config:
        out, tuned, ws = mgt.transpose_device(d, plan=mgt.plan_for(d, cfg))
        torch.cuda.synchronize()
        assert_output_equals_oracle(out, ref, P=P)


def _largest_batched_members(k: int, min_rows: int = 1_000_000):
    """Indices of the k largest members (>= min_rows rows) of the batched
    workload, read from the member sizes alone (nothing generated)."""
    sizes = [(synth.batched_member(seed=0, m=m).n_rows, m) for m in range(512)]
    big = sorted([s for s in sizes if s[0] >= min_rows], reverse=True)[:k]
    return [m for _, m in big]


def test_batched_largest_members_in_a_batch():
    """The largest batched-workload members (up to 2M rows), with autotuned
    plans as the benchmark uses, transposed inside one batch together with
    small members and replayed from the batch's CUDA graph: every member
    equals the oracle."""
    _need_host_gb(40)
    from paper_2012_06012_gb300 import mgt
    big = _largest_batched_members(3)
    members = big + [m for m in range(16) if m not in big][:5]
    xs = [synth.generate(synth.batched_member(seed=0, m=m)) for m in members]
    assert max(x.n_rows for x in xs) >= 1_000_000
    devs = [mgt.to_device(x) for x in xs]
    tune = mgt.TuneCache(reps=1, path="")
    plans = [mgt.plan_for(d, tune.cfg_for(d)) for d in devs]
    outs = [mgt.alloc_output(d) for d in devs]
    for o in outs:
        for t in o:
            if t is not None:
                t.fill_(0x33 if t.dtype == torch.uint8 else -5)
    bws = mgt.alloc_workspace(mgt.batched_workspace(plans))
    batch = mgt.Batch(plans, [d.arrays() for d in devs], outs, bws)
    batch.launch()
    batch.launch()  # a replay recomputes everything from the inputs
    assert batch.status() == [0] * len(devs)
    torch.cuda.synchronize()
    for x, o in zip(xs, outs):
        ref = oracle.transpose(x)
        assert_output_equals_oracle(o, ref, P=1)
    batch.close()


def test_serving_large_request_in_a_mix():
    """A large request of the serving workload (4,194,304 rows, heterogeneous
    distributions: Zipf columns, geometric runs of 32-byte values) served
    through the request loop together with small batched-workload requests
    (some of them fused): every result equals the oracle."""
    _need_host_gb(50)
    from paper_2012_06012_gb300 import mgt
    large = synth.generate(synth.large_member(seed=2, m=0))
    small = [synth.generate(synth.batched_member(seed=1, m=m)) for m in range(6)]
    xs = [small[0], small[1], large, small[2], small[3], small[4], small[5]]
    devs = [mgt.to_device(x) for x in xs]
    plans = [mgt.plan_for(d) for d in devs]
    outs = [mgt.alloc_output(d) for d in devs]
    srv = mgt.Server(hbm_budget_bytes=180 * 10**9, max_slots=16, n_streams=4, batch_max=8,
                     fuse_max_cells=1 << 22)
    try:
        tickets = [srv.submit(p, d.arrays(), o) for p, d, o in zip(plans, devs, outs)]
        srv.drain()
        for t in tickets:
            done, st, _ = srv.poll(t)
            assert done and st == 0
    finally:
        srv.close()
    torch.cuda.synchronize()
    for x, o in zip(xs, outs):
        assert_output_equals_oracle(o, oracle.transpose(x), P=1)


def test_var_width_full_size():
    """The variable-width workload at full size (8,388,608 x 8,388,608, widths
    from 4 to 64 bytes, ~22 GB of value bytes): every output element and value
    offset against the oracle's variable-width transpose."""
    _need_host_gb(110)
    from paper_2012_06012_gb300 import mgt
    x = synth.generate_var(synth.heterogeneous(seed=0))
    d = mgt.to_device_var(x)
    plan = mgt.plan_for_var(d)
    ws = mgt.alloc_workspace(plan.workspace_bytes)
    out, ovo = mgt.alloc_output_var(d, parts=False)
    mgt.transpose_var(plan, d.arrays(), d.val_off, out, ovo, ws)
    assert mgt.read_status(ws) == 0
    torch.cuda.synchronize()
    del d, ws
    ref = oracle.transpose_var(x)
    del x
    assert_equal_chunked(out[0], ref.row_ptr, "row_ptr'")
    assert_equal_chunked(out[1], ref.col_idx, "col_idx'")
    assert_equal_chunked(out[2], ref.cell_ptr, "cell_ptr'")
    assert_equal_chunked(ovo, ref.val_off, "val_off'")
    assert_equal_chunked(out[3], ref.values, "values'")
