"""Batched transposes (one launch per phase over many matrices, and the same
captured in a CUDA graph): every member equals the oracle and the
single-matrix call, bit for bit, in mixed batches that span several launch
groups, empty members and ragged sizes."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import assert_same_as_oracle, gpu_available, random_small

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def _members():
    xs = []
    xs.append(synth.generate(synth.tiny(seed=0)))
    xs.append(synth.generate(synth.balanced(seed=1, n=20_011, parts=8)))
    xs.append(synth.generate(synth.heterogeneous(seed=2, n=12_289, parts=16)))
    for k in range(6):
        xs.append(synth.generate(synth.batched_member(seed=3, m=k, rows_hi=40_000)))
    xs.append(random_small(41, 300, 300, max_cells=40, n_parts=5, stride=8, sorted_rows=False,
                           dup_cols=True))
    xs.append(random_small(42, 1000, 37, max_cells=30, stride=12))
    # empty matrix and a single cell
    xs.append(synth.from_arrays(np.zeros(8, np.int64), np.zeros(0, np.int32), np.zeros(1, np.int64),
                                np.zeros(0, np.uint8), 5, 8))
    xs.append(synth.from_arrays(np.array([0, 1], np.int64), np.array([0], np.int32),
                                np.array([0, 3], np.int64), np.arange(3, dtype=np.int64).view(np.uint8),
                                1, 8))
    return xs


# tile configurations that put members into different launch groups
CFGS = [None, {"cluster": 2, "chunk_cap": 1024, "bucket_shift": 5, "copy_unroll": 4},
        {"cluster": 1, "chunk_cap": 512, "scatter_tile": 1024, "copy_unroll": 1}]


def _setup(xs, cfg_of):
    from paper_2012_06012_gb300 import mgt
    devs = [mgt.to_device(x) for x in xs]
    plans = [mgt.plan_for(d, cfg_of(i)) for i, d in enumerate(devs)]
    outs = [mgt.alloc_output(d) for d in devs]
    ws = mgt.alloc_workspace(mgt.batched_workspace(plans))
    return devs, plans, outs, ws


def _got(out, plan, status=0):
    """In the shape assert_same_as_oracle takes."""
    return (*[t.cpu().numpy() if t is not None else None for t in out], status, plan)


@pytest.mark.parametrize("mixed", [False, True], ids=["one-group", "three-groups"])
def test_batched_matches_oracle_and_single(mixed):
    from paper_2012_06012_gb300 import mgt
    xs = _members()
    devs, plans, outs, ws = _setup(xs, (lambda i: CFGS[i % 3]) if mixed else (lambda i: None))
    mgt.transpose_batched(plans, [d.arrays() for d in devs], outs, ws)
    torch.cuda.synchronize()
    for x, d, p, o in zip(xs, devs, plans, outs):
        assert_same_as_oracle(x, _got(o, p), oracle.transpose(x))
        single, _, _ = mgt.transpose_device(d, plan=p)
        for a, b in zip(o, single):
            if a is not None:
                assert torch.equal(a, b)


def test_batch_graph_replays_and_recomputes():
    from paper_2012_06012_gb300 import mgt
    xs = _members()
    devs, plans, outs, ws = _setup(xs, lambda i: CFGS[i % 3])
    b = mgt.Batch(plans, [d.arrays() for d in devs], outs, ws)
    assert b.kernel_launches >= 10
    for _ in range(2):
        b.launch()
    assert b.status() == [0] * len(xs)
    for x, p, o in zip(xs, plans, outs):
        assert_same_as_oracle(x, _got(o, p), oracle.transpose(x))
    # new payloads in place: the replay recomputes from the bound inputs
    rng = np.random.default_rng(7)
    for x, d in zip(xs, devs):
        x.values[:] = rng.integers(0, 256, size=x.values.shape, dtype=np.uint8)
        d.values.copy_(torch.from_numpy(x.values))
    for o in outs:
        o[3].zero_()
    b.launch()
    torch.cuda.synchronize()
    for x, p, o in zip(xs, plans, outs):
        assert_same_as_oracle(x, _got(o, p), oracle.transpose(x))
    b.close()


def test_batched_rejects_small_workspace():
    from paper_2012_06012_gb300 import mgt
    xs = _members()[:3]
    devs, plans, outs, ws = _setup(xs, lambda i: None)
    with pytest.raises(mgt.MgtError) as e:
        mgt.transpose_batched(plans, [d.arrays() for d in devs], outs, ws[: ws.numel() // 2])
    assert e.value.code == mgt.MGT_ENOMEM
