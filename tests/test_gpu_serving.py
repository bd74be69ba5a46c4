"""The serving loop: requests admitted by HBM footprint and run concurrently
(several streams, fused small launches) give, for every request, exactly the
result the request gets alone; the admitted footprint never exceeds the
budget; a full queue answers MGT_EAGAIN."""
from __future__ import annotations

import time

import numpy as np
import pytest
import torch

import oracle
import synth
from helpers import assert_same_as_oracle, gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def _mix(n_small=24):
    xs = [synth.generate(synth.batched_member(seed=5, m=k, rows_hi=30_000)) for k in range(n_small)]
    xs.insert(3, synth.generate(synth.heterogeneous(seed=6, n=40_000, parts=16)))
    xs.insert(11, synth.generate(synth.balanced(seed=7, n=30_000, parts=4)))
    xs.append(synth.generate(synth.tiny(seed=8)))
    return xs


def _wait_all(srv, tickets, timeout_s=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(tickets):
        for t in tickets:
            if t in res:
                continue
            done, st, lat = srv.poll(t)
            if done:
                res[t] = (st, lat)
        assert time.time() - t0 < timeout_s, "requests did not finish"
        time.sleep(0.001)
    return res


def _got(out, plan, status):
    return (*[t.cpu().numpy() if t is not None else None for t in out], status, plan)


@pytest.mark.parametrize("batch_max", [1, 8], ids=["no-fusion", "fused"])
def test_each_result_same_alone_and_in_the_mix(batch_max):
    from paper_2012_06012_gb300 import mgt
    xs = _mix()
    devs = [mgt.to_device(x) for x in xs]
    plans = [mgt.plan_for(d) for d in devs]
    srv = mgt.Server(hbm_budget_bytes=8 << 30, max_slots=16, n_streams=4, batch_max=batch_max,
                     fuse_max_cells=1 << 20, batch_window_us=20_000 if batch_max > 1 else 0)
    outs = [mgt.alloc_output(d) for d in devs]
    tickets = [srv.submit(p, d.arrays(), o) for p, d, o in zip(plans, devs, outs)]
    res = _wait_all(srv, tickets)
    torch.cuda.synchronize()
    st = srv.stats()
    assert st["completed"] == len(xs) and st["failed"] == 0
    assert st["peak_inflight_bytes"] <= 8 << 30
    if batch_max > 1:
        assert st["fused_requests"] > 0
    for x, d, p, o, t in zip(xs, devs, plans, outs, tickets):
        status, lat = res[t]
        assert lat > 0
        assert_same_as_oracle(x, _got(o, p, status), oracle.transpose(x))
        alone, _, _ = mgt.transpose_device(d, plan=p)
        for a, b in zip(o, alone):
            if a is not None:
                assert torch.equal(a, b)
    srv.close()


def test_admission_respects_budget_and_queue():
    from paper_2012_06012_gb300 import mgt
    xs = [synth.generate(synth.batched_member(seed=9, m=k, rows_lo=20_000, rows_hi=40_000))
          for k in range(12)]
    devs = [mgt.to_device(x) for x in xs]
    plans = [mgt.plan_for(d) for d in devs]
    fp = [p.workspace_bytes + p.minimal_bytes() for p in plans]
    budget = int(max(fp) * 1.5)  # at most one request of the largest size at once
    srv = mgt.Server(hbm_budget_bytes=budget, max_slots=8, n_streams=2, max_queue=4, batch_max=1)
    outs = [mgt.alloc_output(d) for d in devs]
    tickets, refused = [], 0
    for p, d, o in zip(plans, devs, outs):
        while True:
            try:
                tickets.append((srv.submit(p, d.arrays(), o), p, o))
                break
            except mgt.MgtError as e:
                assert e.code == mgt.MGT_EAGAIN
                refused += 1
                time.sleep(0.0005)
    res = _wait_all(srv, [t for t, _, _ in tickets])
    st = srv.stats()
    assert st["peak_inflight_bytes"] <= budget
    assert st["rejected"] == refused
    for x, (t, p, o) in zip(xs, tickets):
        assert_same_as_oracle(x, _got(o, p, res[t][0]), oracle.transpose(x))
    # a request that can never fit
    tiny = mgt.Server(hbm_budget_bytes=1024, max_slots=1, n_streams=1)
    with pytest.raises(mgt.MgtError) as e:
        tiny.submit(plans[0], devs[0].arrays(), outs[0])
    assert e.value.code == mgt.MGT_ENOMEM
    with pytest.raises(mgt.MgtError) as e:
        srv.poll(123456789)
    assert e.value.code == mgt.MGT_ENOTFOUND
    tiny.close()
    srv.close()


def test_autotuned_plan_gives_the_same_result():
    from paper_2012_06012_gb300 import mgt
    x = synth.generate(synth.heterogeneous(seed=10, n=30_000, parts=8))
    d = mgt.to_device(x)
    cfg, ms = mgt.autotune(d, reps=1)
    assert ms > 0
    p = mgt.plan_for(d, cfg)
    out, _, _ = mgt.transpose_device(d, plan=p)
    torch.cuda.synchronize()
    assert_same_as_oracle(x, _got(out, p, 0), oracle.transpose(x))
