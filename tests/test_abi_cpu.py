"""The C-ABI library without a GPU: it loads, exports every symbol the
public headers declare, and its host-side planning validates descriptors."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2012_06012_gb300 import build as mgt_build
    mgt_build.build()
    from paper_2012_06012_gb300 import mgt
    return mgt.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(mgt_[a-z_0-9]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("mgt_plan", "mgt_transpose", "mgt_transpose_batched", "mgt_read_status"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_names_match_header(lib):
    from paper_2012_06012_gb300 import mgt
    assert set(mgt.EXPORTS) <= set(declared_functions())


def test_version_and_strerror(lib):
    from paper_2012_06012_gb300 import mgt
    assert "sm_103a" in mgt.version()
    for code in range(0, -9, -1):
        assert mgt.strerror(code)
    assert mgt.strerror(-99) == "unknown error"


def _plan(**kw):
    from paper_2012_06012_gb300 import mgt
    base = dict(n_rows=1000, n_cols=1000, n_cells=8000, n_values=32000, offset_bytes=4,
                payload_stride=8)
    base.update(kw)
    part_off = base.pop("part_off", None)
    cfg = base.pop("cfg", None)
    return mgt.Plan(part_off=part_off, cfg=cfg, **base)


def test_plan_on_host(lib):
    p = _plan(part_off=[0, 250, 500, 750, 1000])
    assert p.workspace_bytes > 0
    assert p.n_parts == 4
    cfg = p.config
    assert cfg["cluster"] in (1, 2, 4, 8) and cfg["chunk_cap"] % 512 == 0
    assert p.phases[0] == "setup" and p.phases[-1] == "copy"
    assert p.kernel_launches >= 6
    assert p.minimal_bytes() == (1001 * 4 + 4 * 8000 + 8001 * 4 + 32000 * 8) * 2


@pytest.mark.parametrize("bad", [
    dict(offset_bytes=2), dict(payload_stride=6), dict(payload_stride=0), dict(n_rows=-1),
    dict(n_cells=1 << 31, n_values=1 << 31), dict(part_off=[0, 600, 500, 1000]),
    dict(part_off=[0, 500, 999]), dict(n_rows=1000, n_cols=999, part_off=[0, 500, 1000]),
    dict(n_rows=0, n_cols=10, n_cells=5), dict(cfg={"cluster": 3}),
    dict(cfg={"chunk_cap": 1000}), dict(cfg={"copy_unroll": 3}),
    dict(cfg={"scatter_tile": 100}),
])
def test_plan_rejects_bad_descriptors(lib, bad):
    from paper_2012_06012_gb300 import mgt
    with pytest.raises(mgt.MgtError) as e:
        _plan(**bad)
    assert e.value.code == mgt.MGT_EINVAL


def test_plan_tile_heuristic_shapes(lib):
    from paper_2012_06012_gb300 import mgt
    # balanced 4M x 4M, 32 cells/row: every bucket fits one 8-CTA cluster
    p = mgt.Plan(4194304, 4194304, 134217728, 536870912, 8, 8,
                 part_off=np.arange(0, 4194305, 65536))
    c = p.config
    w = 1 << c["bucket_shift"]
    assert 32 * w <= 0.8 * c["cluster"] * c["chunk_cap"]
    # explicit tiles are honoured
    q = mgt.Plan(1000, 1000, 8000, 32000, 4, 8,
                 cfg={"cluster": 2, "chunk_cap": 1024, "bucket_shift": 5, "scatter_tile": 2048})
    assert q.config["cluster"] == 2 and q.config["chunk_cap"] == 1024
    assert q.config["bucket_shift"] == 5 and q.config["scatter_tile"] == 2048


def test_transpose_argument_checks_without_gpu(lib):
    """Argument validation happens before any device work."""
    from paper_2012_06012_gb300 import mgt
    p = _plan()
    xi = mgt.XcsrIn(None, None, None, None)
    xo = mgt.XcsrOut(None, None, None, None, None, None)
    rc = lib.mgt_transpose(p.handle, ctypes.byref(xi), ctypes.byref(xo), None, 0, None)
    assert rc == mgt.MGT_EINVAL
    rc = lib.mgt_transpose(p.handle, ctypes.byref(xi), ctypes.byref(xo), ctypes.c_void_p(256), 0, None)
    assert rc == mgt.MGT_ENOMEM


def test_host_transpose_argument_checks_without_gpu(lib):
    """mgt_transpose_host validates its arguments before any CUDA call."""
    from paper_2012_06012_gb300 import mgt
    p = _plan()
    hi = mgt.XcsrIn(None, None, None, None)
    ho = mgt.XcsrOut(None, None, None, None, None, None)
    di = mgt.XcsrBuf(None, None, None, None)
    do = mgt.XcsrOut(None, None, None, None, None, None)
    args = (ctypes.byref(hi), ctypes.byref(ho), ctypes.byref(di), ctypes.byref(do))
    assert lib.mgt_transpose_host(None, *args, ctypes.c_void_p(256), 1 << 40, None, None) == mgt.MGT_EINVAL
    assert lib.mgt_transpose_host(p.handle, None, ctypes.byref(ho), ctypes.byref(di), ctypes.byref(do),
                                  ctypes.c_void_p(256), 1 << 40, None, None) == mgt.MGT_EINVAL
    assert lib.mgt_transpose_host(p.handle, *args, ctypes.c_void_p(256), 0, None, None) == mgt.MGT_ENOMEM
    # device buffers present, host arrays missing
    fake = [ctypes.c_void_p(4096 * (k + 1)) for k in range(6)]
    di = mgt.XcsrBuf(*fake[:4])
    do = mgt.XcsrOut(*fake[:4], None, None)
    rc = lib.mgt_transpose_host(p.handle, ctypes.byref(hi), ctypes.byref(ho), ctypes.byref(di),
                                ctypes.byref(do), ctypes.c_void_p(256), 1 << 40, None, None)
    assert rc == mgt.MGT_EINVAL


def test_autotune_candidates_are_valid_plans(lib):
    from paper_2012_06012_gb300 import mgt
    import synth
    x = synth.generate(synth.balanced(seed=1, n=20_000, parts=8))
    cands = mgt.autotune_candidates(x)
    assert 4 <= len(cands) <= 64
    default = mgt.plan_for(x).config
    # the default plan's complete shape is always among them, so tuning can
    # only keep it or find a faster one
    assert cands[0] == default
    shapes = {(c["bucket_shift"], c["cluster"]) for c in cands}
    assert len(shapes) > 1
    for c in cands:
        p = mgt.plan_for(x, c)
        assert p.workspace_bytes > 0


@pytest.mark.parametrize("bad", [dict(max_slots=0), dict(n_streams=0), dict(max_queue=0),
                                 dict(batch_max=0), dict(hbm_budget_bytes=0),
                                 dict(n_streams=65), dict(batch_max=257),
                                 dict(batch_window_us=-1)])
def test_server_rejects_bad_config(lib, bad):
    from paper_2012_06012_gb300 import mgt
    kw = dict(hbm_budget_bytes=1 << 30, max_slots=4, n_streams=2, max_queue=8, batch_max=4)
    kw.update(bad)
    with pytest.raises(mgt.MgtError) as e:
        mgt.Server(**kw)
    assert e.value.code == mgt.MGT_EINVAL


def test_tune_cache_file_round_trip(lib, tmp_path):
    """A tuned shape written to the cache file comes back in a new cache, and
    the stored shapes are valid plans."""
    from paper_2012_06012_gb300 import mgt
    path = str(tmp_path / "tune.json")
    c = mgt.TuneCache(path=path)
    base = dict(n_rows=4096, n_cols=4096, n_cells=65536, n_values=262144, offset_bytes=8,
                payload_stride=16)
    cfg = mgt.Plan(**base, cfg={"cluster": 2, "chunk_cap": 1024, "bucket_shift": 5}).config
    key = (8, 16, False, 12, 4)
    c.best[key] = cfg
    c.save()
    d = mgt.TuneCache(path=path)
    assert d.best == {key: cfg}
    p = mgt.Plan(**base, cfg=d.best[key])
    assert p.config == cfg
    # no file: nothing is written
    e = mgt.TuneCache(path="")
    e.best[key] = cfg
    e.save()
    assert not (tmp_path / "").joinpath("tune.json.tmp").exists()


def test_host_pointer_marshalling():
    """The host-buffer call takes the caller's memory as is: contiguous arrays
    only (a hidden copy could be freed before an asynchronous copy reads it)."""
    import torch
    from paper_2012_06012_gb300 import mgt
    a = np.arange(32, dtype=np.int64)
    assert mgt._hptr(a).value == a.ctypes.data
    t = torch.arange(16, dtype=torch.int32)
    assert mgt._hptr(t).value == t.data_ptr()
    assert mgt._hptr(None) is None
    with pytest.raises(ValueError):
        mgt._hptr(a[::2])
    with pytest.raises(ValueError):
        mgt._hptr(t[::2])


def test_host_transpose_refuses_wrong_sizes(lib):
    """The library copies exactly the plan's sizes through raw host pointers,
    so the binding refuses, before any call, a host array that is too short
    or has the wrong offset width (it would be read or written past its end)."""
    from paper_2012_06012_gb300 import mgt
    R = N = 50
    C, V, s = 200, 600, 8
    p = mgt.Plan(R, N, C, V, 8, s)
    good_in = [np.zeros(R + 1, np.int64), np.zeros(C, np.int32), np.zeros(C + 1, np.int64),
               np.zeros(V * s, np.uint8)]
    good_out = [np.zeros(N + 1, np.int64), np.zeros(C, np.int32), np.zeros(C + 1, np.int64),
                np.zeros(V * s, np.uint8), np.zeros(1, np.int64), np.zeros(1, np.int64)]
    mgt.check_arrays(p, good_in, good_out, device=False)   # accepted
    raw_in = [np.zeros(a.nbytes, np.uint8) for a in good_in]
    mgt.check_arrays(p, raw_in, None, device=False)         # raw byte buffers too
    bad_cases = [
        (0, np.zeros(R, np.int64)),            # one entry short
        (0, np.zeros(2 * (R + 1), np.int32)),  # right bytes, 4-byte offsets for an 8-byte plan
        (1, np.zeros(C - 1, np.int32)),
        (2, np.zeros(C + 1, np.int32)),        # int32 cell_ptr with 8-byte offsets
        (3, np.zeros(V * s - 1, np.uint8)),
    ]
    for k, arr in bad_cases:
        ins = list(good_in)
        ins[k] = arr
        with pytest.raises(ValueError):
            mgt.check_arrays(p, ins, good_out, device=False)
        with pytest.raises(ValueError):  # the call itself refuses before touching the library
            mgt.transpose_host(p, ins, good_out, [None] * 4, [None] * 6, None)
    for k in range(4):
        outs = list(good_out)
        outs[k] = outs[k][:-1]
        with pytest.raises(ValueError):
            mgt.check_arrays(p, good_in, outs, device=False)
    outs = list(good_out)
    outs[4] = np.zeros(0, np.int64)  # P x P arrays shorter than P * P
    with pytest.raises(ValueError):
        mgt.check_arrays(p, good_in, outs, device=False)
    outs[4] = None  # optional
    outs[5] = None
    mgt.check_arrays(p, good_in, outs, device=False)
    with pytest.raises(ValueError):  # device arrays where host ones are expected
        import torch
        mgt.check_arrays(p, [torch.zeros(R + 1, dtype=torch.int64)], None, device=True)


def test_var_width_descriptors(lib):
    """MGT_FLAG_VAR_WIDTH plans need payload_stride 1; unknown flags are
    refused; batches and the static entry point refuse such plans; the
    minimal-byte count takes the value offsets (the byte count is added by
    the caller)."""
    import ctypes
    from paper_2012_06012_gb300 import mgt
    R, C, V = 100, 700, 2000
    p = mgt.Plan(R, R, C, V, 8, 1, var_width=True)
    assert p.workspace_bytes > mgt.Plan(R, R, C, V, 8, 4).workspace_bytes  # run sizes and tile sums
    for stride, flags in ((4, mgt.MGT_FLAG_VAR_WIDTH), (1, 0), (4, 2)):
        d, _ = mgt.make_desc(R, R, C, V, 8, stride, flags=flags)
        h, ws = ctypes.c_void_p(), ctypes.c_size_t()
        assert lib.mgt_plan(ctypes.byref(d), ctypes.byref(h), ctypes.byref(ws)) == mgt.MGT_EINVAL
    sz = ctypes.c_size_t()
    arr = (ctypes.c_void_p * 1)(p.handle)
    assert lib.mgt_batched_workspace(1, arr, ctypes.byref(sz)) == mgt.MGT_EINVAL
    d, _ = mgt.make_desc(R, R, C, V, 8, 1, flags=mgt.MGT_FLAG_VAR_WIDTH)
    xi = mgt.XcsrIn(None, None, None, None)
    xo = mgt.XcsrOut(None, None, None, None, None, None)
    assert lib.mgt_transpose_static(ctypes.byref(d), ctypes.byref(xi), ctypes.byref(xo), None) == mgt.MGT_EINVAL
    side = 4 * C + (C + 1) * 8 + 8 * (V + 1)
    assert lib.mgt_minimal_bytes(ctypes.byref(d)) == (R + 1) * 8 + side + (R + 1) * 8 + side
