"""Malformed inputs are detected on the device: the kernels clamp every
index they derive from the input, flag the workspace status and place
nothing, so the call reports MGT_EBADINPUT and the context stays usable."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from helpers import assert_same_as_oracle, gpu_available, gpu_transpose, random_small

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def _base(seed=3):
    return random_small(seed, 400, 400, max_cells=20, n_parts=4, stride=8)


def _with(x, **arrays):
    d = dict(row_ptr=x.row_ptr.copy(), col_idx=x.col_idx.copy(), cell_ptr=x.cell_ptr.copy(),
             values=x.values.copy())
    d.update(arrays)
    return synth.from_arrays(d["row_ptr"], d["col_idx"], d["cell_ptr"], d["values"], x.n_cols,
                             x.stride, x.part_off)


def _cases():
    x = _base()
    C = x.n_cells
    out = []
    col = x.col_idx.copy(); col[C // 2] = x.n_cols; out.append(("col == n_cols", _with(x, col_idx=col)))
    col = x.col_idx.copy(); col[0] = -1; out.append(("col < 0", _with(x, col_idx=col)))
    col = x.col_idx.copy(); col[-1] = 2**31 - 1; out.append(("col huge", _with(x, col_idx=col)))
    rp = x.row_ptr.copy(); mid = len(rp) // 2; rp[mid] = rp[mid + 1] + 3
    out.append(("row_ptr decreasing", _with(x, row_ptr=rp)))
    rp = x.row_ptr.copy(); rp[-1] = C - 1; out.append(("row_ptr[R] != C", _with(x, row_ptr=rp)))
    cp = x.cell_ptr.copy(); cp[C // 3] = cp[C // 3 + 1] + 5
    out.append(("cell_ptr decreasing", _with(x, cell_ptr=cp)))
    cp = x.cell_ptr.copy(); cp[-1] = cp[-1] - 1; out.append(("cell_ptr[C] != V", _with(x, cell_ptr=cp)))
    return out


@pytest.mark.parametrize("cfg", [None, {"cluster": 1, "chunk_cap": 512, "scatter_tile": 1024}],
                         ids=["default", "small-tiles"])
def test_malformed_inputs_are_flagged(cfg):
    from paper_2012_06012_gb300 import mgt
    for name, y in _cases():
        got = gpu_transpose(y, cfg)
        assert got[6] == mgt.MGT_EBADINPUT, f"{name}: status {got[6]}"
    # the context is still healthy: a valid transpose right after
    x = _base()
    assert_same_as_oracle(x, gpu_transpose(x, cfg), oracle.transpose(x))
