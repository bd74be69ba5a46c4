"""The memory-system probe (mgt_probe_runs) moves the runs it claims to
move: each mode checked against plain tensor indexing on small buffers,
including a run count that leaves the last TMA chunk partial."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rb", [16, 32, 48, 128])
@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4, 5])
def test_probe_modes(mode, rb):
    from paper_2012_06012_gb300 import mgt
    g = torch.Generator(device="cpu").manual_seed(1000 * mode + rb)
    n = 70_001  # not a multiple of the TMA chunk (32 runs)
    src = torch.randint(0, 256, (n * rb,), dtype=torch.uint8, generator=g).cuda()
    dst = torch.zeros(n * rb, dtype=torch.uint8, device="cuda")
    perm = torch.randperm(n, generator=g).to(torch.int32).cuda()
    st = torch.cuda.current_stream()
    before = mgt.probe_errors()
    mgt.probe_runs(mode, src, dst, perm, n, rb, st)
    torch.cuda.synchronize()
    assert mgt.probe_errors() == before
    s, d, p = src.view(n, rb), dst.view(n, rb), perm.long()
    if mode in (0, 4, 5):
        assert torch.equal(d, s[p])
    elif mode == 1:
        want = torch.empty_like(s)
        want[p] = s
        assert torch.equal(d, want)
    elif mode == 2:
        got = dst[: 4 * n].view(torch.int32).long()
        want = torch.empty(n, dtype=torch.long, device="cuda")
        want[p] = torch.arange(n, device="cuda")
        assert torch.equal(got, want)
    else:
        assert torch.equal(d, s)


def test_probe_rejects():
    from paper_2012_06012_gb300 import mgt
    src = torch.zeros(4096 * 64, dtype=torch.uint8, device="cuda")
    dst = torch.zeros_like(src)
    perm = torch.arange(64, dtype=torch.int32, device="cuda")
    with pytest.raises(Exception):
        mgt.probe_runs(5, src, dst, perm, 64, 2048)  # four stages of 32 runs would not fit
    with pytest.raises(Exception):
        mgt.probe_runs(0, src, dst, perm, 64, 24)  # not a multiple of 16


def test_l2_fetch_granularity_round_trip():
    from paper_2012_06012_gb300 import mgt
    torch.cuda.init()
    before = mgt.l2_fetch_granularity()
    try:
        mgt.l2_fetch_granularity(32)
        assert mgt.l2_fetch_granularity() == 32
    finally:
        mgt.l2_fetch_granularity(before)
    assert mgt.l2_fetch_granularity() == before
    with pytest.raises(Exception):
        mgt.l2_fetch_granularity(256)
