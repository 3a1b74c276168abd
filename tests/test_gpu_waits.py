"""Bounded waits: every wait of the scan kernel for a staged text tile is
bounded (pm_config.wait_clocks SM clocks; default about 2 s). With a budget
far below a copy's latency the waits run out: the kernel records
PM_ERR_TIMEOUT in its device error word, waits (with the full budget) for
its copies in flight, and returns; nothing traps, the context stays usable,
and the next scan with the default budget is bit-exact. Before each
short-budget scan a write larger than L2 evicts the text, so that the
first copies come from HBM."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1702_03657_gb300 import pm
from paper_1702_03657_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_03657_gb300 import build as B
    B.build()
    pm.load()
    yield


@pytest.mark.parametrize("sched", [1, 2])
def test_wait_that_runs_out_reports_timeout(sched):
    """Both schedules; the dynamic one also waits (bounded by the same
    budget) for its CTA's next run of tiles to be published."""
    wl = W.paper_scale(6, text_bytes=16 * W.MiB + 3, n_patterns=3000)
    t = pm.pm_build(wl.patterns)
    cfg = pm.pm_get_config(t)
    tv = torch.from_numpy(wl.text).cuda()
    ids = torch.empty(len(wl.text), dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    assert pm.pm_device_error() == pm.PM_OK
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for budget in (1, 64):
        # the text out of L2 (a write larger than L2 in between), so that the
        # first tile's copy comes from HBM, far later than the budget allows
        flush.fill_(budget)
        pm.pm_scan_ex(t, tv, None, ids, cnt, cfg=dict(cfg, wait_clocks=budget, schedule=sched))
        torch.cuda.synchronize()                      # the launch returned
        assert pm.pm_device_error() == pm.PM_ERR_TIMEOUT
        assert pm.pm_device_error() == pm.PM_OK       # read and cleared
    # the context is usable and the default budget gives the oracle's bits
    pm.pm_scan_ex(t, tv, None, ids, cnt, cfg=dict(cfg, schedule=sched))
    torch.cuda.synchronize()
    assert pm.pm_device_error() == pm.PM_OK
    o_ids, o_cnt, _ = oracle.Trie(wl.patterns).scan(wl.text, threads=8)
    assert np.array_equal(ids.cpu().numpy(), o_ids) and int(cnt.item()) == o_cnt
