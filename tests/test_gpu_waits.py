"""Bounded waits: every wait of the scan kernel for a staged text tile is
bounded (pm_config.wait_clocks SM clocks; default about 2 s). With a budget
far below a copy's latency the waits run out: the kernel records
PM_ERR_TIMEOUT in its device error word, waits (with the full budget) for
its copies in flight, and returns; nothing traps, the context stays usable,
and the next scan with the default budget is bit-exact."""
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


def test_wait_that_runs_out_reports_timeout():
    wl = W.paper_scale(6, text_bytes=16 * W.MiB + 3, n_patterns=3000)
    t = pm.pm_build(wl.patterns)
    cfg = pm.pm_get_config(t)
    tv = torch.from_numpy(wl.text).cuda()
    ids = torch.empty(len(wl.text), dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    assert pm.pm_device_error() == pm.PM_OK
    for budget in (1, 64):
        pm.pm_scan_ex(t, tv, None, ids, cnt, cfg=dict(cfg, wait_clocks=budget))
        torch.cuda.synchronize()                      # the launch returned
        assert pm.pm_device_error() == pm.PM_ERR_TIMEOUT
        assert pm.pm_device_error() == pm.PM_OK       # read and cleared
    # the context is usable and the default budget gives the oracle's bits
    pm.pm_scan(t, tv, ids, cnt)
    torch.cuda.synchronize()
    assert pm.pm_device_error() == pm.PM_OK
    o_ids, o_cnt, _ = oracle.Trie(wl.patterns).scan(wl.text, threads=8)
    assert np.array_equal(ids.cpu().numpy(), o_ids) and int(cnt.item()) == o_cnt
