"""Failure detection on the GPU without a fault: a kernel whose bounded
mbarrier wait cannot complete gives up, reports through the stream's device
error word (the path the copy engine uses), and leaves the context usable."""
import pytest

from paper_1304_3771_b300 import workload as W
from tests.gpu_helpers import assert_same, run_both

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_reports():
    import torch
    from paper_1304_3771_b300 import cvd
    assert cvd.stream_check() == 0
    assert cvd.selftest_wait_timeout(tries=1 << 10) == 1
    assert cvd.stream_check() == 0                    # the report was cleared
    s = torch.cuda.Stream()
    assert cvd.selftest_wait_timeout(tries=1 << 12, stream=s) == 1
    assert cvd.stream_check(s) == 0
    # the context still runs work, bit-exact against the oracle
    img = W.make_guest(64 << 20, 260)
    pool = W.materialize_pool(img)
    wl = W.tiny_requests(img, 260, nreq=200)
    stg = W.payload_bytes(261, wl.staging_bytes)
    assert_same(run_both(img, pool, wl.reqs, wl.segs, stg))
    assert cvd.stream_check() == 0
