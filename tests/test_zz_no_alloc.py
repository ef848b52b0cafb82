"""cvd_copy_batch_noalloc against cvd_copy_batch.

The no-allocation entry point exists for callers that cannot allocate device
memory on their request path (cudaMalloc/cudaFree synchronise the whole
device, and a device whose memory another allocator already holds can make a
late cudaMalloc fail).  It must give exactly what the regular hazard-free
batch gives -- results, staging bytes and guest memory, bit for bit, the
same tolerance as every other parity test here -- on two calls in a row, the
second smaller than the first so that leftovers of the shared fixed scratch
cannot leak into it.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1304_3771_b300 import workload as W

pytestmark = pytest.mark.gpu


def _state(pool_np, stg_np):
    import torch
    return torch.from_numpy(pool_np.copy()).cuda(), torch.from_numpy(stg_np.copy()).cuda()


def test_noalloc_matches_copy_batch_on_two_calls():
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(256 << 20, 901, huge_frac=0.5, np_frac=0.02, ro_frac=0.02, nslots=3, slot_gap_pages=256)
    pool = W.materialize_pool(img)
    sizes = np.minimum(W.batching_sizes(901, 6000), 400_000)
    wl = W.batched_requests(img, 901, sizes, 32)
    stg = W.payload_bytes(902, wl.staging_bytes)
    pool_a, stg_a = _state(pool, stg)     # no-allocation entry point
    pool_b, stg_b = _state(pool, stg)     # regular entry point
    ga = cvd.Guest.from_image(img, pool_a)
    gb = cvd.Guest.from_image(img, pool_b)
    lo, hi = wl.batches[0]
    first = wl.reqs[lo:hi]
    second = wl.reqs[lo:lo + max(1, (hi - lo) // 3)].copy()
    second["dir"] ^= 1                    # different work on the second call
    seg_d = cvd.records_to_device(wl.segs)
    for reqs in (first, second):
        req_d = cvd.records_to_device(reqs)
        res_a = torch.full((len(reqs) * 24,), 0x5A, dtype=torch.uint8, device="cuda")
        res_b = torch.zeros(len(reqs) * 24, dtype=torch.uint8, device="cuda")
        cvd.copy_batch_noalloc(ga, req_d, len(reqs), seg_d, len(wl.segs), stg_a, res_a)
        cvd.copy_batch([gb], req_d, len(reqs), seg_d, len(wl.segs), stg_b, res_b, flags=cvd.BATCH_HAZARD_FREE)
        torch.cuda.synchronize()
        ra = cvd.records_from_device(res_a, W.RESULT_DTYPE, len(reqs))
        rb = cvd.records_from_device(res_b, W.RESULT_DTYPE, len(reqs))
        np.testing.assert_array_equal(ra, rb)
        assert torch.equal(stg_a, stg_b), "staging bytes differ"
        assert torch.equal(pool_a, pool_b), "guest memory differs"
        assert (ra["fault_code"] != 0).any() and (ra["fault_code"] == 0).any()
    ga.close()
    gb.close()


def test_noalloc_rejects_batches_beyond_its_scratch():
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(64 << 20, 903, np_frac=0, ro_frac=0)
    pool_d = torch.from_numpy(W.materialize_pool(img, fill=False)).cuda()
    g = cvd.Guest.from_image(img, pool_d)
    z = torch.zeros(64, dtype=torch.uint8, device="cuda")
    stg = torch.zeros(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(cvd.CvdError) as ei:
        cvd.copy_batch_noalloc(g, z, 65536 + 1, z, 1, stg, z)
    assert ei.value.status == cvd.E2BIG
    with pytest.raises(cvd.CvdError) as ei:
        cvd.copy_batch_noalloc(g, z, 1, z, 262144 + 1, stg, z)
    assert ei.value.status == cvd.E2BIG
    g.close()
