"""cvd_copy_batch_noalloc against the oracle.

The no-allocation entry point exists for callers that cannot allocate device
memory on their request path (cudaMalloc/cudaFree synchronise the whole
device, and a device whose memory another allocator already holds can make a
late cudaMalloc fail).  Its results, staging bytes and guest memory must be
the oracle's, bit for bit -- the tolerance of every other parity test here --
on two calls in a row, the second smaller than the first and in the other
direction, so that leftovers of the shared fixed scratch cannot leak into it.
The call must also leave the device's free memory unchanged on a stream it
has never seen, launch exactly its own kernels, and report through
cvd_stream_check.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W

pytestmark = pytest.mark.gpu

def noalloc_kernels(nreq):
    """k_store_ptr, k_req_sizes, the scan (one kernel up to 2,048 requests,
    else three), k_plan, k_long_scan, the copy engine."""
    return 5 + (1 if nreq <= 2048 else 3)


def _workload(seed):
    img = W.make_guest(256 << 20, seed, huge_frac=0.5, np_frac=0.02, ro_frac=0.02, nslots=3, slot_gap_pages=256)
    pool = W.materialize_pool(img)
    sizes = np.minimum(W.batching_sizes(seed, 6000), 400_000)
    wl = W.batched_requests(img, seed, sizes, 32)
    stg = W.payload_bytes(seed + 1, wl.staging_bytes)
    return img, pool, wl, stg


def test_noalloc_matches_oracle_on_two_calls():
    import torch
    from paper_1304_3771_b300 import cvd
    img, pool, wl, stg = _workload(901)
    o_pool, o_stg = pool.copy(), stg.copy()
    og = O.Guest.from_image(img, o_pool)
    pool_d = torch.from_numpy(pool.copy()).cuda()
    stg_d = torch.from_numpy(stg.copy()).cuda()
    g = cvd.Guest.from_image(img, pool_d)
    lo, hi = wl.batches[0]
    first = wl.reqs[lo:hi]
    second = wl.reqs[lo:lo + max(1, (hi - lo) // 3)].copy()
    second["dir"] ^= 1                    # other work on the second call (still hazard-free)
    seg_d = cvd.records_to_device(wl.segs)
    assert cvd.stream_check() == 0
    for reqs in (first, second):
        o_res = O.copy_batch([og], reqs, wl.segs, o_stg)
        req_d = cvd.records_to_device(reqs)
        res_d = torch.full((len(reqs) * 24,), 0x5A, dtype=torch.uint8, device="cuda")
        cvd.copy_batch_noalloc(g, req_d, len(reqs), seg_d, len(wl.segs), stg_d, res_d)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(cvd.records_from_device(res_d, W.RESULT_DTYPE, len(reqs)), o_res)
        assert np.array_equal(stg_d.cpu().numpy(), o_stg), "staging bytes differ from the oracle"
        assert np.array_equal(pool_d.cpu().numpy(), o_pool), "guest memory differs from the oracle"
        assert (o_res["fault_code"] != 0).any() and (o_res["fault_code"] == 0).any()
    assert cvd.stream_check() == 0        # no bounded wait gave up
    g.close()


def test_noalloc_allocates_nothing_on_a_fresh_stream():
    import torch
    from paper_1304_3771_b300 import cvd
    img, pool, wl, stg = _workload(905)
    pool_d = torch.from_numpy(pool).cuda()
    stg_d = torch.from_numpy(stg).cuda()
    g = cvd.Guest.from_image(img, pool_d)
    lo, hi = wl.batches[0]
    reqs = wl.reqs[lo:hi]
    req_d, seg_d = cvd.records_to_device(reqs), cvd.records_to_device(wl.segs)
    res_d = torch.zeros(len(reqs) * 24, dtype=torch.uint8, device="cuda")
    cvd.copy_batch_noalloc(g, req_d, len(reqs), seg_d, len(wl.segs), stg_d, res_d)   # warm-up: module and scratch
    fresh, other = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    n0 = cvd.launch_count()
    cvd.copy_batch_noalloc(g, req_d, len(reqs), seg_d, len(wl.segs), stg_d, res_d, stream=fresh)
    fresh.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert cvd.launch_count() - n0 == noalloc_kernels(len(reqs))
    assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
    # the regular call on a stream it has not seen grows that stream's scratch
    cvd.copy_batch([g], req_d, len(reqs), seg_d, len(wl.segs), stg_d, res_d, flags=cvd.BATCH_HAZARD_FREE,
                   stream=other)
    other.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 < free1
    assert cvd.stream_check(fresh) == 0
    g.close()


def test_noalloc_rejects_batches_beyond_its_scratch_and_overflowing_streams():
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
    # 65,536 requests over a staging buffer just under 2^52 bytes: the stream
    # positions could pass 2^62, so the call is refused like cvd_copy_batch
    # (the staging pointer lies past the pool and is never dereferenced)
    far = C.c_void_p(pool_d.data_ptr() + pool_d.numel() + (1 << 20))
    for fn in ("cvd_copy_batch_noalloc",):
        rc = getattr(cvd.lib(), fn)(g.handle, C.c_void_p(z.data_ptr()), 65536, C.c_void_p(z.data_ptr()), 1, far,
                                    (1 << 52) - 1, C.c_void_p(z.data_ptr()), None)
        assert rc == cvd.EINVAL
    arr = (C.c_void_p * 1)(g.handle.value)
    assert cvd.lib().cvd_copy_batch(C.cast(arr, C.c_void_p), 1, C.c_void_p(z.data_ptr()), 65536,
                                    C.c_void_p(z.data_ptr()), 1, far, (1 << 52) - 1, C.c_void_p(z.data_ptr()),
                                    cvd.BATCH_HAZARD_FREE, None) == cvd.EINVAL
    g.close()
