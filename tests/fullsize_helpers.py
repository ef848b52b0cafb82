"""Exhaustive parity at full workload sizes (shared by the full-size GPU
tests): the oracle's host state is a pinned copy of the device's initial
state; comparisons stream it back to the device in 1 GiB chunks."""
import numpy as np

import oracle as O
from paper_1304_3771_b300 import workload as W

CHUNK = 1 << 30


def upload_guest(img, gen, fill=True):
    import torch
    from paper_1304_3771_b300 import cvd
    pool = torch.empty(img.pool_bytes, dtype=torch.uint8, device="cuda")
    if fill:
        fill_random(pool, gen)
    else:
        pool.zero_()
    offs, data = W.table_blob(img)
    idx = torch.from_numpy((offs[:, None] + np.arange(4096)[None, :]).reshape(-1)).cuda()
    pool[idx] = torch.from_numpy(data.reshape(-1)).cuda()
    p2m = torch.full((max(img.rsv_n, 1),), -1, dtype=torch.int64, device="cuda")
    return cvd.Guest.from_image(img, pool, p2m=p2m), pool


def fill_random(t, gen):
    import torch
    n = t.numel()
    for a in range(0, n, CHUNK):
        b = min(n, a + CHUNK)
        t[a:b] = torch.randint(0, 256, (b - a,), dtype=torch.uint8, device="cuda", generator=gen)


def table_shadow(img):
    pool = np.zeros(img.pool_bytes, dtype=np.uint8)      # lazily backed: only touched pages cost memory
    W.write_tables(img, pool)
    return pool


def to_host_pinned(t):
    """A pinned host copy of a device tensor (numpy view and the tensor)."""
    import torch
    h = torch.empty(t.numel(), dtype=torch.uint8, pin_memory=True)
    for a in range(0, t.numel(), CHUNK):
        b = min(t.numel(), a + CHUNK)
        h[a:b].copy_(t[a:b])
    torch.cuda.synchronize()
    return h, h.numpy()


def assert_equal_streamed(dev, host_t, what):
    """dev (device) == host_t (pinned host), compared on the device chunk by chunk."""
    import torch
    tmp = torch.empty(min(CHUNK, dev.numel()), dtype=torch.uint8, device="cuda")
    for a in range(0, dev.numel(), CHUNK):
        b = min(dev.numel(), a + CHUNK)
        tmp[:b - a].copy_(host_t[a:b], non_blocking=True)
        ne = torch.ne(dev[a:b], tmp[:b - a])
        if bool(ne.any()):
            first = a + int(torch.nonzero(ne)[0])
            raise AssertionError(f"{what} differs from the oracle at byte {first} (of {dev.numel()})")


def batch_records(wl):
    out = []
    for lo, hi in wl.batches:
        r = wl.reqs[lo:hi].copy()
        s0 = int(r["seg_begin"][0])
        s1 = int(r["seg_begin"][-1] + r["seg_count"][-1])
        r["seg_begin"] -= s0
        out.append((r, wl.segs[s0:s1].copy()))
    return out


def exhaustive_batches(img, wl, gen):
    """Every hazard-free batch of `wl` on the oracle, in order, beside the GPU
    twice from the same initial state (random pool and staging bytes from
    `gen`): once as one planned-ahead cvd_copy_batches call over all batches,
    once as one cvd_copy_batch call per batch in lockstep with the oracle.
    Every result is compared; the whole staging buffer and guest pool after
    every lockstep batch and after the planned-ahead call.  Returns the
    number of requests compared."""
    import torch
    from paper_1304_3771_b300 import cvd
    batches = batch_records(wl)
    g0, pool0 = upload_guest(img, gen)
    stg0 = torch.empty(wl.staging_bytes, dtype=torch.uint8, device="cuda")
    fill_random(stg0, gen)
    pool_ht, pool_h = to_host_pinned(pool0)        # the oracle's copy of the initial state
    stg_ht, stg_h = to_host_pinned(stg0)
    dev = [(cvd.records_to_device(r), len(r), cvd.records_to_device(s), len(s)) for r, s in batches]
    # (1) the planned-ahead step over all batches, on a clone of the initial state
    pool_a, stg_a = pool0.clone(), stg0.clone()
    ga = cvd.Guest.from_image(img, pool_a, p2m=torch.full((max(img.rsv_n, 1),), -1, dtype=torch.int64, device="cuda"))
    res_a = [torch.zeros(n * 24, dtype=torch.uint8, device="cuda") for _, n, _, _ in dev]
    cvd.copy_batches([ga], [(rq, nr, sg, ns, ra) for (rq, nr, sg, ns), ra in zip(dev, res_a)], stg_a)
    torch.cuda.synchronize()
    assert cvd.stream_check() == 0
    # (2) lockstep: one GPU call per batch on the initial state itself, oracle beside it
    og = O.Guest.from_image(img, pool_h)
    res_b = torch.zeros(max(n for _, n, _, _ in dev) * 24, dtype=torch.uint8, device="cuda")
    nreq = 0
    for k, ((r, s), (rq, nr, sg, ns)) in enumerate(zip(batches, dev)):
        o_res = O.copy_batch([og], r, s, stg_h)
        cvd.copy_batch([g0], rq, nr, sg, ns, stg0, res_b, flags=cvd.BATCH_HAZARD_FREE)
        torch.cuda.synchronize()
        assert cvd.stream_check() == 0
        np.testing.assert_array_equal(cvd.records_from_device(res_b, W.RESULT_DTYPE, nr), o_res, err_msg=f"batch {k}")
        np.testing.assert_array_equal(cvd.records_from_device(res_a[k], W.RESULT_DTYPE, nr), o_res,
                                      err_msg=f"planned-ahead batch {k}")
        assert_equal_streamed(stg0, stg_ht, f"staging after batch {k}")
        assert_equal_streamed(pool0, pool_ht, f"guest pool after batch {k}")
        nreq += nr
    assert_equal_streamed(stg_a, stg_ht, "staging after the planned-ahead step")
    assert_equal_streamed(pool_a, pool_ht, "guest pool after the planned-ahead step")
    ga.close()
    g0.close()
    del pool0, stg0, pool_a, stg_a, res_a, pool_ht, stg_ht
    torch.cuda.empty_cache()
    return nreq
