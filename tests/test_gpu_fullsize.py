"""Parity at the full workload sizes, in the launch configuration bench.py
times (library default copy parameters, hazard-free batches, one guest).

* Batching (16 GiB guest, 1,000,000 requests): the GPU runs the whole first
  batch; the oracle recomputes a sample of its requests one by one against a
  host shadow holding the page tables and the sampled requests' source bytes,
  read from the device before the GPU call (inputs only).  Hazard-free
  requests are independent, so each sampled result must match exactly.
* Frames (32 GiB guest, 4 KiB pages permuted, 4,096 page-aligned frames of
  8,294,400 or 33,177,600 B): the GPU runs the whole first batch (1,661
  frames, ~28 GB); sampled frames recomputed by the oracle the same way.
* Translation (8 GiB guest, 2^26 gVAs): every output compared.
* mmap install (8 GiB guest, 10,000 requests, 2.55 M pages): every page
  status, the whole p2m array and every page-table frame compared."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W

pytestmark = pytest.mark.gpu

SEED = W.DEFAULT_SEED


def _upload_guest(img, gen, fill=True):
    import torch
    from paper_1304_3771_b300 import cvd
    pool = torch.empty(img.pool_bytes, dtype=torch.uint8, device="cuda")
    if fill:
        n = pool.numel()
        for a in range(0, n, 1 << 30):
            b = min(n, a + (1 << 30))
            pool[a:b] = torch.randint(0, 256, (b - a,), dtype=torch.uint8, device="cuda", generator=gen)
    else:
        pool.zero_()
    offs, data = W.table_blob(img)
    idx = torch.from_numpy((offs[:, None] + np.arange(4096)[None, :]).reshape(-1)).cuda()
    pool[idx] = torch.from_numpy(data.reshape(-1)).cuda()
    p2m = torch.full((max(img.rsv_n, 1),), -1, dtype=torch.int64, device="cuda")
    return cvd.Guest.from_image(img, pool, p2m=p2m), pool


def _shadow(img):
    pool = np.zeros(img.pool_bytes, dtype=np.uint8)      # lazily backed: only touched pages cost memory
    W.write_tables(img, pool)
    return pool


def _host_runs(og, segs, write):
    """(host offset, length) of every page piece the segments touch (oracle walk)."""
    runs = []
    for s in segs:
        va, end = int(s["gva"]), int(s["gva"]) + int(s["len"])
        while va < end:
            code, gpa, hpa = og.walk(va, write)
            if code:
                break
            n = min(end, (va & ~4095) + 4096) - va
            runs.append((hpa, n))
            va += n
    return runs


def test_batching_full_size_sampled():
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(16 << 30, SEED, huge_frac=0.7, np_frac=0.0, ro_frac=0.0, nslots=4, slot_gap_pages=512)
    wl = W.batched_requests(img, SEED, W.batching_sizes(SEED, 1_000_000), 32)
    lo, hi = wl.batches[0]
    reqs = wl.reqs[lo:hi].copy()
    s0 = int(reqs["seg_begin"][0])
    s1 = int(reqs["seg_begin"][-1] + reqs["seg_count"][-1])
    reqs["seg_begin"] -= s0
    segs = wl.segs[s0:s1].copy()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1)
    g, pool_d = _upload_guest(img, gen)
    stg_d = torch.randint(0, 256, (wl.staging_bytes,), dtype=torch.uint8, device="cuda", generator=gen)

    rng = np.random.default_rng(2)
    L = np.add.reduceat(segs["len"].astype(np.int64), reqs["seg_begin"].astype(np.int64))
    big = np.nonzero(L > (1 << 20))[0]
    sample = np.unique(np.concatenate([rng.choice(len(reqs), 1500, replace=False), rng.choice(big, 40, replace=False)]))
    shadow = _shadow(img)
    og = O.Guest.from_image(img, shadow)
    stg_shadow = np.zeros(wl.staging_bytes, dtype=np.uint8)
    guest_pages = {}
    for i in sample:
        r = reqs[i]
        ss = segs[r["seg_begin"]:r["seg_begin"] + r["seg_count"]]
        runs = _host_runs(og, ss, r["dir"] == 1)
        guest_pages[i] = runs
        for p in sorted({h & ~4095 for h, _ in runs}):   # inputs: guest bytes of the touched pages
            shadow[p:p + 4096] = pool_d[p:p + 4096].cpu().numpy()
        h = int(r["host_off"])
        if r["dir"] == 1:                                 # inputs: staging source bytes
            stg_shadow[h:h + L[i]] = stg_d[h:h + L[i]].cpu().numpy()
    # the GPU runs the whole batch with the library defaults (bench's configuration)
    req_d, seg_d = cvd.records_to_device(reqs), cvd.records_to_device(segs)
    res_d = torch.zeros(len(reqs) * 24, dtype=torch.uint8, device="cuda")
    cvd.copy_batch([g], req_d, len(reqs), seg_d, len(segs), stg_d, res_d, flags=cvd.BATCH_HAZARD_FREE)
    torch.cuda.synchronize()
    assert cvd.stream_check() == 0
    g_res = cvd.records_from_device(res_d, W.RESULT_DTYPE, len(reqs))
    # the oracle computes the sampled requests one by one
    for i in sample:
        r = reqs[i:i + 1].copy()
        ss = segs[r["seg_begin"][0]:r["seg_begin"][0] + r["seg_count"][0]].copy()
        r["seg_begin"] = 0
        o_res = O.copy_batch([og], r, ss, stg_shadow)
        np.testing.assert_array_equal(g_res[i:i + 1], o_res)
        h = int(r["host_off"][0])
        if r["dir"][0] == 0:
            assert np.array_equal(stg_d[h:h + L[i]].cpu().numpy(), stg_shadow[h:h + L[i]]), i
        else:
            for hp, n in guest_pages[i]:                  # only the bytes this request writes
                assert np.array_equal(pool_d[hp:hp + n].cpu().numpy(), shadow[hp:hp + n]), (i, hp)
    assert (g_res["fault_code"] == 0).all() and (g_res["done"] == L.astype(np.uint64)).all()
    g.close()


def _pages_to_host(pool_d, pages):
    """Bytes of the given 4 KiB pages of a device pool, in one gather."""
    import torch
    idx = torch.from_numpy(np.asarray(pages, dtype=np.int64)).cuda()
    return torch.index_select(pool_d.view(-1, 4096), 0, idx).cpu().numpy()


def test_frames_full_size_sampled():
    import torch
    from paper_1304_3771_b300 import cvd
    seed = SEED + 4
    img = W.make_guest(32 << 30, seed, np_frac=0.0, ro_frac=0.0)
    wl = W.batched_requests(img, seed, W.frame_sizes(seed, 4096), 1, page_aligned=True)
    lo, hi = wl.batches[0]
    reqs = wl.reqs[lo:hi].copy()
    s0 = int(reqs["seg_begin"][0])
    reqs["seg_begin"] -= s0
    segs = wl.segs[s0:s0 + len(reqs)].copy()
    assert (reqs["seg_count"] == 1).all() and img.pool_bytes % 4096 == 0
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    g, pool_d = _upload_guest(img, gen)
    stg_d = torch.empty(wl.staging_bytes, dtype=torch.uint8, device="cuda")
    for a0 in range(0, stg_d.numel(), 1 << 30):
        b0 = min(stg_d.numel(), a0 + (1 << 30))
        stg_d[a0:b0] = torch.randint(0, 256, (b0 - a0,), dtype=torch.uint8, device="cuda", generator=gen)

    rng = np.random.default_rng(4)
    L = segs["len"].astype(np.int64)
    sample = np.unique(np.concatenate([rng.choice(np.nonzero(reqs["dir"] == d)[0], 8, replace=False) for d in (0, 1)]))
    shadow = _shadow(img)
    og = O.Guest.from_image(img, shadow)
    stg_shadow = np.zeros(wl.staging_bytes, dtype=np.uint8)   # lazily backed
    runs = {i: _host_runs(og, segs[i:i + 1], reqs["dir"][i] == 1) for i in sample}
    pages = sorted({h >> 12 for i in sample for h, _ in runs[i]})
    shadow.reshape(-1, 4096)[pages] = _pages_to_host(pool_d, pages)   # inputs: the touched guest pages
    for i in sample:
        h = int(reqs["host_off"][i])
        if reqs["dir"][i] == 1:                                          # inputs: staging sources
            stg_shadow[h:h + L[i]] = stg_d[h:h + L[i]].cpu().numpy()
    req_d, seg_d = cvd.records_to_device(reqs), cvd.records_to_device(segs)
    res_d = torch.zeros(len(reqs) * 24, dtype=torch.uint8, device="cuda")
    cvd.copy_batch([g], req_d, len(reqs), seg_d, len(segs), stg_d, res_d, flags=cvd.BATCH_HAZARD_FREE)
    torch.cuda.synchronize()
    assert cvd.stream_check() == 0
    g_res = cvd.records_from_device(res_d, W.RESULT_DTYPE, len(reqs))
    assert (g_res["fault_code"] == 0).all() and (g_res["done"] == L.astype(np.uint64)).all()
    for i in sample:
        r = reqs[i:i + 1].copy()
        r["seg_begin"] = 0
        o_res = O.copy_batch([og], r, segs[i:i + 1].copy(), stg_shadow)
        np.testing.assert_array_equal(g_res[i:i + 1], o_res)
        h = int(r["host_off"][0])
        if r["dir"][0] == 0:
            assert np.array_equal(stg_d[h:h + L[i]].cpu().numpy(), stg_shadow[h:h + L[i]]), i
        else:                                                            # the frame's guest pages
            fp = sorted({hp >> 12 for hp, _ in runs[i]})
            assert np.array_equal(_pages_to_host(pool_d, fp), shadow.reshape(-1, 4096)[fp]), i
    g.close()
    del pool_d, stg_d
    torch.cuda.empty_cache()


def test_translate_full_size_all_outputs():
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(8 << 30, SEED + 3, np_frac=0.05, ro_frac=0.05)
    gen = torch.Generator(device="cuda")
    g, pool_d = _upload_guest(img, gen, fill=False)
    gva = W.translate_gvas(img, SEED + 3, 1 << 26)
    out = g.translate(cvd.u64_to_device(gva))
    torch.cuda.synchronize()
    og = O.Guest.from_image(img, _shadow(img))
    for write in (False,):
        exp = og.translate(gva, write)
        np.testing.assert_array_equal(cvd.u64_from_device(out[0]), exp[0])
        np.testing.assert_array_equal(cvd.u64_from_device(out[1]), exp[1])
        np.testing.assert_array_equal(out[2].cpu().numpy().view(np.uint32), exp[2])
    g.close()


def test_mmap_full_size_all_outputs():
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(8 << 30, SEED + 3, np_frac=0.05, ro_frac=0.05, pt_pool_n=40000, rsv_n=3 << 20)
    reqs, hf, _ = W.mmap_requests(img, SEED + 3, 10000)
    npg = int(reqs["npages"].astype(np.int64).sum())
    gen = torch.Generator(device="cuda")
    g, pool_d = _upload_guest(img, gen, fill=False)
    st = torch.zeros(npg, dtype=torch.int32, device="cuda")
    g.mmap_install(cvd.records_to_device(reqs), len(reqs), cvd.u64_to_device(hf), len(hf), st)
    shadow = _shadow(img)
    og = O.Guest.from_image(img, shadow)
    o_st = og.mmap_install(reqs, hf)
    np.testing.assert_array_equal(st.cpu().numpy(), o_st)
    np.testing.assert_array_equal(cvd.u64_from_device(g.p2m), og.p2m)
    assert g.alloc_state() == (og.pt_used, og.rsv_used)
    # every table frame: the generator's tables and the PT pool
    frames = sorted(set(img.tables) | set(range(img.pt_pool_gfn, img.pt_pool_gfn + img.pt_pool_n)))
    host = np.array([img.gpa_to_host(f << 12) for f in frames], dtype=np.int64)
    runs = np.split(host, np.nonzero(np.diff(host) != 4096)[0] + 1)
    for run in runs:
        a, b = int(run[0]), int(run[-1]) + 4096
        assert np.array_equal(pool_d[a:b].cpu().numpy(), shadow[a:b]), hex(a)
    assert (o_st == 0).sum() > 1_000_000
    g.close()
