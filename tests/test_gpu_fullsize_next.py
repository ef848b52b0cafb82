"""Parity at the measured sizes of the rows beyond the base path, in the
launch configuration bench.py times.

* Software EPT and PAE guests (2 GiB guests of the ept / pae arms, 2^26
  gVAs): every translation output compared with the oracle.
* The batching mix on the same EPT and PAE guests (200,000 requests in
  hazard-free batches): the GPU runs the whole first batch; sampled requests
  are recomputed by the oracle one by one from a host shadow holding the
  tables and the pages and staging bytes those requests read (inputs only).
* Chained gathers (8 GiB guest, 50,000 descriptor tables, 7.75 GB payload):
  the GPU runs the whole call; a sample of requests is recomputed by the
  oracle one by one from a host shadow holding the guest's tables and the
  pages those requests read (inputs only); payload places are the prefix
  sums of the lengths.
* Driver-initiated maps (the place arm: 64 GiB window fragmented by 2,000
  installs, 10,000 requests): the GPU result is checked against properties
  that hold at any size -- every range inside the window, ranges pairwise
  disjoint and clear of the fragmenting installs, every page installed and
  translating to its host frame (sampled), and first fit for a sample of
  requests against the exact free map below their range.  The oracle itself
  runs the same call on smaller windows in test_gpu_place.py."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W

pytestmark = pytest.mark.gpu

SEED = W.DEFAULT_SEED


def _upload(img, fill_seed=None):
    import torch
    from paper_1304_3771_b300 import cvd
    pool = torch.zeros(img.pool_bytes, dtype=torch.uint8, device="cuda")
    if fill_seed is not None:
        gen = torch.Generator(device="cuda")
        gen.manual_seed(fill_seed)
        n = pool.numel()
        for a in range(0, n, 1 << 30):
            b = min(n, a + (1 << 30))
            pool[a:b] = torch.randint(0, 256, (b - a,), dtype=torch.uint8, device="cuda", generator=gen)
    offs, data = W.table_blob(img)
    idx = torch.from_numpy((offs[:, None] + np.arange(4096)[None, :]).reshape(-1)).cuda()
    pool[idx] = torch.from_numpy(data.reshape(-1)).cuda()
    p2m = torch.full((max(img.rsv_n, 1),), -1, dtype=torch.int64, device="cuda")
    return cvd.Guest.from_image(img, pool, p2m=p2m), pool, p2m


def _shadow(img):
    pool = np.zeros(img.pool_bytes, dtype=np.uint8)
    W.write_tables(img, pool)
    return pool


def _arm_image(kind):
    """The 2 GiB guest of the ept or pae arm, and its seed."""
    if kind == "ept":
        img0 = W.make_guest(2 << 30, SEED + 12, huge_frac=0.3, np_frac=0.0, ro_frac=0.0, nslots=4,
                            slot_gap_pages=512, host_base=2 << 20)
        return W.add_ept(img0, SEED + 12, huge_frac=0.5), SEED + 12
    return W.make_guest(2 << 30, SEED + 8, paging="pae", huge_frac=0.3, np_frac=0.0, ro_frac=0.0, nslots=4,
                        slot_gap_pages=512), SEED + 8


@pytest.mark.parametrize("kind", ["ept", "pae"])
def test_translate_bench_size_ept_and_pae(kind):
    import torch
    from paper_1304_3771_b300 import cvd
    img, _ = _arm_image(kind)
    g, pool, _ = _upload(img)
    gva = W.translate_gvas(img, SEED + 12, 1 << 26)
    out = g.translate(cvd.u64_to_device(gva), write=True)
    torch.cuda.synchronize()
    exp = O.Guest.from_image(img, _shadow(img)).translate(gva, True)
    np.testing.assert_array_equal(out[2].cpu().numpy().view(np.uint32), exp[2])
    np.testing.assert_array_equal(cvd.u64_from_device(out[0]), exp[0])
    np.testing.assert_array_equal(cvd.u64_from_device(out[1]), exp[1])
    assert (exp[2] == 0).sum() > (1 << 24)
    g.close()


@pytest.mark.parametrize("kind", ["ept", "pae"])
def test_batching_bench_size_ept_and_pae_sampled(kind):
    import torch
    from paper_1304_3771_b300 import cvd
    img, seed = _arm_image(kind)
    g, pool, _ = _upload(img, fill_seed=seed + 1)
    wl = W.batched_requests(img, seed, W.batching_sizes(seed, 200_000), 32)
    lo, hi = wl.batches[0]
    reqs = wl.reqs[lo:hi].copy()
    s0 = int(reqs["seg_begin"][0])
    s1 = int(reqs["seg_begin"][-1] + reqs["seg_count"][-1])
    reqs["seg_begin"] -= s0
    segs = wl.segs[s0:s1].copy()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed + 2)
    stg_d = torch.randint(0, 256, (wl.staging_bytes,), dtype=torch.uint8, device="cuda", generator=gen)
    rng = np.random.default_rng(seed)
    L = np.add.reduceat(segs["len"].astype(np.int64), reqs["seg_begin"].astype(np.int64))
    big = np.nonzero(L > (1 << 20))[0]
    sample = np.unique(np.concatenate([rng.choice(len(reqs), 600, replace=False),
                                       rng.choice(big, min(20, len(big)), replace=False)]))
    shadow = _shadow(img)
    og = O.Guest.from_image(img, shadow)
    stg_shadow = np.zeros(wl.staging_bytes, dtype=np.uint8)
    runs = {}
    for i in sample:
        r = reqs[i]
        rr = []
        for sg in segs[r["seg_begin"]:r["seg_begin"] + r["seg_count"]]:
            va, end = int(sg["gva"]), int(sg["gva"]) + int(sg["len"])
            while va < end:
                code, gpa, hpa = og.walk(va, r["dir"] == 1)
                if code:
                    break
                n = min(end, (va & ~4095) + 4096) - va
                rr.append((hpa, n))
                va += n
        runs[i] = rr
    pages = np.array(sorted({h >> 12 for i in sample for h, _ in runs[i]}), dtype=np.int64)
    pidx = torch.from_numpy(pages).cuda()
    shadow.reshape(-1, 4096)[pages] = torch.index_select(pool.view(-1, 4096), 0, pidx).cpu().numpy()
    for i in sample:
        h = int(reqs["host_off"][i])
        if reqs["dir"][i] == 1:
            stg_shadow[h:h + L[i]] = stg_d[h:h + L[i]].cpu().numpy()
    req_d, seg_d = cvd.records_to_device(reqs), cvd.records_to_device(segs)
    res_d = torch.zeros(len(reqs) * 24, dtype=torch.uint8, device="cuda")
    cvd.copy_batch([g], req_d, len(reqs), seg_d, len(segs), stg_d, res_d, flags=cvd.BATCH_HAZARD_FREE)
    torch.cuda.synchronize()
    assert cvd.stream_check() == 0
    g_res = cvd.records_from_device(res_d, W.RESULT_DTYPE, len(reqs))
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
            for hp, n in runs[i]:                        # only the bytes this request writes
                assert np.array_equal(pool[hp:hp + n].cpu().numpy(), shadow[hp:hp + n]), (i, hp)
    assert (g_res["fault_code"] == 0).all() and (g_res["done"] == L.astype(np.uint64)).all()
    g.close()


def test_chain_bench_size_sampled():
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(8 << 30, SEED + 15, huge_frac=0.7, np_frac=0.0, ro_frac=0.0, nslots=4, slot_gap_pages=512)
    wl = W.chained_requests(img, SEED + 15, 50_000)
    g, pool, _ = _upload(img, fill_seed=5)
    offs = W.host_of_gva_array(img, wl.entry_gvas())
    idx = torch.from_numpy((offs[:, None] + np.arange(16)[None, :]).reshape(-1)).cuda()
    pool[idx] = torch.from_numpy(wl.entries.reshape(-1).view(np.uint8)).cuda()
    desc = torch.zeros(wl.desc_bytes, dtype=torch.uint8, device="cuda")
    pay = torch.zeros(wl.payload_bytes, dtype=torch.uint8, device="cuda")
    res = torch.zeros(len(wl.reqs) * W.CHAIN_RES_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cvd.gather_chained([g], cvd.records_to_device(wl.reqs), len(wl.reqs), desc, pay, res,
                       flags=cvd.BATCH_HAZARD_FREE)
    torch.cuda.synchronize()
    g_res = cvd.records_from_device(res, W.CHAIN_RES_DTYPE, len(wl.reqs))
    L = np.add.reduceat(wl.entries[:, 1].astype(np.int64), wl.first[:-1])
    assert (g_res["level"] == 0).all() and (g_res["payload_len"] == L.astype(np.uint64)).all()
    assert (g_res["payload_off"] == np.concatenate([[0], np.cumsum(L)[:-1]]).astype(np.uint64)).all()
    assert np.array_equal(desc.cpu().numpy(), wl.entries.reshape(-1).view(np.uint8))
    # the oracle recomputes a sample, one request at a time, from a shadow of its input pages
    shadow = _shadow(img)
    og = O.Guest.from_image(img, shadow)
    rng = np.random.default_rng(3)
    for r in rng.choice(len(wl.reqs), 300, replace=False):
        q = wl.reqs[r:r + 1].copy()
        q["desc_off"] = 0
        ent = wl.entries[wl.first[r]:wl.first[r + 1]]
        pages = set()
        for gv, n in ent:
            gv, n = int(gv), int(n)
            for p in range(gv & ~4095, gv + n, 4096):
                pages.add(W.host_of_gva(img, p))
        g0 = int(q["table_gva"][0])
        for p in range(g0 & ~4095, g0 + 16 * len(ent), 4096):
            pages.add(W.host_of_gva(img, p))
        for h in pages:
            shadow[h:h + 4096] = pool[h:h + 4096].cpu().numpy()
        o_desc = np.zeros(16 * len(ent), np.uint8)
        o_pay = np.zeros(int(L[r]), np.uint8)
        o_res = O.gather_chained([og], q, o_desc, o_pay)
        assert o_res["done"][0] == L[r] and o_res["level"][0] == 0
        a = int(g_res["payload_off"][r])
        assert np.array_equal(pay[a:a + int(L[r])].cpu().numpy(), o_pay), r
    g.close()


def test_place_bench_size_properties():
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(8 << 30, SEED + 3, np_frac=0.05, ro_frac=0.05, pt_pool_n=60000, rsv_n=3 << 20)
    frag, fhf, win = W.mmap_requests(img, SEED + 13, 2000, max_pages=64, window_bytes=16 << 30, busy_frac=0.0)
    reqs, hf = W.place_requests(img, SEED + 14, 10000)
    g, pool, p2m = _upload(img)
    fst = torch.zeros(int(frag["npages"].astype(np.int64).sum()), dtype=torch.int32, device="cuda")
    g.mmap_install(cvd.records_to_device(frag), len(frag), cvd.u64_to_device(fhf), len(fhf), fst)
    # the free map of the window's first 16 GiB before the call: the fragmenting installs take their pages
    npg_w = (16 << 30) // 4096
    taken = np.zeros(npg_w, dtype=bool)
    ok = fst.cpu().numpy() == 0
    off = 0
    for q in frag:
        k = int(q["npages"])
        p0 = (int(q["gva"]) - win) // 4096
        taken[p0:p0 + k] |= ok[off:off + k]
        off += k
    npg = int(reqs["npages"].astype(np.int64).sum())
    st = torch.zeros(npg, dtype=torch.int32, device="cuda")
    gva = torch.zeros(len(reqs), dtype=torch.int64, device="cuda")
    g.mmap_place(win, win + (64 << 30), cvd.records_to_device(reqs), len(reqs), cvd.u64_to_device(hf), len(hf),
                 gva, st)
    torch.cuda.synchronize()
    gv = cvd.u64_from_device(gva)
    assert (st.cpu().numpy() == 0).all() and (gv != O.NO_FRAME).all()
    start = (gv.astype(np.int64) - win) // 4096
    n = reqs["npages"].astype(np.int64)
    assert (gv % 4096 == 0).all() and (start >= 0).all() and (start + n <= (64 << 30) // 4096).all()
    order = np.argsort(start)
    assert (start[order][1:] >= (start + n)[order][:-1]).all(), "ranges overlap"
    # clear of the fragmenting installs; first fit for a sample against the exact free map
    used = taken.copy()
    for r in range(len(reqs)):
        a, k = int(start[r]), int(n[r])
        if a < npg_w:
            assert not used[a:min(a + k, npg_w)].any(), r
        if r % 97 == 0:   # no lower start fits: every earlier run of free pages is shorter than k
            free = ~used[:min(a, npg_w)]
            if len(free):
                edges = np.flatnonzero(np.diff(np.concatenate([[0], free.astype(np.int8), [0]])))
                assert ((edges[1::2] - edges[0::2]) < k).all(), r
        used[a:min(a + k, npg_w)] = True
    # translation after the install: a sample of pages reaches its host frame
    og_pool = np.zeros(img.pool_bytes, dtype=np.uint8)
    frames = sorted(set(img.tables) | set(range(img.pt_pool_gfn, img.pt_pool_gfn + img.pt_pool_n)))
    host = np.array([img.gpa_to_host(f << 12) for f in frames], dtype=np.int64)
    for run in np.split(host, np.nonzero(np.diff(host) != 4096)[0] + 1):   # every table frame, as the GPU left it
        a, b = int(run[0]), int(run[-1]) + 4096
        og_pool[a:b] = pool[a:b].cpu().numpy()
    og = O.Guest.from_image(img, og_pool, p2m=cvd.u64_from_device(p2m).copy())
    hf_off = reqs["hf_begin"].astype(np.int64)
    rng = np.random.default_rng(4)
    for r in rng.choice(len(reqs), 200, replace=False):
        k = int(rng.integers(0, n[r]))
        code, _, hpa = og.walk(int(gv[r]) + 4096 * k + 7)
        assert code == 0 and hpa == int(hf[hf_off[r] + k]) * 4096 + 7, r
    g.close()
