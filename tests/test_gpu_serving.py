"""Serving loop (cvd_server_*): continuous batching of forwarded copies from
several guests.  Each guest's requests must take effect in arrival order
(the oracle run on that guest's requests in arrival order gives every result,
every copied-out byte and the final guest memory), and a guest's results must
be the same when it is served alone and when it is served in a mix."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W

pytestmark = pytest.mark.gpu


def _guests(n, seed=700, **kw):
    imgs, pools = [], []
    for k in range(n):
        img = W.make_guest(64 << 20, seed + k, **kw)
        imgs.append(img)
        pools.append(W.materialize_pool(img))
    return imgs, pools


def _requests(img, seed, nreq):
    wl = W.tiny_requests(img, seed, nreq=nreq, hi=40000, frame_frac=0.05)
    items = []
    for i, r in enumerate(wl.reqs):
        segs = wl.segs[r["seg_begin"]:r["seg_begin"] + r["seg_count"]]
        items.append((int(r["dir"]), segs, int(r["host_off"])))
    return wl, items


def _serve(guest_list, pools_np, streams_of_items, src_all, arrivals, max_batch=32, two_streams=False, carve=False):
    """streams_of_items: per guest index, list of (dir, segs, src_off).  Returns
    per guest: list of (result, out_bytes or None) in submission order, and the
    final pools.  carve: the pools are views 512 bytes past a 4 KiB boundary
    inside one allocation (as a caching allocator hands them out), so guest
    pages straddle device frames."""
    import torch
    from paper_1304_3771_b300 import cvd
    if carve:
        sizes = [((len(p) + 4095) // 4096 + 1) * 4096 for p in pools_np]
        whole = torch.empty(sum(sizes), dtype=torch.uint8, device="cuda")
        pools_d, at = [], 0
        for p, n in zip(pools_np, sizes):
            v = whole[at + 512:at + 512 + len(p)]
            v.copy_(torch.from_numpy(p))
            pools_d.append(v)
            at += n
    else:
        pools_d = [torch.from_numpy(p.copy()).cuda() for p in pools_np]
    gs = [cvd.Guest.from_image(img, pd) for img, pd in zip(guest_list, pools_d)]
    staging = torch.zeros(64 << 20, dtype=torch.uint8, device="cuda")
    srv = cvd.Server(gs, staging, max_batch=max_batch, max_inflight=256, two_streams=two_streams)
    t0 = srv.now_ns()
    items, meta = [], []
    for (g, k), at in zip(arrivals, range(len(arrivals))):
        d, segs, off = streams_of_items[g][k]
        src = src_all.data_ptr() + off if d == 1 else 0
        items.append((g, d, segs, src, t0 + at * 2000, len(items)))
        meta.append((g, k))
    tickets = srv.submit(items)
    assert len(tickets) == len(items)
    got = {}
    while len(got) < len(items):
        for c in srv.poll(timeout_us=2_000_000):
            out = None
            if c.dir == 0 and c.len:
                out = staging[c.staging_off:c.staging_off + c.len].cpu().numpy().copy()
                srv.release(c.ticket)
            got[c.tag] = ((c.res.done, c.res.fault_gva, c.res.fault_code), out,
                          (c.arrival_ns, c.admit_ns, c.launch_ns, c.complete_ns))
            # the wave's GPU time: positive, and inside its launch-to-completion span
            assert 0 < c.wave_device_ns <= c.complete_ns - c.launch_ns + 1_000_000
    srv.close()
    per_guest = [[None] * len(x) for x in streams_of_items]
    for tag, (g, k) in enumerate(meta):
        per_guest[g][k] = got[tag]
    out_pools = [pd.cpu().numpy() for pd in pools_d]
    for g in gs:
        g.close()
    return per_guest, out_pools


def _oracle(img, pool_np, wl, src_np):
    pool = pool_np.copy()
    stg = src_np[:wl.staging_bytes].copy()
    res = O.copy_batch([O.Guest.from_image(img, pool)], wl.reqs, wl.segs, stg)
    outs = []
    for r in wl.reqs:
        L = int(wl.segs["len"][r["seg_begin"]:r["seg_begin"] + r["seg_count"]].sum())
        h = int(r["host_off"])
        outs.append(stg[h:h + L].copy() if r["dir"] == 0 and L else None)
    return res, outs, pool


def _arrivals(counts, seed):
    order = np.concatenate([np.full(c, g) for g, c in enumerate(counts)])
    np.random.default_rng(seed).shuffle(order)
    k = [0] * len(counts)
    out = []
    for g in order:
        out.append((int(g), k[g]))
        k[g] += 1
    return out


def test_serving_matches_oracle_per_guest_arrival_order():
    import torch
    imgs, pools = _guests(3)
    wls, items = zip(*[_requests(img, 710 + k, 200) for k, img in enumerate(imgs)])
    src_np = W.payload_bytes(99, max(w.staging_bytes for w in wls))
    src_all = torch.from_numpy(src_np.copy()).cuda()
    arrivals = _arrivals([len(x) for x in items], 5)
    got, out_pools = _serve(imgs, pools, items, src_all, arrivals)
    for g in range(3):
        res, outs, pool = _oracle(imgs[g], pools[g], wls[g], src_np)
        for k in range(len(items[g])):
            (done, fgva, code), out, _t = got[g][k]
            assert (done, fgva, code) == (int(res[k]["done"]), int(res[k]["fault_gva"]), int(res[k]["fault_code"])), (g, k)
            if outs[k] is not None:
                assert np.array_equal(out, outs[k]), (g, k)
        assert np.array_equal(out_pools[g], pool), f"guest {g} memory differs"
        assert (res["fault_code"] != 0).any() and (res["fault_code"] == 0).any()


def test_guest_results_same_alone_and_in_mix():
    import torch
    imgs, pools = _guests(3, seed=720)
    wls, items = zip(*[_requests(img, 730 + k, 150) for k, img in enumerate(imgs)])
    src_np = W.payload_bytes(98, max(w.staging_bytes for w in wls))
    src_all = torch.from_numpy(src_np.copy()).cuda()
    alone, pools_alone = _serve([imgs[0]], [pools[0]], [items[0]], src_all, [(0, k) for k in range(len(items[0]))],
                                max_batch=8)
    mix, pools_mix = _serve(imgs, pools, items, src_all, _arrivals([len(x) for x in items], 6), max_batch=64)
    for k in range(len(items[0])):
        assert alone[0][k][0] == mix[0][k][0], k
        a, m = alone[0][k][1], mix[0][k][1]
        assert (a is None and m is None) or np.array_equal(a, m), k
    assert np.array_equal(pools_alone[0], pools_mix[0])
    # timestamps are ordered
    for g in range(3):
        for (_, _, (arr, adm, lau, com)) in mix[g]:
            assert arr <= adm <= lau <= com


def test_poll_timeout_and_bad_submit():
    import torch
    from paper_1304_3771_b300 import cvd
    imgs, pools = _guests(1, seed=740)
    pd = torch.from_numpy(pools[0]).cuda()
    g = cvd.Guest.from_image(imgs[0], pd)
    staging = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    srv = cvd.Server([g], staging, max_batch=4, max_inflight=4)
    assert srv.poll(timeout_us=1000) == []
    segs = np.array([(imgs[0].data_gva, 16)], dtype=W.SEG_DTYPE)
    with pytest.raises(cvd.CvdError):
        srv.submit([(1, 0, segs, 0, 0, 0)])          # guest 1 of 1
    with pytest.raises(cvd.CvdError):
        big = np.array([(imgs[0].data_gva, 2 << 20)], dtype=W.SEG_DTYPE)
        srv.submit([(0, 0, big, 0, 0, 0)])           # longer than the staging arena
    srv.close()
    g.close()


def test_serving_full_size_one_guest_against_oracle():
    """The serving workload at its measured size and launch configuration:
    8 guests x 4 GiB (4 KiB pages, 2% not present), the tiny mixture with 10%
    YUYV frames, 2 GiB staging, waves of up to 256 requests, 6,000 requests
    arriving at once.  Guest 0's requests are checked completely against the
    oracle run on them in arrival order (results, copied-out bytes and the
    final bytes of every guest page they touch), from a host shadow of guest
    0 holding its tables and the touched pages read before serving."""
    import torch
    from paper_1304_3771_b300 import cvd
    G, N = 8, 6000
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    imgs, pools_d, guests, wls = [], [], [], []
    for k in range(G):
        img = W.make_guest(4 << 30, 740 + k, np_frac=0.02, ro_frac=0.0)
        pool = torch.empty(img.pool_bytes, dtype=torch.uint8, device="cuda")
        for a0 in range(0, pool.numel(), 1 << 30):
            b0 = min(pool.numel(), a0 + (1 << 30))
            pool[a0:b0] = torch.randint(0, 256, (b0 - a0,), dtype=torch.uint8, device="cuda", generator=gen)
        offs, data = W.table_blob(img)
        idx = torch.from_numpy((offs[:, None] + np.arange(4096)[None, :]).reshape(-1)).cuda()
        pool[idx] = torch.from_numpy(data.reshape(-1)).cuda()
        p2m = torch.full((max(img.rsv_n, 1),), -1, dtype=torch.int64, device="cuda")
        imgs.append(img)
        pools_d.append(pool)
        guests.append(cvd.Guest.from_image(img, pool, p2m=p2m))
        wls.append(W.tiny_requests(img, 760 + k, nreq=4000, frame_frac=0.1))
    src_d = torch.randint(0, 256, (64 << 20,), dtype=torch.uint8, device="cuda", generator=gen)
    src_np = src_d.cpu().numpy()
    rng = np.random.default_rng(12)
    gsel, pick = rng.integers(0, G, N), rng.integers(0, 4000, N)
    items, mine = [], []
    for i in range(N):
        wl = wls[gsel[i]]
        r = wl.reqs[pick[i]]
        segs = wl.segs[r["seg_begin"]:r["seg_begin"] + r["seg_count"]].copy()
        L = int(segs["len"].sum())
        so = int(rng.integers(0, (64 << 20) - L)) if r["dir"] == 1 else 0
        items.append((int(gsel[i]), int(r["dir"]), segs, src_d.data_ptr() + so if r["dir"] == 1 else 0, L, so))
        if gsel[i] == 0:
            mine.append(i)
    # host shadow of guest 0: tables plus every page its requests touch, read before serving
    img0 = imgs[0]
    shadow = np.zeros(img0.pool_bytes, dtype=np.uint8)     # lazily backed
    W.write_tables(img0, shadow)
    og = O.Guest.from_image(img0, shadow)
    touched = set()
    for i in mine:
        for s in items[i][2]:
            va, end = int(s["gva"]), int(s["gva"]) + int(s["len"])
            while va < end:
                code, gpa, hpa = og.walk(va, items[i][1] == 1)
                if code:
                    break
                touched.add(hpa >> 12)
                va = (va & ~4095) + 4096
    pages = np.array(sorted(touched), dtype=np.int64)
    pidx = torch.from_numpy(pages).cuda()
    shadow.reshape(-1, 4096)[pages] = torch.index_select(pools_d[0].view(-1, 4096), 0, pidx).cpu().numpy()

    staging = torch.zeros(2 << 30, dtype=torch.uint8, device="cuda")
    srv = cvd.Server(guests, staging, max_batch=256, max_inflight=4096)
    t0 = srv.now_ns()
    srv.submit([(g, d, segs, sp, t0, i) for i, (g, d, segs, sp, L, so) in enumerate(items)])
    got = {}
    while len(got) < N:
        for c in srv.poll(timeout_us=5_000_000):
            out = None
            if c.dir == 0 and c.len and items[c.tag][0] == 0:
                out = staging[c.staging_off:c.staging_off + c.len].cpu().numpy().copy()
            if c.dir == 0 and c.len:
                srv.release(c.ticket)
            got[c.tag] = ((c.res.done, c.res.fault_gva, c.res.fault_code), out)
    srv.close()

    # the oracle: guest 0's requests in arrival order (submission order: all arrive at once)
    reqs = np.zeros(len(mine), dtype=W.REQ_DTYPE)
    segs_all, off, sb = [], 0, 0
    for k, i in enumerate(mine):
        g, d, segs, sp, L, so = items[i]
        reqs[k] = (sb, len(segs), d, 0, off)
        segs_all.append(segs)
        sb += len(segs)
        off += (L + 15) & ~15
    stg = np.zeros(max(off, 16), dtype=np.uint8)
    for k, i in enumerate(mine):
        g, d, segs, sp, L, so = items[i]
        if d == 1:
            stg[int(reqs[k]["host_off"]):int(reqs[k]["host_off"]) + L] = src_np[so:so + L]
    res = O.copy_batch([og], reqs, np.concatenate(segs_all), stg)
    for k, i in enumerate(mine):
        (done, fgva, code), out = got[i]
        assert (done, fgva, code) == (int(res[k]["done"]), int(res[k]["fault_gva"]), int(res[k]["fault_code"])), k
        if out is not None:
            h = int(reqs[k]["host_off"])
            assert np.array_equal(out, stg[h:h + len(out)]), k
    after = torch.index_select(pools_d[0].view(-1, 4096), 0, pidx).cpu().numpy()
    assert np.array_equal(after, shadow.reshape(-1, 4096)[pages])
    assert len(mine) > 600 and (res["fault_code"] != 0).any() and (res["fault_code"] == 0).any()
    for g in guests:
        g.close()


def _with_long_requests(img, seed, nreq):
    """The tiny mixture plus four requests of one 5-6 MiB segment each (over
    the planner's 1,024-page threshold, so the long-segment pass runs in
    their waves), staging laid out request after request."""
    wl = W.tiny_requests(img, seed, nreq=nreq, hi=40000, frame_frac=0.05)
    rng = np.random.default_rng(seed)
    span = img.data_pages * W.PAGE
    longs = [(5 << 20, 0), ((6 << 20) + 100, 1), ((5 << 20) + 4095, 0), (6 << 20, 1)]
    segs = [wl.segs]
    reqs = list(wl.reqs)
    nseg = len(wl.segs)
    for L, d in longs:
        gva = img.data_gva + int(rng.integers(0, span - L))
        segs.append(np.array([(gva, L)], dtype=W.SEG_DTYPE))
        reqs.insert(int(rng.integers(0, len(reqs) + 1)), (nseg, 1, d, 0, 0))
        nseg += 1
    reqs = np.array(reqs, dtype=W.REQ_DTYPE)
    segs = np.concatenate(segs)
    off = 0   # staging in request order
    for i in range(len(reqs)):
        reqs[i]["host_off"] = off
        off += int(segs["len"][reqs[i]["seg_begin"]:reqs[i]["seg_begin"] + reqs[i]["seg_count"]].sum()) + 64
    wl2 = W.CopyWorkload(reqs=reqs, segs=segs, staging_bytes=off, batches=[(0, len(reqs))],
                         payload_bytes=int(segs["len"].sum()))
    items = [(int(r["dir"]), segs[r["seg_begin"]:r["seg_begin"] + r["seg_count"]], int(r["host_off"])) for r in reqs]
    return wl2, items


@pytest.mark.parametrize("two_streams,carve", [(False, False), (True, False), (False, True)])
def test_serving_long_segments_and_two_streams(two_streams, carve):
    """Waves holding segments over 1,024 pages (the server must let the
    long-segment pass run); with CVD_SERVER_TWO_STREAMS, guests spread over
    two streams; with carved pools, guest pages straddling device frames (a
    wave's conflict check must still see a page written from its first byte
    and read from its last ones): every guest's results, copied-out bytes and
    memory equal the oracle run on its requests in arrival order."""
    import torch
    from paper_1304_3771_b300 import cvd
    imgs, pools = _guests(2, seed=760, np_frac=0.0, ro_frac=0.0)   # the long requests complete
    wls, items = zip(*[_with_long_requests(img, 770 + k, 60) for k, img in enumerate(imgs)])
    src_np = W.payload_bytes(97, max(w.staging_bytes for w in wls))
    src_all = torch.from_numpy(src_np.copy()).cuda()
    arrivals = _arrivals([len(x) for x in items], 8)
    got, out_pools = _serve(imgs, pools, items, src_all, arrivals, max_batch=16, two_streams=two_streams, carve=carve)
    for g in range(2):
        res, outs, pool = _oracle(imgs[g], pools[g], wls[g], src_np)
        for k in range(len(items[g])):
            (done, fgva, code), out, _t = got[g][k]
            assert (done, fgva, code) == (int(res[k]["done"]), int(res[k]["fault_gva"]), int(res[k]["fault_code"])), (g, k)
            if outs[k] is not None:
                assert np.array_equal(out, outs[k]), (g, k)
        assert np.array_equal(out_pools[g], pool), f"guest {g} memory differs"
        assert (res["done"] > (4 << 20)).any()
