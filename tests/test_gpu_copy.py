"""GPU parity of the gather/scatter path (Sec. 4.2 copy_from_user /
copy_to_user) against the oracle, bit-exact on results (done, fault gVA,
code), on every staging byte and on every byte of the host pool."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W
from tests.gpu_helpers import assert_same, device_guest, run_both
from tests.oracle_fixtures import golden_pool, parse_golden

pytestmark = pytest.mark.gpu

DEFAULT = dict(vec_bytes=16, unroll=4, chunk_bytes=256 << 10, blocks_per_sm=1, warps_per_block=16, small_bytes=256,
               engine=1, stages=8, stage_bytes=4096, ring_bytes=8320)


@pytest.fixture(autouse=True)
def _reset_params():
    from paper_1304_3771_b300 import cvd
    cvd.set_copy_params(**DEFAULT)
    yield
    assert cvd.stream_check() == 0, "a kernel reported a timed-out wait"
    cvd.set_copy_params(**DEFAULT)


def _tiny(seed=201, nreq=1000):
    img = W.make_guest(64 << 20, seed)
    pool = W.materialize_pool(img)
    wl = W.tiny_requests(img, seed, nreq=nreq)
    stg = W.payload_bytes(seed + 1, wl.staging_bytes)
    return img, pool, wl, stg


def test_tiny_levelled_mixed_directions():
    """Tiny workload: 1000 requests, 1-8 segments, 16 B-64 KiB, 50/50 direction,
    5% non-present and 5% read-only pages, overlapping requests."""
    from paper_1304_3771_b300 import cvd
    img, pool, wl, stg = _tiny()
    out = run_both(img, pool, wl.reqs, wl.segs, stg)
    assert_same(out)
    codes = out["o_res"]["fault_code"]
    assert (codes == 0).sum() > 100 and (codes == 0x101).sum() > 50 and (codes == 2).sum() > 10
    assert cvd.last_levels() > 1


@pytest.mark.parametrize("basic", ["from", "to"])
def test_tiny_basic_calls(basic):
    img, pool, wl, stg = _tiny(202, 400)
    reqs = wl.reqs.copy()
    reqs["dir"] = 0 if basic == "from" else 1
    out = run_both(img, pool, reqs, wl.segs, stg, basic=basic)
    assert_same(out)


def _batched(seed, arena=256 << 20, nreq=3000, huge=0.7, nslots=4, max_segs=32, cap=1 << 20):
    img = W.make_guest(arena, seed, huge_frac=huge, np_frac=0, ro_frac=0, nslots=nslots, slot_gap_pages=512)
    pool = W.materialize_pool(img)
    sizes = np.minimum(W.batching_sizes(seed, nreq), cap)
    wl = W.batched_requests(img, seed, sizes, max_segs)
    return img, pool, wl


@pytest.mark.parametrize("vec,unroll", [(16, 1), (16, 2), (16, 4), (8, 2), (8, 4), (4, 4)])
def test_hazard_free_batch_all_vector_variants(vec, unroll):
    from paper_1304_3771_b300 import cvd
    img, pool, wl = _batched(210)
    lo, hi = wl.batches[0]
    stg = W.payload_bytes(211, wl.staging_bytes)
    out = run_both(img, pool, wl.reqs[lo:hi], wl.segs, stg, flags=cvd.BATCH_HAZARD_FREE,
                   params=dict(engine=0, vec_bytes=vec, unroll=unroll, blocks_per_sm=4, warps_per_block=8))
    assert_same(out)
    assert (out["o_res"]["fault_code"] == 0).all()


@pytest.mark.parametrize("warps,stages,stage,ring", [(8, 4, 4096, 16512), (16, 2, 4096, 4224), (4, 1, 512, 640),
                                                     (8, 3, 8192, 8320), (32, 16, 2048, 4352), (4, 32, 2048, 8192),
                                                     (20, 8, 4096, 8320), (32, 2, 512, 640), (20, 5, 3072, 6272)])
def test_hazard_free_batch_bulk_engine_shapes(warps, stages, stage, ring):
    from paper_1304_3771_b300 import cvd
    img, pool, wl = _batched(218)
    lo, hi = wl.batches[0]
    stg = W.payload_bytes(219, wl.staging_bytes)
    out = run_both(img, pool, wl.reqs[lo:hi], wl.segs, stg, flags=cvd.BATCH_HAZARD_FREE,
                   params=dict(engine=1, warps_per_block=warps, stages=stages, stage_bytes=stage, ring_bytes=ring))
    assert_same(out)


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("chunk,small,bps,wpb", [(4096, 0, 1, 4), (16 << 10, 64, 2, 8), (256 << 10, 4096, 8, 8),
                                                  (1 << 20, 256, 16, 4), (64 << 10, 32, 1, 32)])
def test_hazard_free_batch_chunking(chunk, small, bps, wpb, engine):
    from paper_1304_3771_b300 import cvd
    if engine == 0 and wpb > 8:
        pytest.skip("engine 0 runs 4 or 8 warps per block")
    img, pool, wl = _batched(212, nreq=2000)
    lo, hi = wl.batches[-1]
    stg = W.payload_bytes(213, wl.staging_bytes)
    params = dict(engine=engine, chunk_bytes=chunk, small_bytes=small, blocks_per_sm=bps, warps_per_block=wpb)
    if engine == 1 and wpb > 20:
        params.update(stages=4, ring_bytes=4224)   # 32 rings of 8320 B do not fit in shared memory
    out = run_both(img, pool, wl.reqs[lo:hi], wl.segs, stg, flags=cvd.BATCH_HAZARD_FREE, params=params)
    assert_same(out)


def test_hazard_free_batch_with_faults_4k_pages():
    """Hazard-free batch on a guest with non-present / read-only pages: faults
    end requests mid-stream; copy-from zero-fills, copy-to stops."""
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(128 << 20, 214, np_frac=0.03, ro_frac=0.03)
    pool = W.materialize_pool(img)
    sizes = np.minimum(W.batching_sizes(214, 2000), 300_000)
    wl = W.batched_requests(img, 214, sizes, 16)   # layout ignores faults: they come from the tables
    lo, hi = wl.batches[0]
    stg = W.payload_bytes(215, wl.staging_bytes)
    out = run_both(img, pool, wl.reqs[lo:hi], wl.segs, stg, flags=cvd.BATCH_HAZARD_FREE)
    assert_same(out)
    codes = out["o_res"]["fault_code"]
    assert (codes != 0).sum() > 20 and (codes == 0).sum() > 100


def test_frames_page_aligned_single_segment():
    """Frame workload shape, scaled: one contiguous page-aligned gVA range per frame
    over a permuted 4 KiB guest."""
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(256 << 20, 216, np_frac=0, ro_frac=0)
    pool = W.materialize_pool(img)
    sizes = np.array([640 * 480 * 4, 1920 * 1080 * 4, 320 * 240 * 2, 8_294_400 // 4] * 6)
    wl = W.batched_requests(img, 216, sizes, 1, page_aligned=True)
    stg = W.payload_bytes(217, wl.staging_bytes)
    for lo, hi in wl.batches[:2]:
        out = run_both(img, pool, wl.reqs[lo:hi], wl.segs, stg, flags=cvd.BATCH_HAZARD_FREE)
        assert_same(out)


def test_fault_semantics_hand_tables():
    import torch
    import oracle as O
    from paper_1304_3771_b300 import cvd
    g = parse_golden("walk_hand.txt")
    pool, slots = golden_pool(g)
    pool[0x3000:0x3000 + 10 * 4096] = np.random.default_rng(9).integers(0, 256, 10 * 4096, dtype=np.uint8)
    specs = [
        (0, 0, [(0x0F00, 0x200), (0x1F00, 0x200)]),
        (1, 0x1000, [(0x0800, 0x100), (0x1000, 0x10)]),
        (0, 0x2000, [(0x0010, 0), (0x5000, 0x10)]),
        (0, 0x3000, [(0x0000, 0x10), (0x0000800000000000, 4)]),
        (0, 0x4000, [(0x7FFFFFFFFFF0, 0x20)]),
        (0, 0x5000, [(0x6FF0, 0x20)]),
        (0, 0x5800, [(0x3000, 0x10)]),                 # USER
        (0, 0x5900, [(0x4000, 0x10)]),                 # NOSLOT leaf
        (0, 0x5A00, [(0x10000000000, 0x10)]),          # RSVD
        (1, 0x5B00, [(0x600000, 0x10)]),               # 2 MiB read-only leaf, write
        (0, 0x5C00, [(0x201000, 0x3000)]),             # 2 MiB leaf, clipped at the slot end
    ]
    segs, reqs = [], []
    for d, host, ss in specs:
        reqs.append((len(segs), len(ss), d, 0, host))
        segs.extend(ss)
    reqs = np.array(reqs, dtype=W.REQ_DTYPE)
    segs = np.array(segs, dtype=W.SEG_DTYPE)
    stg = np.full(0x9000, 0xEE, np.uint8)
    o_pool, o_stg = pool.copy(), stg.copy()
    o_res = O.copy_batch([O.Guest(o_pool, slots, g["cr3"])], reqs, segs, o_stg)
    for flags in (0, cvd.BATCH_HAZARD_FREE):
        pool_d = torch.from_numpy(pool.copy()).cuda()
        gg = cvd.Guest(pool_d, slots, g["cr3"])
        stg_d = torch.from_numpy(stg.copy()).cuda()
        res_d = torch.zeros(len(reqs) * 24, dtype=torch.uint8, device="cuda")
        cvd.copy_batch([gg], cvd.records_to_device(reqs), len(reqs), cvd.records_to_device(segs), len(segs),
                       stg_d, res_d, flags=flags)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(cvd.records_from_device(res_d, W.RESULT_DTYPE, len(reqs)), o_res)
        assert np.array_equal(stg_d.cpu().numpy(), o_stg)
        assert np.array_equal(pool_d.cpu().numpy(), o_pool)
        gg.close()


def test_malformed_and_empty():
    import torch
    from paper_1304_3771_b300 import cvd
    img, pool, wl, stg = _tiny(220, 50)
    reqs = wl.reqs.copy()
    reqs["dir"][3] = 7                       # BADREQ
    reqs["guest"][5] = 3                     # BADREQ (1 guest)
    reqs["seg_begin"][7] = len(wl.segs)      # BADREQ (segments out of range)
    reqs["host_off"][9] = len(stg) - 1       # HOSTBUF
    out = run_both(img, pool, reqs, wl.segs, stg)
    assert_same(out)
    assert out["g_res"]["fault_code"][[3, 5, 7]].tolist() == [9, 9, 9]
    assert out["g_res"]["fault_code"][9] == 8
    g, _ = device_guest(img, pool)
    z = torch.zeros(16, dtype=torch.uint8, device="cuda")
    cvd.copy_batch([g], z, 0, z, 0, z, z)   # nreq = 0 is a no-op
    with pytest.raises(cvd.CvdError):       # staging overlapping the guest pool
        cvd.copy_batch([g], cvd.records_to_device(reqs), len(reqs), cvd.records_to_device(wl.segs), len(wl.segs),
                       g.pool[:1024], z)
    g.close()


def test_shared_segments_capacity_rule():
    """Requests that reuse segment descriptors beyond the segment array length
    fault with BADREQ exactly where the oracle says."""
    img = W.make_guest(64 << 20, 221, np_frac=0, ro_frac=0)
    pool = W.materialize_pool(img)
    segs = np.array([(img.data_gva + 100, 50), (img.data_gva + 9000, 70), (img.data_gva + 20000, 30)],
                    dtype=W.SEG_DTYPE)
    reqs = np.array([(0, 2, 0, 0, 0), (1, 2, 0, 0, 200), (0, 1, 1, 0, 400), (2, 1, 0, 0, 600)], dtype=W.REQ_DTYPE)
    out = run_both(img, pool, reqs, segs, W.payload_bytes(3, 1000))
    assert_same(out)
    assert out["g_res"]["fault_code"].tolist() == [0, 9, 9, 9]


def test_multi_guest_batch():
    """Two guests in one host pool, one mixed (levelled) batch, requests of
    both guests interleaved."""
    import torch
    import oracle as O
    from paper_1304_3771_b300 import cvd
    a = W.make_guest(64 << 20, 230, host_base=0x10000)
    b = W.make_guest(64 << 20, 231, host_base=a.pool_bytes + 0x20000)
    pool = np.zeros(b.pool_bytes, np.uint8)
    W.materialize_pool(a, pool)
    W.materialize_pool(b, pool)
    wa = W.tiny_requests(a, 230, nreq=300)
    wb = W.tiny_requests(b, 231, nreq=300, guest=1)
    segs = np.concatenate([wa.segs, wb.segs])
    rb = wb.reqs.copy()
    rb["seg_begin"] += len(wa.segs)
    rb["host_off"] += wa.staging_bytes
    reqs = np.concatenate([wa.reqs, rb])[np.random.default_rng(1).permutation(600)]
    stg = W.payload_bytes(5, wa.staging_bytes + wb.staging_bytes)
    o_pool, o_stg = pool.copy(), stg.copy()
    o_res = O.copy_batch([O.Guest.from_image(a, o_pool), O.Guest.from_image(b, o_pool)], reqs, segs, o_stg)
    pool_d = torch.from_numpy(pool).cuda()
    ga, gb = cvd.Guest.from_image(a, pool_d), cvd.Guest.from_image(b, pool_d)
    stg_d = torch.from_numpy(stg.copy()).cuda()
    res_d = torch.zeros(len(reqs) * 24, dtype=torch.uint8, device="cuda")
    cvd.copy_batch([ga, gb], cvd.records_to_device(reqs), len(reqs), cvd.records_to_device(segs), len(segs), stg_d,
                   res_d)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cvd.records_from_device(res_d, W.RESULT_DTYPE, len(reqs)), o_res)
    assert np.array_equal(stg_d.cpu().numpy(), o_stg)
    assert np.array_equal(pool_d.cpu().numpy(), o_pool)
    ga.close()
    gb.close()


@pytest.mark.parametrize("flags", ["levelled", "hazard_free"])
def test_batch_at_the_guest_limit(flags):
    """64 guests (CVD_MAX_GUESTS_PER_BATCH), each in its own host pool, one
    batch with their requests interleaved -- every result, every staging byte
    and every guest's memory against the oracle."""
    import torch
    import oracle as O
    from paper_1304_3771_b300 import cvd
    G = 64
    imgs = [W.make_guest(8 << 20, 800 + k, np_frac=0.03, ro_frac=0.03) for k in range(G)]
    pools = [W.materialize_pool(img) for img in imgs]
    reqs, segs, off = [], [], 0
    for k, img in enumerate(imgs):
        if flags == "levelled":
            wl = W.tiny_requests(img, 900 + k, nreq=20, hi=20000, guest=k)
        else:   # one request per guest: requests of different guests never share bytes
            wl = W.tiny_requests(img, 900 + k, nreq=1, hi=20000, guest=k)
        r = wl.reqs.copy()
        r["seg_begin"] += sum(len(x) for x in segs)
        r["host_off"] += off
        off += wl.staging_bytes
        reqs.append(r)
        segs.append(wl.segs)
    reqs = np.concatenate(reqs)
    reqs = reqs[np.random.default_rng(801).permutation(len(reqs))]
    segs = np.concatenate(segs)
    stg = W.payload_bytes(802, off)
    o_pools, o_stg = [p.copy() for p in pools], stg.copy()
    o_res = O.copy_batch([O.Guest.from_image(img, p) for img, p in zip(imgs, o_pools)], reqs, segs, o_stg)
    made = [device_guest(img, p) for img, p in zip(imgs, pools)]
    stg_d = torch.from_numpy(stg.copy()).cuda()
    res_d = torch.zeros(len(reqs) * W.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cvd.copy_batch([g for g, _ in made], cvd.records_to_device(reqs), len(reqs), cvd.records_to_device(segs),
                   len(segs), stg_d, res_d, flags=cvd.BATCH_HAZARD_FREE if flags == "hazard_free" else 0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cvd.records_from_device(res_d, W.RESULT_DTYPE, len(reqs)), o_res)
    assert np.array_equal(stg_d.cpu().numpy(), o_stg)
    for (g, pd), op in zip(made, o_pools):
        assert np.array_equal(pd.cpu().numpy(), op)
        g.close()


def test_graph_replay_and_check_flag():
    import torch
    import oracle as O
    from paper_1304_3771_b300 import cvd
    img, pool, wl = _batched(240, nreq=1500)
    lo, hi = wl.batches[0]
    reqs = wl.reqs[lo:hi].copy()
    reqs["dir"] = 0            # gather only: repeating the call is idempotent
    stg = W.payload_bytes(241, wl.staging_bytes)
    o_pool, o_stg = pool.copy(), stg.copy()
    o_res = O.copy_batch([O.Guest.from_image(img, o_pool)], reqs, wl.segs, o_stg)
    g, pool_d = device_guest(img, pool)
    req_d, seg_d = cvd.records_to_device(reqs), cvd.records_to_device(wl.segs)
    stg_d = torch.zeros(len(stg), dtype=torch.uint8, device="cuda")
    res_d = torch.zeros(len(reqs) * 24, dtype=torch.uint8, device="cuda")
    mask = np.zeros(len(stg), bool)
    L = [int(wl.segs["len"][r["seg_begin"]:r["seg_begin"] + r["seg_count"]].sum()) for r in reqs]
    for r, ln in zip(reqs, L):
        mask[r["host_off"]:r["host_off"] + ln] = True
    for _ in range(3):
        stg_d.fill_(0xAB)
        cvd.copy_batch([g], req_d, len(reqs), seg_d, len(wl.segs), stg_d, res_d,
                       flags=cvd.BATCH_HAZARD_FREE | cvd.BATCH_GRAPH)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(cvd.records_from_device(res_d, W.RESULT_DTYPE, len(reqs)), o_res)
        got = stg_d.cpu().numpy()
        assert np.array_equal(got[mask], o_stg[mask])
        assert (got[~mask] == 0xAB).all()
    # CHECK accepts this hazard-free batch ...
    cvd.copy_batch([g], req_d, len(reqs), seg_d, len(wl.segs), stg_d, res_d,
                   flags=cvd.BATCH_HAZARD_FREE | cvd.BATCH_CHECK)
    # ... and rejects one with two writers of the same guest bytes
    bad = reqs[:2].copy()
    bad["dir"] = 1
    segs2 = wl.segs.copy()
    segs2["gva"][bad[1]["seg_begin"]] = segs2["gva"][bad[0]["seg_begin"]]
    with pytest.raises(cvd.CvdError) as ei:
        cvd.copy_batch([g], cvd.records_to_device(bad), 2, cvd.records_to_device(segs2), len(segs2), stg_d, res_d,
                       flags=cvd.BATCH_HAZARD_FREE | cvd.BATCH_CHECK)
    assert ei.value.status == cvd.EHAZARD
    g.close()


def test_host_buffer_batch():
    import torch
    import oracle as O
    from paper_1304_3771_b300 import cvd
    img, pool, wl = _batched(250, nreq=800)
    lo, hi = wl.batches[0]
    reqs = wl.reqs[lo:hi]
    stg = W.payload_bytes(251, wl.staging_bytes)
    o_pool, o_stg = pool.copy(), stg.copy()
    o_res = O.copy_batch([O.Guest.from_image(img, o_pool)], reqs, wl.segs, o_stg)
    g, pool_d = device_guest(img, pool)
    h_req = torch.from_numpy(np.ascontiguousarray(reqs).view(np.uint8).copy()).pin_memory()
    h_seg = torch.from_numpy(wl.segs.view(np.uint8).copy()).pin_memory()
    h_stg = torch.from_numpy(stg.copy()).pin_memory()
    h_res = torch.zeros(len(reqs) * 24, dtype=torch.uint8).pin_memory()
    cvd.copy_batch_host([g], h_req, len(reqs), h_seg, len(wl.segs), h_stg, h_res, flags=cvd.BATCH_HAZARD_FREE)
    np.testing.assert_array_equal(h_res.numpy().view(W.RESULT_DTYPE), o_res)
    assert np.array_equal(h_stg.numpy(), o_stg)
    assert np.array_equal(pool_d.cpu().numpy(), o_pool)
    g.close()


@pytest.mark.parametrize("flags", ["hazard_free", "levelled"])
def test_long_segments_with_faults(flags):
    """Segments of 0.5-24 MiB (many 256-page blocks each, walked across the
    grid) over a guest with scattered not-present and read-only pages: first
    faults in late blocks, after earlier long segments, in either direction."""
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(512 << 20, 262, huge_frac=0.3, np_frac=0.002, ro_frac=0.002, nslots=3)
    pool = W.materialize_pool(img)
    rng = np.random.default_rng(262)
    sizes = W.log_uniform(rng, 2 << 20, 24 << 20, 40)
    wl = W.batched_requests(img, 262, sizes, 4)
    lo, hi = wl.batches[0]
    stg = W.payload_bytes(263, wl.staging_bytes)
    f = cvd.BATCH_HAZARD_FREE if flags == "hazard_free" else 0
    out = run_both(img, pool, wl.reqs[lo:hi], wl.segs, stg, flags=f)
    assert_same(out)
    codes = out["o_res"]["fault_code"]
    assert (codes != 0).any() and (codes == 0).any()
    assert (out["o_res"]["done"][codes != 0] > (1 << 20)).any()   # some first faults deep inside


def _host_call(img, pool, reqs, segs, stg, flags):
    import torch
    from paper_1304_3771_b300 import cvd
    g, pool_d = device_guest(img, pool)
    h_req = torch.from_numpy(np.ascontiguousarray(reqs).view(np.uint8).copy()).pin_memory()
    h_seg = torch.from_numpy(np.ascontiguousarray(segs).view(np.uint8).copy()).pin_memory()
    h_stg = torch.from_numpy(stg.copy()).pin_memory()
    h_res = torch.zeros(len(reqs) * 24, dtype=torch.uint8).pin_memory()
    cvd.copy_batch_host([g], h_req, len(reqs), h_seg, len(segs), h_stg, h_res, flags=flags)
    out = h_res.numpy().view(W.RESULT_DTYPE).copy(), h_stg.numpy().copy(), pool_d.cpu().numpy()
    g.close()
    return out


def test_host_buffer_grouped_layout_moves_only_request_ranges():
    """Copy-to sources first, copy-from destinations after them, with gaps:
    every byte of the host buffer (gaps included) ends as the oracle leaves it."""
    import oracle as O
    from paper_1304_3771_b300 import cvd
    img, pool, wl = _batched(252, nreq=800)
    lo, hi = wl.batches[0]
    reqs = wl.reqs[lo:hi].copy()
    L = np.add.reduceat(wl.segs["len"].astype(np.int64), reqs["seg_begin"].astype(np.int64))
    L[reqs["seg_count"] == 0] = 0
    off, cur = np.zeros(len(reqs), dtype=np.uint64), 0
    for d in (1, 0):
        for i in np.nonzero(reqs["dir"] == d)[0]:
            off[i] = cur
            cur += int(L[i]) + 16 * (1 + i % 7)          # ragged gaps
    reqs["host_off"] = off
    stg = W.payload_bytes(253, cur + 4096)
    o_pool, o_stg = pool.copy(), stg.copy()
    o_res = O.copy_batch([O.Guest.from_image(img, o_pool)], reqs, wl.segs, o_stg)
    res, h_stg, d_pool = _host_call(img, pool, reqs, wl.segs, stg, cvd.BATCH_HAZARD_FREE)
    np.testing.assert_array_equal(res, o_res)
    assert np.array_equal(h_stg, o_stg)
    assert np.array_equal(d_pool, o_pool)


def test_host_buffer_levelled_with_malformed_requests():
    """Overlapping tiny-workload requests (levelled) plus requests the device rejects
    (guest out of range, staging range outside the buffer, dir > 1): rejected
    copy-from ranges must come back untouched."""
    import oracle as O
    img = W.make_guest(64 << 20, 254)
    pool = W.materialize_pool(img)
    wl = W.tiny_requests(img, 254, nreq=400, frame_frac=0.05)
    reqs = wl.reqs.copy()
    reqs["guest"][5::37] = 3
    reqs["dir"][7::41] = 2
    reqs["host_off"][11::43] = wl.staging_bytes + 1
    stg = W.payload_bytes(255, wl.staging_bytes)
    o_pool, o_stg = pool.copy(), stg.copy()
    o_res = O.copy_batch([O.Guest.from_image(img, o_pool)], reqs, wl.segs, o_stg)
    assert (o_res["fault_code"] == 9).any() and (o_res["fault_code"] == 8).any()
    res, h_stg, d_pool = _host_call(img, pool, reqs, wl.segs, stg, 0)
    np.testing.assert_array_equal(res, o_res)
    assert np.array_equal(h_stg, o_stg)
    assert np.array_equal(d_pool, o_pool)


@pytest.mark.parametrize("buffers", ["alternate", "shared"])
def test_host_batches_pipelined_equal_sequential_batches(buffers):
    """cvd_copy_batches_host over 5 hazard-free batches of one guest (later
    batches read guest bytes earlier ones wrote) equals the oracle applying
    them in order.  'alternate': batches use two host buffers in turn
    (transfers overlap); 'shared': every batch uses one buffer (each batch's
    inputs wait for the previous batch's write-back)."""
    import torch
    import oracle as O
    from paper_1304_3771_b300 import cvd
    img, pool, wl = _batched(257, arena=64 << 20, nreq=3000)
    assert len(wl.batches) >= 4
    nbuf = 2 if buffers == "alternate" else 1
    bufs = [W.payload_bytes(258 + k, wl.staging_bytes) for k in range(nbuf)]
    parts = []
    for lo, hi in wl.batches:
        r = wl.reqs[lo:hi].copy()
        s0 = int(r["seg_begin"][0])
        s1 = int(r["seg_begin"][-1] + r["seg_count"][-1])
        r["seg_begin"] -= s0
        parts.append((r, wl.segs[s0:s1].copy()))
    o_pool, o_bufs = pool.copy(), [b.copy() for b in bufs]
    og = O.Guest.from_image(img, o_pool)
    o_res = [O.copy_batch([og], r, sg, o_bufs[i % nbuf]) for i, (r, sg) in enumerate(parts)]
    g, pool_d = device_guest(img, pool)
    h_bufs = [torch.from_numpy(b.copy()).pin_memory() for b in bufs]
    items = []
    for i, (r, sg) in enumerate(parts):
        items.append((torch.from_numpy(np.ascontiguousarray(r).view(np.uint8).copy()).pin_memory(), len(r),
                      torch.from_numpy(np.ascontiguousarray(sg).view(np.uint8).copy()).pin_memory(), len(sg),
                      h_bufs[i % nbuf], torch.zeros(len(r) * 24, dtype=torch.uint8).pin_memory()))
    cvd.copy_batches_host([g], items, flags=cvd.BATCH_HAZARD_FREE)
    for i in range(len(parts)):
        np.testing.assert_array_equal(items[i][5].numpy().view(W.RESULT_DTYPE), o_res[i])
    for k in range(nbuf):
        assert np.array_equal(h_bufs[k].numpy(), o_bufs[k]), k
    assert np.array_equal(pool_d.cpu().numpy(), o_pool)
    g.close()


def test_tune_picks_a_valid_candidate():
    import torch
    from paper_1304_3771_b300 import cvd
    img, pool, wl = _batched(260, nreq=1000)
    lo, hi = wl.batches[0]
    reqs = wl.reqs[lo:hi].copy()
    reqs["dir"] = 0
    g, pool_d = device_guest(img, pool)
    stg_d = torch.zeros(wl.staging_bytes, dtype=torch.uint8, device="cuda")
    res_d = torch.zeros(len(reqs) * 24, dtype=torch.uint8, device="cuda")
    p, ms = cvd.tune([g], cvd.records_to_device(reqs), len(reqs), cvd.records_to_device(wl.segs), len(wl.segs),
                     stg_d, res_d, reps=1)
    assert ms > 0 and p.engine in (0, 1)
    assert cvd.get_copy_params().as_dict() == p.as_dict()
    g.close()


def test_tune_batches_times_the_step_caches_and_stays_exact():
    """cvd_tune_batches times whole planned-ahead steps, keeps a valid
    bulk-copy engine shape for the device, returns it from its cache on the
    same shape, and the step under the chosen parameters still equals the
    oracle (fresh data after tuning, which repeats the batches)."""
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(64 << 20, 482, huge_frac=0.5, np_frac=0.002, ro_frac=0.002, nslots=3)
    pool = W.materialize_pool(img)
    wl = W.batched_requests(img, 482, W.batching_sizes(482, 2500), 8)
    assert len(wl.batches) >= 2
    stg = W.payload_bytes(483, wl.staging_bytes)
    seg_d = cvd.records_to_device(wl.segs)
    items, outs = [], []
    for lo, hi in wl.batches:
        o = torch.zeros((hi - lo) * 24, dtype=torch.uint8, device="cuda")
        items.append((cvd.records_to_device(wl.reqs[lo:hi]), hi - lo, seg_d, len(wl.segs), o))
        outs.append(o)
    g, pool_d = device_guest(img, pool)
    stg_d = torch.from_numpy(stg.copy()).cuda()
    p, ms, cached = cvd.tune_batches([g], items, stg_d, reps=1)
    assert ms > 0 and p.engine == 1 and not cached
    assert cvd.get_copy_params().as_dict() == p.as_dict()
    p2, ms2, cached2 = cvd.tune_batches([g], items, stg_d, reps=1)
    assert cached2 and p2.as_dict() == p.as_dict() and ms2 == ms
    g.close()
    # the tuned step on fresh data against the oracle
    o_pool, o_stg = pool.copy(), stg.copy()
    og = O.Guest.from_image(img, o_pool)
    o_res = [O.copy_batch([og], wl.reqs[lo:hi], wl.segs, o_stg) for lo, hi in wl.batches]
    g, pool_d = device_guest(img, pool)
    stg_d = torch.from_numpy(stg.copy()).cuda()
    cvd.copy_batches([g], items, stg_d)
    torch.cuda.synchronize()
    for (lo, hi), o, e in zip(wl.batches, outs, o_res):
        np.testing.assert_array_equal(cvd.records_from_device(o, W.RESULT_DTYPE, hi - lo), e)
    assert np.array_equal(stg_d.cpu().numpy(), o_stg)
    assert np.array_equal(pool_d.cpu().numpy(), o_pool)
    g.close()


def test_copy_batches_planned_ahead_equal_sequential_calls():
    """cvd_copy_batches (batch i + 1 planned while batch i copies) gives the
    results, staging bytes and guest memory of the oracle running the batches
    one after another."""
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(64 << 20, 480, huge_frac=0.5, np_frac=0.002, ro_frac=0.002, nslots=3)
    pool = W.materialize_pool(img)
    sizes = np.concatenate([W.batching_sizes(480, 3000), W.log_uniform(np.random.default_rng(480), 2 << 20, 6 << 20, 6)])
    wl = W.batched_requests(img, 480, sizes, 8)
    assert len(wl.batches) >= 3
    stg = W.payload_bytes(481, wl.staging_bytes)
    o_pool, o_stg = pool.copy(), stg.copy()
    og = O.Guest.from_image(img, o_pool)
    o_res = []
    for lo, hi in wl.batches:
        o_res.append(O.copy_batch([og], wl.reqs[lo:hi], wl.segs, o_stg))
    pool_d = torch.from_numpy(pool.copy()).cuda()
    g = cvd.Guest.from_image(img, pool_d)
    stg_d = torch.from_numpy(stg.copy()).cuda()
    seg_d = cvd.records_to_device(wl.segs)
    items, outs = [], []
    for lo, hi in wl.batches:
        r = cvd.records_to_device(wl.reqs[lo:hi])
        o = torch.zeros((hi - lo) * 24, dtype=torch.uint8, device="cuda")
        items.append((r, hi - lo, seg_d, len(wl.segs), o))
        outs.append(o)
    stream = torch.cuda.Stream()
    cvd.copy_batches([g], items, stg_d, stream=stream)
    stream.synchronize()
    for (lo, hi), o, e in zip(wl.batches, outs, o_res):
        np.testing.assert_array_equal(cvd.records_from_device(o, W.RESULT_DTYPE, hi - lo), e)
    assert np.array_equal(stg_d.cpu().numpy(), o_stg)
    assert np.array_equal(pool_d.cpu().numpy(), o_pool)
    g.close()


def test_levelled_calls_of_different_sizes_on_one_stream():
    """Levelled calls on one stream share its scratch (run lists, marks,
    pinned copies): a first call of ~8,000 runs with conflicts (the buffers
    grow), the same call again (reused at their size), then a small call
    after the large ones -- each bit-exact against the oracle."""
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(64 << 20, 461, huge_frac=0.0, np_frac=0.02, ro_frac=0.02)
    pool = W.materialize_pool(img)
    big = W.tiny_requests(img, 461, nreq=600)
    small = W.tiny_requests(img, 462, nreq=60)
    assert int(big.reqs["seg_count"].sum()) > 2000 and big.payload_bytes > (16 << 20)   # > 4,096 runs
    st = torch.cuda.Stream()
    for wl, seed in ((big, 463), (big, 463), (small, 464)):
        stg = W.payload_bytes(seed, wl.staging_bytes)
        o_pool, o_stg = pool.copy(), stg.copy()
        o_res = O.copy_batch([O.Guest.from_image(img, o_pool)], wl.reqs, wl.segs, o_stg)
        g, pool_d = device_guest(img, pool)
        stg_d = torch.from_numpy(stg.copy()).cuda()
        res_d = torch.zeros(len(wl.reqs) * W.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        req_d, seg_d = cvd.records_to_device(wl.reqs), cvd.records_to_device(wl.segs)
        torch.cuda.synchronize()
        cvd.copy_batch([g], req_d, len(wl.reqs), seg_d, len(wl.segs), stg_d, res_d, stream=st)
        st.synchronize()
        np.testing.assert_array_equal(cvd.records_from_device(res_d, W.RESULT_DTYPE, len(wl.reqs)), o_res)
        assert np.array_equal(stg_d.cpu().numpy(), o_stg) and np.array_equal(pool_d.cpu().numpy(), o_pool)
        if wl is big:
            assert cvd.last_levels(st) > 1
        g.close()


@pytest.mark.parametrize("flags,engine", [(0, 1), (1, 1), (1, 0)])
def test_staging_view_at_odd_offsets_keeps_its_guards(flags, engine):
    """The staging buffer is a view starting at an odd byte of a larger
    allocation and ending at an odd length, with guard bytes on both sides:
    reads of whole aligned 16-byte blocks may touch the guards, never write
    them, and every result and byte inside equals the oracle."""
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(128 << 20, 231, huge_frac=0.5, np_frac=0.02, ro_frac=0.02, nslots=2, slot_gap_pages=512)
    pool = W.materialize_pool(img)
    if flags:
        wl = W.batched_requests(img, 231, np.minimum(W.batching_sizes(231, 2500), 200_000), 32)
        lo, hi = wl.batches[0]
        reqs = wl.reqs[lo:hi]
    else:
        wl = W.tiny_requests(img, 231, nreq=600)
        reqs = wl.reqs
    n = wl.staging_bytes | 1                  # odd length
    stg = W.payload_bytes(232, n)
    o_pool, o_stg = pool.copy(), stg.copy()
    o_res = O.copy_batch([O.Guest.from_image(img, o_pool)], reqs, wl.segs, o_stg)
    guard = 4099
    big = torch.from_numpy(np.concatenate([np.full(guard, 0xA5, np.uint8), stg,
                                           np.full(guard, 0x5A, np.uint8)])).cuda()
    view = big[guard:guard + n]
    assert view.data_ptr() % 16 != 0
    g, pool_d = device_guest(img, pool)
    res_d = torch.zeros(len(reqs) * 24, dtype=torch.uint8, device="cuda")
    cvd.set_copy_params(engine=engine, **({} if engine else dict(warps_per_block=8, blocks_per_sm=4)))
    cvd.copy_batch([g], cvd.records_to_device(reqs), len(reqs), cvd.records_to_device(wl.segs), len(wl.segs), view,
                   res_d, flags=flags)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cvd.records_from_device(res_d, W.RESULT_DTYPE, len(reqs)), o_res)
    host = big.cpu().numpy()
    assert (host[:guard] == 0xA5).all() and (host[guard + n:] == 0x5A).all(), "a guard byte changed"
    assert np.array_equal(host[guard:guard + n], o_stg), "staging bytes differ from the oracle"
    assert np.array_equal(pool_d.cpu().numpy(), o_pool), "guest memory differs from the oracle"
    g.close()


def _levelled_launches(img, pool, reqs, segs, stg):
    """Run a levelled call (no flags) against the oracle; returns the kernel
    launches of a second identical call on the device and its levels (equal
    results each time)."""
    import torch
    from paper_1304_3771_b300 import cvd
    out = run_both(img, pool, reqs, segs, stg)
    assert_same(out)
    g, pool_d = device_guest(img, pool)
    req_d, seg_d = cvd.records_to_device(reqs), cvd.records_to_device(segs)
    stg_d = torch.from_numpy(stg.copy()).cuda()
    res_d = torch.zeros(len(reqs) * 24, dtype=torch.uint8, device="cuda")
    cvd.copy_batch([g], req_d, len(reqs), seg_d, len(segs), stg_d, res_d)
    torch.cuda.synchronize()
    n0 = cvd.launch_count()
    cvd.copy_batch([g], req_d, len(reqs), seg_d, len(segs), stg_d, res_d)
    torch.cuda.synchronize()
    n = cvd.launch_count() - n0
    levels = cvd.last_levels()
    g.close()
    return n, levels


def levelled_kernels(nreq):
    """Sizing, the scan (one kernel up to 2,048 requests, else three), plan,
    long-segment scan, frame insert, staging order, marks and the parallel
    copy; the ordered pass comes on top when requests were marked."""
    return 7 + (1 if nreq <= 2048 else 3)


def test_levelled_conflict_free_call_runs_in_one_parallel_pass():
    """A levelled call whose requests touch disjoint 4 KiB frames and staging
    ranges in order (a generator batch with page-aligned segments) marks
    nothing: every request runs in the parallel launch (one level, no
    ordered pass)."""
    img = W.make_guest(256 << 20, 233, huge_frac=0.5, np_frac=0.02, ro_frac=0.02, nslots=4, slot_gap_pages=512)
    pool = W.materialize_pool(img)
    wl = W.batched_requests(img, 233, np.minimum(W.batching_sizes(233, 2000), 300_000), 32, page_aligned=True)
    lo, hi = wl.batches[0]
    stg = W.payload_bytes(234, wl.staging_bytes)
    n, levels = _levelled_launches(img, pool, wl.reqs[lo:hi], wl.segs, stg)
    assert n == levelled_kernels(hi - lo) and levels == 1, (n, levels)


def test_levelled_shared_frames_and_unordered_staging_run_in_order():
    """Byte-disjoint requests sharing a 4 KiB frame with a writer, a copy-to
    request writing one frame from two segments, and staging ranges out of
    request order: the conservative device check marks them and they run in
    index order after the parallel launch (two levels); every result equals
    the oracle's."""
    img = W.make_guest(64 << 20, 235, np_frac=0, ro_frac=0)
    pool = W.materialize_pool(img)
    base = img.data_gva + 40 * 4096
    segs = np.zeros(6, dtype=W.SEG_DTYPE)
    segs["gva"] = [base, base + 1000, base + 3 * 4096, base + 3 * 4096 + 64, base + 9 * 4096, base + 9 * 4096 + 16]
    segs["len"] = [500, 600, 64, 64, 32, 32]
    reqs = np.zeros(5, dtype=W.REQ_DTYPE)
    reqs["seg_begin"] = [0, 1, 2, 3, 4]
    reqs["seg_count"] = [1, 1, 1, 1, 2]
    reqs["dir"] = [1, 0, 0, 0, 1]                          # a write and a read in one frame
    reqs["host_off"] = [0, 1024, 8192, 4096, 12288]        # requests 2 and 3 out of order
    stg = W.payload_bytes(236, 16384)
    for sel in ([0, 1], [2, 3], [4]):
        n, levels = _levelled_launches(img, pool, reqs[sel], segs, stg)
        assert n == levelled_kernels(len(sel)) + 1 and levels == 2, (sel, n, levels)


_TUNE_CHILD = r'''
import json, sys
sys.path.insert(0, sys.argv[1])
import torch
from paper_1304_3771_b300 import cvd
from paper_1304_3771_b300 import workload as W
img = W.make_guest(64 << 20, 482, huge_frac=0.5, np_frac=0.002, ro_frac=0.002, nslots=3)
pool = torch.from_numpy(W.materialize_pool(img)).cuda()
wl = W.batched_requests(img, 482, W.batching_sizes(482, 2500), 8)
seg_d = cvd.records_to_device(wl.segs)
items = [(cvd.records_to_device(wl.reqs[lo:hi]), hi - lo, seg_d, len(wl.segs),
          torch.zeros((hi - lo) * 24, dtype=torch.uint8, device="cuda")) for lo, hi in wl.batches]
g = cvd.Guest.from_image(img, pool)
stg = torch.zeros(wl.staging_bytes, dtype=torch.uint8, device="cuda")
p, ms, cached = cvd.tune_batches([g], items, stg, reps=1)
print(json.dumps({"params": p.as_dict(), "ms": ms, "cached": bool(cached)}))
'''


def test_tune_cache_file_carries_choices_across_processes(tmp_path):
    """With CVD_TUNE_CACHE naming a file, a process's tuned choice is
    appended to it and a later process gets it from the file without timing
    (cached, same parameters and time)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.tsv"
    env = dict(os.environ, CVD_TUNE_CACHE=str(cache))
    runs = []
    for _ in range(2):
        out = subprocess.run([sys.executable, "-c", _TUNE_CHILD, root], env=env, capture_output=True, text=True,
                             timeout=600)
        assert out.returncode == 0, out.stderr[-2000:]
        runs.append(json.loads(out.stdout.strip().splitlines()[-1]))
    assert not runs[0]["cached"] and runs[1]["cached"]
    assert runs[1]["params"] == runs[0]["params"] and abs(runs[1]["ms"] - runs[0]["ms"]) < 1e-3
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith(torch_gpu_name())


def torch_gpu_name():
    import torch
    return torch.cuda.get_device_name(0)


def test_levelled_copy_to_segments_overwrite_in_order_beside_a_reader():
    """A copy-to request whose two segments write the same bytes (the later
    segment must win) in a frame another request also reads: the frame
    conflicts, both requests go to the ordered pass, and the copy-to
    request's segments must still take effect one after another.  Repeated,
    because which request the frame table records first is a race of the
    insert pass; every run equals the oracle."""
    img = W.make_guest(64 << 20, 237, np_frac=0, ro_frac=0)
    pool = W.materialize_pool(img)
    base = img.data_gva + 70 * 4096
    segs = np.zeros(4, dtype=W.SEG_DTYPE)
    segs["gva"] = [base + 100, base + 512, base + 512 + 64, base + 3000]
    segs["len"] = [1500, 700, 700, 200]
    reqs = np.zeros(3, dtype=W.REQ_DTYPE)
    reqs["seg_begin"] = [0, 1, 3]
    reqs["seg_count"] = [1, 2, 1]
    reqs["dir"] = [0, 1, 0]                    # a reader, the overwriting writer, a reader after it
    reqs["host_off"] = [0, 2048, 4096]
    for rep in range(20):
        stg = W.payload_bytes(238 + rep, 8192)
        out = run_both(img, pool, reqs, segs, stg)
        assert_same(out)
        assert np.array_equal(out["g_pool"], out["o_pool"]), rep


def test_levelled_conflicts_with_a_pool_off_4k_alignment():
    """The guest pool is a view 512 bytes past a 4 KiB boundary (as a caching
    allocator hands out), so every guest page straddles two device frames.
    Copy-to requests write whole pages and later copy-from requests read
    their last 300 bytes: the conflict check must see each pair as touching
    the same page, whichever byte each access starts at, and order them.
    Repeated against the oracle."""
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(64 << 20, 239, np_frac=0, ro_frac=0)
    pool = W.materialize_pool(img)
    npairs = 64
    pages = img.data_gva + (100 + 2 * np.arange(npairs, dtype=np.uint64)) * 4096
    segs = np.zeros(2 * npairs, dtype=W.SEG_DTYPE)
    segs["gva"][0::2] = pages
    segs["len"][0::2] = 4096
    segs["gva"][1::2] = pages + 3796
    segs["len"][1::2] = 300
    reqs = np.zeros(2 * npairs, dtype=W.REQ_DTYPE)
    reqs["seg_begin"] = np.arange(2 * npairs)
    reqs["seg_count"] = 1
    reqs["dir"][0::2] = 1
    reqs["host_off"] = np.concatenate([[0], np.cumsum(segs["len"])[:-1]])
    whole = torch.empty(len(pool) + 8192, dtype=torch.uint8, device="cuda")
    for rep in range(10):
        stg = W.payload_bytes(240 + rep, int(segs["len"].sum()))
        o_pool, o_stg = pool.copy(), stg.copy()
        o_res = O.copy_batch([O.Guest.from_image(img, o_pool)], reqs, segs, o_stg)
        view = whole[512:512 + len(pool)]
        view.copy_(torch.from_numpy(pool))
        g = cvd.Guest.from_image(img, view)
        stg_d = torch.from_numpy(stg.copy()).cuda()
        res_d = torch.zeros(len(reqs) * 24, dtype=torch.uint8, device="cuda")
        cvd.copy_batch([g], cvd.records_to_device(reqs), len(reqs), cvd.records_to_device(segs), len(segs), stg_d,
                       res_d)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(cvd.records_from_device(res_d, W.RESULT_DTYPE, len(reqs)), o_res)
        assert np.array_equal(stg_d.cpu().numpy(), o_stg), rep
        assert np.array_equal(view.cpu().numpy(), o_pool), rep
        assert cvd.last_levels() > 1
        g.close()


def test_batches_refuse_pools_aliased_off_a_4k_multiple():
    """Two guests of one call whose pools overlap must start a multiple of
    4 KiB apart (the same guest twice is fine): a guest page is keyed by the
    device frame it starts in, which other aliasing would not match."""
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(64 << 20, 241, np_frac=0, ro_frac=0)
    pool = W.materialize_pool(img)
    whole = torch.zeros(len(pool) + 3 * 4096, dtype=torch.uint8, device="cuda")
    stg = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    views = {off: whole[off:off + len(pool)] for off in (0, 512, 8192)}
    gs = {off: cvd.Guest.from_image(img, v) for off, v in views.items()}
    try:
        for pair, ok in (((0, 512), False), ((512, 8192), False), ((0, 8192), True), ((0, 0), True)):
            g = [gs[pair[0]], gs[pair[1]]]
            if ok:
                cvd.copy_batch(g, None, 0, None, 0, stg, None)
            else:
                with pytest.raises(cvd.CvdError) as e:
                    cvd.copy_batch(g, None, 0, None, 0, stg, None)
                assert e.value.status == cvd.EINVAL
        torch.cuda.synchronize()
    finally:
        for g in gs.values():
            g.close()
