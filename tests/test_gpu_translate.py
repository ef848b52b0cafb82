"""GPU parity of cvd_translate (Sec. 4.2 walk + memslot step) against the
oracle, bit-exact: gPA, hPA and fault code for every address."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W
from tests.gpu_helpers import assert_same, device_guest, run_both
from tests.oracle_fixtures import golden_pool, parse_golden

pytestmark = pytest.mark.gpu


def _gpu_translate(g, gva, write):
    import torch
    from paper_1304_3771_b300 import cvd
    out = g.translate(cvd.u64_to_device(gva), write)
    torch.cuda.synchronize()
    return (cvd.u64_from_device(out[0]), cvd.u64_from_device(out[1]),
            out[2].cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("n", [1, 255, 257, 100_003])
def test_translate_tiny_shape(n):
    img = W.make_guest(64 << 20, 101)
    pool = W.materialize_pool(img, fill=False)
    gva = W.translate_gvas(img, 101, n)
    og = O.Guest.from_image(img, pool)
    g, _ = device_guest(img, pool)
    for write in (False, True):
        exp = og.translate(gva, write)
        got = _gpu_translate(g, gva, write)
        for e, o in zip(exp, got):
            np.testing.assert_array_equal(o, e)
    g.close()


def test_translate_huge_multislot():
    img = W.make_guest(512 << 20, 102, huge_frac=0.7, np_frac=0.02, ro_frac=0.02, nslots=4, slot_gap_pages=64)
    pool = W.materialize_pool(img, fill=False)
    rng = np.random.default_rng(5)
    gva = np.concatenate([W.translate_gvas(img, 102, 50_000),
                          (img.data_gva + rng.integers(0, img.data_pages * 4096, 50_000)).astype(np.uint64)])
    og = O.Guest.from_image(img, pool)
    g, _ = device_guest(img, pool)
    exp = og.translate(gva)
    got = _gpu_translate(g, gva, False)
    for e, o in zip(exp, got):
        np.testing.assert_array_equal(o, e)
    assert (exp[2] == 0).sum() > 40_000
    g.close()


@pytest.mark.parametrize("paging", ["x86_64", "pae"])
def test_translate_slots_off_2mib_boundaries(paging):
    """The same memory map split into slots at 4 KiB points (no 2 MiB unit
    tables then: lookups search the slots) gives the oracle's results and the
    unsplit guest's (unit tables), for every address, 4-level and PAE."""
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(512 << 20, 104, huge_frac=0.5, np_frac=0.02, ro_frac=0.02, nslots=3, slot_gap_pages=64,
                       paging=paging)
    pool = W.materialize_pool(img, fill=False)
    parts = []
    for s in img.slots:
        cut = int(s["npages"]) // 2 + 3            # odd page count: off every 2 MiB boundary
        parts.append((int(s["base_gfn"]), cut, int(s["host_off"])))
        parts.append((int(s["base_gfn"]) + cut, int(s["npages"]) - cut, int(s["host_off"]) + cut * 4096))
    split = np.array(parts, dtype=W.SLOT_DTYPE)
    gva = W.translate_gvas(img, 104, 200_003)
    pool_d = torch.from_numpy(pool).cuda()
    a = cvd.Guest.from_image(img, pool_d)
    b = cvd.Guest(pool_d, split, img.cr3_gpa, pt_pool_gfn=img.pt_pool_gfn, pt_pool_n=img.pt_pool_n,
                  rsv_gfn=img.rsv_gfn, rsv_n=img.rsv_n, paging=img.paging)
    og = O.Guest.from_image(img, pool)
    for write in (False, True):
        exp = og.translate(gva, write)
        ga, gb = _gpu_translate(a, gva, write), _gpu_translate(b, gva, write)
        for e, x, y in zip(exp, ga, gb):
            np.testing.assert_array_equal(x, e)
            np.testing.assert_array_equal(y, e)
        assert (exp[2] == 0).sum() > 60_000 and (exp[2] != 0).sum() > 60_000
    a.close()
    b.close()


@pytest.mark.parametrize("split", [False, True])
def test_translate_and_copy_at_the_memslot_limit(split):
    """64 memslots (CVD_MAX_SLOTS): on 2 MiB boundaries (unit tables), or 32
    slots each split at an odd 4 KiB point (slot search over 64) -- every
    translation and a levelled copy batch against the oracle."""
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(512 << 20, 470, huge_frac=0.5, np_frac=0.02, ro_frac=0.02,
                       nslots=32 if split else 64, slot_gap_pages=512)
    if split:
        parts = []
        for s in img.slots:
            cut = int(s["npages"]) // 2 + 1
            parts.append((int(s["base_gfn"]), cut, int(s["host_off"])))
            parts.append((int(s["base_gfn"]) + cut, int(s["npages"]) - cut, int(s["host_off"]) + cut * 4096))
        img.slots = np.array(parts, dtype=W.SLOT_DTYPE)
    assert len(img.slots) == 64
    pool = W.materialize_pool(img)
    g, pool_d = device_guest(img, pool)
    gva = W.translate_gvas(img, 470, 100_003)
    og = O.Guest.from_image(img, pool)
    for write in (False, True):
        exp = og.translate(gva, write)
        got = _gpu_translate(g, gva, write)
        for e, o in zip(exp, got):
            np.testing.assert_array_equal(o, e)
    g.close()
    wl = W.tiny_requests(img, 471, nreq=500, hi=60000, frame_frac=0.05)
    out = run_both(img, pool, wl.reqs, wl.segs, W.payload_bytes(472, wl.staging_bytes))
    assert_same(out)
    assert (out["o_res"]["fault_code"] == 0).any() and (out["o_res"]["fault_code"] != 0).any()


def test_translate_hand_tables_and_p2m():
    import torch
    from paper_1304_3771_b300 import cvd
    gd = parse_golden("walk_hand.txt")
    pool, slots = golden_pool(gd)
    # map VA 0x7000 to reserved gfn 0x1002 whose p2m entry is host frame 0x11
    h = 0x3000 + 12 * 4096 + 7 * 8
    pool[h:h + 8] = np.frombuffer(((0x1002 << 12) | 7).to_bytes(8, "little"), np.uint8)
    p2m = np.full(4, (1 << 64) - 1, dtype=np.uint64)
    p2m[2] = 0x11
    og = O.Guest(pool, slots, gd["cr3"], rsv_gfn=0x1000, rsv_n=4, p2m=p2m.copy())
    pool_d = torch.from_numpy(pool.copy()).cuda()
    g = cvd.Guest(pool_d, slots, gd["cr3"], rsv_gfn=0x1000, rsv_n=4, p2m=cvd.u64_to_device(p2m))
    gva = np.array([c[0] for c in gd["cases"]] + [0x7ABC, 0x7000], dtype=np.uint64)
    for write in (False, True):
        exp = og.translate(gva, write)
        got = _gpu_translate(g, gva, write)
        for e, o in zip(exp, got):
            np.testing.assert_array_equal(o, e)
    # and against the hand-written expectations directly
    code = _gpu_translate(g, gva[:len(gd["cases"])], False)[2]
    for c, (va, write, exp_code, *_r) in zip(code, gd["cases"]):
        if not write:
            assert c == exp_code
    g.close()


def test_translate_1gib_leaf_into_a_second_memslot():
    """The hand tables' 1 GiB leaf with a second memslot over guest frames
    0x40200-0x4020F: walks inside the leaf past 2 MiB reach it (the oracle's
    hand-derived pin), on the GPU as on the oracle."""
    import torch
    from paper_1304_3771_b300 import cvd
    gd = parse_golden("walk_hand.txt")
    pool, slots = golden_pool(gd)
    pool = np.concatenate([pool, np.zeros(16 * 4096, np.uint8)])
    slots = np.concatenate([slots, np.array([(0x40200, 16, 0x14000)], dtype=W.SLOT_DTYPE)])
    og = O.Guest(pool, slots, gd["cr3"])
    g = cvd.Guest(torch.from_numpy(pool.copy()).cuda(), slots, gd["cr3"])
    gva = np.array([0x80200010, 0x8020F123, 0x80210000, 0x80000005, 0x80200FFF], dtype=np.uint64)
    for write in (False, True):
        for e, o in zip(og.translate(gva, write), _gpu_translate(g, gva, write)):
            np.testing.assert_array_equal(o, e)
    assert _gpu_translate(g, gva[:1], False)[1][0] == 0x14010
    g.close()


def test_translate_empty():
    import torch
    img = W.make_guest(64 << 20, 103)
    pool = W.materialize_pool(img, fill=False)
    g, _ = device_guest(img, pool)
    g.translate(torch.zeros(0, dtype=torch.int64, device="cuda"))
    torch.cuda.synchronize()
    g.close()


def test_latency_probe_and_translate_shape():
    """The pointer chase orders an L2-resident chain below a DRAM-sized one, and
    the translate launch shape is the one the kernel runs."""
    import torch
    from paper_1304_3771_b300 import cvd
    small = torch.empty(8 << 20, dtype=torch.uint8, device="cuda")
    big = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    t_l2 = cvd.probe_latency(small, steps=50_000)
    t_dram = cvd.probe_latency(big, steps=50_000)
    assert 20.0 < t_l2 < t_dram < 5000.0, (t_l2, t_dram)
    threads, walks = cvd.translate_shape()
    assert threads % 256 == 0 and 256 <= threads <= 2048 and walks >= 1
    img = W.make_guest(64 << 20, 101)                 # one 2 MiB aligned slot: unit tables
    g, _ = device_guest(img, W.materialize_pool(img, fill=False))
    tu, wu = cvd.translate_shape(g)
    assert tu % 256 == 0 and 256 <= tu <= 2048 and wu >= 1   # the staged kernel keeps its own count
    g.close()
    with pytest.raises(cvd.CvdError):
        cvd.probe_latency(small[1:], steps=10)        # not 128-byte aligned


def test_translate_after_installs_spread_over_many_tables():
    """Maps installed under three far top-level entries and several 1 GiB
    regions each: walks reach second-level tables and page directories that
    the staged translation did not copy, and leaves in the reserved window
    (p2m).  Every output equals the oracle's after the same installs."""
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(64 << 20, 107, np_frac=0.05, ro_frac=0.05, pt_pool_n=512, rsv_n=8192)
    pool = W.materialize_pool(img, fill=False)
    assert img.data_gva >> 39 < 64
    rng = np.random.default_rng(7)
    reqs = []
    for i4 in (100, 101, 250):
        for i3 in (0, 1, 2, 3, 5, 9):
            base = (i4 << 39) | (i3 << 30) | (int(rng.integers(0, 500)) << 21)
            reqs.append((base, int(rng.integers(1, 40)), int(W.PTE_RW | W.PTE_US) if i3 % 2 else int(W.PTE_US)))
    mreq = np.zeros(len(reqs), dtype=W.MAPREQ_DTYPE)
    mreq["gva"] = [r[0] for r in reqs]
    mreq["npages"] = [r[1] for r in reqs]
    mreq["flags"] = [r[2] for r in reqs]
    mreq["hf_begin"] = np.concatenate([[0], np.cumsum(mreq["npages"].astype(np.int64))[:-1]])
    npg = int(mreq["npages"].astype(np.int64).sum())
    hf = rng.integers(0, img.pool_bytes // 4096, npg).astype(np.uint64)
    og = O.Guest.from_image(img, pool.copy())
    assert (og.mmap_install(mreq, hf) == 0).all()
    g, pool_d = device_guest(img, pool)
    st = torch.zeros(npg, dtype=torch.int32, device="cuda")
    g.mmap_install(cvd.records_to_device(mreq), len(mreq), cvd.u64_to_device(hf), len(hf), st)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    pages = np.concatenate([m["gva"] + 4096 * np.arange(m["npages"] + 2, dtype=np.uint64) for m in mreq])
    gva = np.concatenate([pages + rng.integers(0, 4096, len(pages)).astype(np.uint64),
                          W.translate_gvas(img, 107, 20_000)]).astype(np.uint64)
    for write in (False, True):
        exp = og.translate(gva, write)
        got = _gpu_translate(g, gva, write)
        for e, o in zip(exp, got):
            np.testing.assert_array_equal(o, e)
    assert (exp[2] == 0).sum() > 500 and (exp[2] == 0x101).sum() > 20
    g.close()


def test_translate_16gib_guest_beyond_the_staged_directories():
    """The 16 GiB batching guest (70% 2 MiB leaves, 4 memslots) has more page
    directories than the staged translation copies: walks under the others
    read their directory entry from the pool.  Every output of 2 M addresses
    equals the oracle's."""
    import torch
    img = W.make_guest(16 << 30, 109, huge_frac=0.7, np_frac=0.02, ro_frac=0.02, nslots=4, slot_gap_pages=512)
    pool_d = torch.zeros(img.pool_bytes, dtype=torch.uint8, device="cuda")
    offs, data = W.table_blob(img)
    idx = torch.from_numpy((offs[:, None] + np.arange(4096)[None, :]).reshape(-1)).cuda()
    pool_d[idx] = torch.from_numpy(data.reshape(-1)).cuda()
    del idx
    from paper_1304_3771_b300 import cvd
    g = cvd.Guest.from_image(img, pool_d)
    shadow = np.zeros(img.pool_bytes, dtype=np.uint8)     # lazily backed: the tables only
    W.write_tables(img, shadow)
    og = O.Guest.from_image(img, shadow)
    gva = W.translate_gvas(img, 109, 2_000_000)
    for write in (False, True):
        exp = og.translate(gva, write)
        got = _gpu_translate(g, gva, write)
        for e, o in zip(exp, got):
            np.testing.assert_array_equal(o, e)
    assert (exp[2] == 0).sum() > 900_000
    g.close()
    del pool_d
    torch.cuda.empty_cache()
