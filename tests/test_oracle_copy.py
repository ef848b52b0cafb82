"""Pins of the oracle's gather/scatter (paper Sec. 4.2: copy_from_user /
copy_to_user on a guest buffer, translated once per page) against closed
forms, brute force and invariants."""
import numpy as np

import oracle as O
from paper_1304_3771_b300 import workload as W
from tests.oracle_fixtures import golden_pool, identity_guest, parse_golden


def _reqs(specs):
    """specs: list of (dir, host_off, [(gva, len), ...])"""
    segs, reqs = [], []
    for d, host, ss in specs:
        reqs.append((len(segs), len(ss), d, 0, host))
        segs.extend(ss)
    return np.array(reqs, dtype=W.REQ_DTYPE), np.array(segs, dtype=W.SEG_DTYPE)


def test_identity_map_reduces_to_memcpy():
    base = 3 << 30
    pool, slots, cr3 = identity_guest(256, base_gva=base, host_off=0x9000)
    og = O.Guest(pool, slots, cr3)
    rng = np.random.default_rng(3)
    specs, host = [], 0
    for _ in range(50):
        off = int(rng.integers(0, 200 * 4096))
        ln = int(rng.integers(1, 40000))
        specs.append((0, host, [(base + off, ln)]))
        host += ln
    reqs, segs = _reqs(specs)
    stg = np.zeros(host, np.uint8)
    res = O.copy_batch([og], reqs, segs, stg)
    assert (res["fault_code"] == 0).all()
    for (d, h, [(gva, ln)]), r in zip(specs, res):
        src = 0x9000 + gva - base
        assert r["done"] == ln
        assert np.array_equal(stg[h:h + ln], pool[src:src + ln])


def test_permutation_reduces_to_page_gather():
    img = W.make_guest(64 << 20, 21, np_frac=0, ro_frac=0)
    pool = W.materialize_pool(img)
    og = O.Guest.from_image(img, pool)
    host0 = int(img.slots[0]["host_off"])
    rng = np.random.default_rng(4)
    specs, host = [], 0
    for _ in range(30):
        p = int(rng.integers(0, img.data_pages - 40))
        off = int(rng.integers(0, 4096))
        ln = int(rng.integers(1, 30 * 4096))
        specs.append((0, host, [(img.data_gva + p * 4096 + off, ln)]))
        host += ln
    reqs, segs = _reqs(specs)
    stg = np.zeros(host, np.uint8)
    res = O.copy_batch([og], reqs, segs, stg)
    assert (res["done"] == reqs_len(segs, reqs)).all()
    # expected: byte i of the buffer comes from frame page_gfn[vpage] (generator's permutation)
    for (d, h, [(gva, ln)]) in specs:
        v = gva - img.data_gva + np.arange(ln)
        exp = pool[host0 + img.page_gfn[v // 4096] * 4096 + v % 4096]
        assert np.array_equal(stg[h:h + ln], exp)


def reqs_len(segs, reqs):
    return np.array([segs["len"][r["seg_begin"]:r["seg_begin"] + r["seg_count"]].sum() for r in reqs],
                    dtype=np.uint64)


def test_round_trip_and_canaries():
    img = W.make_guest(64 << 20, 22, np_frac=0, ro_frac=0)
    pool = W.materialize_pool(img)
    og = O.Guest.from_image(img, pool)
    # disjoint multi-segment requests (hazard-free batch) on a fault-free guest
    sizes = W.batching_sizes(5, 300)
    sizes = np.minimum(sizes, 200000)
    wl = W.batched_requests(img, 5, sizes, 8)
    lo, hi = wl.batches[0]
    reqs = wl.reqs[lo:hi].copy()
    reqs["dir"] = 1
    src = np.random.default_rng(6).integers(0, 256, wl.staging_bytes, dtype=np.uint8)
    before = pool.copy()
    res = O.copy_batch([og], reqs, wl.segs, src.copy())
    assert (res["fault_code"] == 0).all()
    # canaries: only bytes inside the target pages' ranges may change
    touched = np.zeros(pool.size, bool)
    host0 = int(img.slots[0]["host_off"])
    for r in reqs:
        for s in wl.segs[r["seg_begin"]:r["seg_begin"] + r["seg_count"]]:
            v = int(s["gva"]) - img.data_gva + np.arange(int(s["len"]))
            touched[host0 + img.page_gfn[v // 4096] * 4096 + v % 4096] = True
    assert np.array_equal(pool[~touched], before[~touched])
    reqs["dir"] = 0
    back = np.zeros(wl.staging_bytes, np.uint8)
    res2 = O.copy_batch([og], reqs, wl.segs, back)
    assert (res2["fault_code"] == 0).all()
    for r in reqs:
        L = int(wl.segs["len"][r["seg_begin"]:r["seg_begin"] + r["seg_count"]].sum())
        h = int(r["host_off"])
        assert np.array_equal(back[h:h + L], src[h:h + L])


def test_fault_offsets_and_prefix_semantics():
    g = parse_golden("walk_hand.txt")
    pool, slots = golden_pool(g)
    # random payload in the data frames gfn 0..9 (tables live in gfn 10..15)
    pool[0x3000:0x3000 + 10 * 4096] = np.random.default_rng(9).integers(0, 256, 10 * 4096, dtype=np.uint8)
    og = O.Guest(pool, slots, g["cr3"])
    # VA 0x0000-0x1FFF present (page 1 read-only), 0x2000 not present.
    specs = [
        (0, 0, [(0x0F00, 0x200), (0x1F00, 0x200)]),          # from: fault at 0x2000 -> done 0x300
        (1, 0x1000, [(0x0800, 0x100), (0x1000, 0x10)]),      # to: RO page at stream 0x100
        (0, 0x2000, [(0x0010, 0), (0x5000, 0x10)]),          # zero-length segment is a no-op
        (0, 0x3000, [(0x0000, 0x10), (0x0000800000000000, 4)]),  # NONCANONICAL at segment start
        (0, 0x4000, [(0x7FFFFFFFFFF0, 0x20)]),               # RANGE (crosses 2^47) at 0
        (0, 0x5000, [(0x6FF0, 0x20)]),                       # 0x7000 not present (PT[7]=0)
    ]
    reqs, segs = _reqs(specs)
    stg = np.full(0x6000, 0xEE, np.uint8)
    pool_before = pool.copy()
    res = O.copy_batch([og], reqs, segs, stg)
    exp = [(0x300, 0x2000, 0x101), (0x100, 0x1000, 2), (0x10, 0, 0), (0x10, 0x0000800000000000, 3),
           (0, 0x7FFFFFFFFFF0, 4), (0x10, 0x7000, 0x101)]
    got = [(int(r["done"]), int(r["fault_gva"]), int(r["fault_code"])) for r in res]
    assert got == exp
    host = lambda gpa: 0x3000 + gpa  # noqa: E731  (single slot at 0x3000)
    # request 0: VA 0x0F00..0x0FFF -> gpa 0x5F00.., VA 0x1000..0x10FF -> gpa 0x7000..,
    # VA 0x1F00..0x1FFF -> gpa 0x7F00..; VA 0x2000 faults; then zero-fill
    assert np.array_equal(stg[0:0x100], pool[host(0x5F00):host(0x6000)])
    assert np.array_equal(stg[0x100:0x200], pool[host(0x7000):host(0x7100)])
    assert np.array_equal(stg[0x200:0x300], pool[host(0x7F00):host(0x8000)])
    assert (stg[0x300:0x400] == 0).all()
    assert (stg[0x400:0x1000] == 0xEE).all()
    # request 1: 0x100 bytes written at gpa 0x5800, nothing at the RO page
    assert np.array_equal(pool[host(0x5800):host(0x5900)], stg[0x1000:0x1100])
    assert np.array_equal(pool[host(0x7000):host(0x7010)], pool_before[host(0x7000):host(0x7010)])
    # request 4: nothing copied, whole staging range zero-filled
    assert (stg[0x4000:0x4020] == 0).all()
    # request 5: 0x10 bytes copied (0x6FF0 -> gpa 0x4FF0), rest zero
    assert np.array_equal(stg[0x5000:0x5010], pool[host(0x4FF0):host(0x5000)])
    assert (stg[0x5010:0x5020] == 0).all()
    assert (stg[0x5020:0x5030] == 0xEE).all()


def test_per_byte_equals_per_page():
    img = W.make_guest(64 << 20, 23)
    pool = W.materialize_pool(img)
    wl = W.tiny_requests(img, 23, nreq=60, hi=12000)
    a_pool, b_pool = pool.copy(), pool.copy()
    a_stg = np.random.default_rng(1).integers(0, 256, wl.staging_bytes, dtype=np.uint8)
    b_stg = a_stg.copy()
    ra = O.copy_batch([O.Guest.from_image(img, a_pool)], wl.reqs, wl.segs, a_stg, per_byte=False)
    rb = O.copy_batch([O.Guest.from_image(img, b_pool)], wl.reqs, wl.segs, b_stg, per_byte=True)
    assert np.array_equal(ra, rb)
    assert np.array_equal(a_pool, b_pool)
    assert np.array_equal(a_stg, b_stg)
    assert (ra["fault_code"] != 0).any() and (ra["fault_code"] == 0).any()


def test_sequential_semantics_in_one_call():
    base = 2 << 30
    pool, slots, cr3 = identity_guest(16, base_gva=base, host_off=0x1000)
    og = O.Guest(pool, slots, cr3)
    stg = np.zeros(0x400, np.uint8)
    stg[0:0x100] = 1
    stg[0x100:0x200] = 2
    # write 1s at [0x10, 0x110), then 2s at [0x80, 0x180), then read [0, 0x200)
    specs = [(1, 0, [(base + 0x10, 0x100)]), (1, 0x100, [(base + 0x80, 0x100)]),
             (0, 0x200, [(base, 0x200)])]
    reqs, segs = _reqs(specs)
    before = pool[0x1000:0x1200].copy()
    res = O.copy_batch([og], reqs, segs, stg)
    assert (res["fault_code"] == 0).all()
    exp = before.copy()
    exp[0x10:0x110] = 1
    exp[0x80:0x180] = 2
    assert np.array_equal(pool[0x1000:0x1200], exp)
    assert np.array_equal(stg[0x200:0x400], exp)


def test_malformed_requests():
    base = 2 << 30
    pool, slots, cr3 = identity_guest(16, base_gva=base, host_off=0x1000)
    og = O.Guest(pool, slots, cr3)
    segs = np.array([(base, 16), (base + 32, 16), (base + 64, 16)], dtype=W.SEG_DTYPE)
    reqs = np.array([
        (0, 1, 2, 0, 0),        # dir 2 -> BADREQ
        (0, 1, 0, 1, 0),        # guest 1 of 1 -> BADREQ
        (2, 2, 0, 0, 0),        # segments 2..3 of 3 -> BADREQ
        (0, 1, 0, 0, 90),       # staging 90..106 of 100 -> HOSTBUF
        (0, 2, 0, 0, 0),        # ok (running total 2)
        (1, 2, 0, 0, 40),       # running total 4 > 3 -> BADREQ (capacity)
        (2, 1, 0, 0, 60),       # running total 5 (request 5 still counts) -> BADREQ
    ], dtype=W.REQ_DTYPE)
    stg = np.full(100, 0xAA, np.uint8)
    res = O.copy_batch([og], reqs, segs, stg)
    assert res["fault_code"].tolist() == [9, 9, 9, 8, 0, 9, 9]
    assert res["done"].tolist() == [0, 0, 0, 0, 32, 0, 0]
    assert (stg[32:40] == 0xAA).all() and (stg[76:100] == 0xAA).all()


def test_zero_length_segments_touch_no_address():
    """A zero-length segment copies no byte, so it reaches no address and
    cannot fault, wherever it points (non-canonical, past the user half);
    the request's other segments copy as if it were absent (Sec. 4.2 checks
    are per byte copied)."""
    base = 3 << 30
    pool, slots, cr3 = identity_guest(16, base_gva=base, host_off=0x9000)
    og = O.Guest(pool, slots, cr3)
    reqs, segs = _reqs([(0, 0, [(1 << 63, 0), (base + 0x10, 100), (1 << 47, 0), (base + 0x2000, 50)])])
    stg = np.zeros(150, np.uint8)
    res = O.copy_batch([og], reqs, segs, stg)
    assert (res["fault_code"][0], res["done"][0]) == (0, 150)
    assert np.array_equal(stg[:100], pool[0x9010:0x9010 + 100])
    assert np.array_equal(stg[100:], pool[0x9000 + 0x2000:0x9000 + 0x2000 + 50])
