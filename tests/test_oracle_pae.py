"""The oracle's 32-bit PAE guests (the paging mode of the paper's own
implementation, Sec. 6.2), pinned without the oracle's own formulas: hand-
encoded tables with hand-derived results, the generator's record of every
page, gathers that must equal the recorded pages byte for byte, per-byte =
per-page, and mmap installs whose resulting entries are written out by hand
or follow from counting distinct 1 GiB / 2 MiB prefixes."""
import numpy as np

import oracle as O
from paper_1304_3771_b300 import workload as W
from tests.oracle_fixtures import ALL_ONES, golden_pool, parse_golden

PAGE = 4096


def test_pae_walk_hand_tables():
    g = parse_golden("walk_pae_hand.txt")
    assert g["paging"] == 1
    pool, slots = golden_pool(g)
    og = O.Guest(pool, slots, g["cr3"], paging=1)
    for va, write, code, gpa, hpa in g["cases"]:
        assert og.walk(va, bool(write)) == (code, gpa, hpa), hex(va)


def _pae_guest(seed, **kw):
    args = dict(np_frac=0.05, ro_frac=0.05, huge_frac=0.3)
    args.update(kw)
    img = W.make_guest(64 << 20, seed, paging="pae", **args)
    return img, W.materialize_pool(img)


def test_pae_walk_matches_generator_record():
    img, pool = _pae_guest(301)
    og = O.Guest.from_image(img, pool)
    assert img.paging == 1 and img.data_gva + img.data_pages * PAGE <= 3 << 30
    for p in range(img.data_pages):
        va = img.data_gva + p * PAGE + (p * 37) % PAGE
        g = int(img.page_gfn[p])
        if g < 0:   # inside a 2 MiB leaf
            gpa = (int(img.huge_gfn[p // 512]) << 12) + (va - img.data_gva) % (2 << 20)
            assert og.walk(va, True)[:2] == (0, gpa)
            continue
        fl = int(img.page_flags[p])
        gpa = (g << 12) + va % PAGE
        if not fl & W.PTE_P:
            assert og.walk(va)[0] == 0x101
        elif not fl & W.PTE_RW:
            assert og.walk(va)[:2] == (0, gpa) and og.walk(va, True)[0] == 2
        else:
            assert og.walk(va, True)[:2] == (0, gpa)
    assert og.walk(img.data_gva - PAGE)[0] in (0x101, 0x201, 0x301)
    assert og.walk(1 << 32)[0] == 4


def test_pae_gather_equals_recorded_pages():
    img, pool = _pae_guest(302, np_frac=0.0, ro_frac=0.0)
    og = O.Guest.from_image(img, pool)
    n = min(img.data_pages, 2048)
    segs = np.array([(img.data_gva + k * 64 * PAGE, 64 * PAGE) for k in range(n // 64)], dtype=W.SEG_DTYPE)
    reqs = np.zeros(1, dtype=W.REQ_DTYPE)
    reqs[0] = (0, len(segs), 0, 0, 0)
    stg = np.zeros(n * PAGE, dtype=np.uint8)
    res = O.copy_batch([og], reqs, segs, stg)
    assert res["fault_code"][0] == 0 and res["done"][0] == n * PAGE
    for p in range(n):
        g = int(img.page_gfn[p])
        if g < 0:
            g = int(img.huge_gfn[p // 512]) + p % 512
        h = img.gpa_to_host(g << 12)
        assert np.array_equal(stg[p * PAGE:(p + 1) * PAGE], pool[h:h + PAGE]), p


def test_pae_per_byte_equals_per_page_and_range():
    img, pool = _pae_guest(303)
    wl = W.tiny_requests(img, 303, nreq=120, hi=20000)
    reqs, segs = wl.reqs.copy(), wl.segs.copy()
    # one segment crossing 2^32 and one starting beyond it
    segs[0] = ((1 << 32) - 100, 200)
    segs[-1] = ((1 << 32) + 8, 16)
    stg = W.payload_bytes(304, wl.staging_bytes)
    out = []
    for per_byte in (False, True):
        p, s = pool.copy(), stg.copy()
        out.append((O.copy_batch([O.Guest.from_image(img, p)], reqs, segs, s, per_byte=per_byte), p, s))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
    r0 = out[0][0][0]
    assert r0["fault_code"] == 4 and r0["done"] == 0 and r0["fault_gva"] == (1 << 32) - 100
    codes = out[0][0]["fault_code"]
    assert (codes == 0x101).any() and (codes == 0).any()


def _empty_pae(pool_bytes=0x40000, ram_frames=0x40):
    """PAE guest whose PDPT (gfn 1) is empty; PT pool gfn 16..31; reserved
    window gfn 0x100..0x107."""
    pool = np.zeros(pool_bytes, dtype=np.uint8)
    slots = np.array([(0, ram_frames, 0)], dtype=W.SLOT_DTYPE)
    og = O.Guest(pool, slots, 0x1000, pt_pool_gfn=16, pt_pool_n=16, rsv_gfn=0x100, rsv_n=8, paging=1)
    return og, pool


def _entry(pool, gfn, idx):
    return int.from_bytes(pool[gfn * PAGE + idx * 8:gfn * PAGE + idx * 8 + 8].tobytes(), "little")


def test_pae_mmap_hand_install():
    og, pool = _empty_pae()
    reqs = np.zeros(2, dtype=W.MAPREQ_DTYPE)
    reqs[0] = (0x40000000, 1, W.PTE_RW | W.PTE_US, 0)      # quarter 1, PDE 0, PTE 0
    reqs[1] = (0x40201000, 1, W.PTE_US, 1)                 # quarter 1, PDE 1, PTE 1
    hf = np.array([0x21, 0x22], dtype=np.uint64)
    st = og.mmap_install(reqs, hf)
    assert list(st) == [0, 0]
    # hand-derived: PD = gfn 16 (linked from PDPTE 1 with P only), PTs = gfn 17, 18
    assert _entry(pool, 1, 1) == (16 << 12) | 0x1
    assert _entry(pool, 16, 0) == (17 << 12) | 0x7
    assert _entry(pool, 17, 0) == (0x100 << 12) | 0x7
    assert _entry(pool, 16, 1) == (18 << 12) | 0x7
    assert _entry(pool, 18, 1) == (0x101 << 12) | 0x5
    assert (og.pt_used, og.rsv_used) == (3, 2)
    assert list(og.p2m[:2]) == [0x21, 0x22]
    # translate after install: reserved frame, then the p2m host frame
    assert og.walk(0x40000123, True) == (0, (0x100 << 12) | 0x123, (0x21 << 12) | 0x123)
    assert og.walk(0x40201010, True)[0] == 2
    # re-install -> EBUSY, nothing allocated
    assert list(og.mmap_install(reqs[:1], hf[:1])) == [-16]
    assert (og.pt_used, og.rsv_used) == (3, 2)


def test_pae_mmap_reserved_pdpte_and_range():
    og, pool = _empty_pae()
    pool[1 * PAGE + 2 * 8] = 0x87 & 0xFF        # PDPTE 2: P | RW | PS (reserved bits)
    pool[1 * PAGE + 2 * 8 + 1] = 0x50           # frame 0x5000
    reqs = np.zeros(3, dtype=W.MAPREQ_DTYPE)
    reqs[0] = (0x80000000, 1, W.PTE_RW | W.PTE_US, 0)      # under the reserved PDPTE -> EBUSY
    reqs[1] = ((1 << 32) - PAGE, 2, W.PTE_US, 1)          # runs past 2^32 -> EINVAL
    reqs[2] = ((1 << 32) - PAGE, 1, W.PTE_US, 3)          # last page of the space -> ok
    hf = np.array([0x21, 0x22, 0x23, 0x24], dtype=np.uint64)
    st = og.mmap_install(reqs, hf)
    assert list(st) == [-16, -22, -22, 0]
    assert og.walk((1 << 32) - 1)[0] == 0


def test_pae_mmap_table_count_closed_form():
    og, pool = _empty_pae(pool_bytes=0x800000, ram_frames=0x800)
    og = O.Guest(pool, og.slots, 0x1000, pt_pool_gfn=16, pt_pool_n=600, rsv_gfn=0x1000, rsv_n=4096, paging=1)
    rng = np.random.default_rng(305)
    pages = np.unique(rng.integers(0x100, (1 << 32) // PAGE, 300))
    reqs = np.zeros(len(pages), dtype=W.MAPREQ_DTYPE)
    reqs["gva"] = pages * PAGE
    reqs["npages"] = 1
    reqs["flags"] = W.PTE_RW | W.PTE_US
    reqs["hf_begin"] = np.arange(len(pages))
    hf = np.arange(len(pages), dtype=np.uint64) + 0x40
    assert (og.mmap_install(reqs, hf) == 0).all()
    # one page directory per distinct 1 GiB quarter, one page table per distinct 2 MiB unit
    assert og.pt_used == len(np.unique(pages >> 18)) + len(np.unique(pages >> 9))
    assert og.rsv_used == len(pages)


def test_pae_space_has_no_noncanonical_addresses():
    """A 32-bit PAE space is [0, 2^32): an address a 4-level guest would call
    non-canonical is simply past its end there -> RANGE, for copies as for
    walks (SDM Vol. 3 sec. 4.4: 32-bit linear addresses)."""
    img, pool = _pae_guest(305)
    og = O.Guest.from_image(img, pool.copy())
    reqs = np.zeros(1, dtype=W.REQ_DTYPE)
    reqs[0] = (0, 1, 0, 0, 0)
    for gva in (1 << 47, 0xFFFF_0000_0000_0000, (1 << 63) | 5):
        segs = np.array([(gva, 16)], dtype=W.SEG_DTYPE)
        res = O.copy_batch([og], reqs, segs, np.zeros(16, np.uint8))
        assert (res["fault_code"][0], res["fault_gva"][0], res["done"][0]) == (4, gva, 0)
        assert og.walk(gva)[0] == 4


def test_pae_pdpt_need_not_start_a_page():
    """cr3 of a PAE guest is 32-byte aligned, not page aligned (SDM Vol. 3
    sec. 4.4.1): the hand tables' PDPT moved to offset 0x60 inside its frame,
    with cr3 moved with it, gives every hand-derived walk unchanged; the four
    entries at the frame's start are cleared, so a walk that read there would
    find nothing present."""
    g = parse_golden("walk_pae_hand.txt")
    pool, slots = golden_pool(g)
    base = 0x3000 + 15 * 4096                        # gfn 15 in the single memslot
    pdpt = pool[base:base + 32].copy()
    pool[base:base + 32] = 0
    pool[base + 0x60:base + 0x80] = pdpt
    og = O.Guest(pool, slots, g["cr3"] + 0x60, paging=1)
    for va, write, code, gpa, hpa in g["cases"]:
        assert og.walk(va, bool(write)) == (code, gpa, hpa), hex(va)
