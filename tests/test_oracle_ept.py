"""The oracle's software EPT (the second dimension without KVM, Sec. 4.2; EPT
format per the Intel SDM Vol. 3 sec. 28.3.2), pinned without the oracle's own
formulas: hand-encoded guest and EPT tables with hand-derived results; an EPT
that maps exactly what the memslots map must give memslot mode's results for
walks and copies; with frames planted unmapped or read-only by the EPT, every
data page's outcome follows from the generator's record; per-byte = per-page;
installs into an EPT guest are refused page by page."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W
from tests.oracle_fixtures import golden_pool, parse_golden

PAGE = 4096


def _hand_guest():
    g = parse_golden("walk_ept_hand.txt")
    pool, slots = golden_pool(g)
    rg, rn = g["rsv"]
    p2m = np.full(rn, O.NO_FRAME, dtype=np.uint64)
    for i, f in g["p2m_set"]:
        p2m[i] = f
    og = O.Guest(pool, slots, g["cr3"], rsv_gfn=rg, rsv_n=rn, p2m=p2m, ept_root=g["ept_root"])
    return g, og


def test_ept_walk_hand_tables():
    g, og = _hand_guest()
    assert len(g["slots"]) == 0          # no memslots: the EPT alone backs guest memory
    for va, write, code, gpa, hpa in g["cases"]:
        assert og.walk(va, bool(write)) == (code, gpa, hpa), (hex(va), write)


def test_ept_hand_tables_batched_translate_agrees():
    g, og = _hand_guest()
    for write in (0, 1):
        cases = [c for c in g["cases"] if c[1] == write]
        va = np.array([c[0] for c in cases], dtype=np.uint64)
        gpa, hpa, code = og.translate(va, bool(write))
        assert list(zip(code.tolist(), gpa.tolist(), hpa.tolist())) == [(c[2], c[3], c[4]) for c in cases]


def _pair(seed, paging="x86_64", **ept):
    img0 = W.make_guest(64 << 20, seed, huge_frac=0.3, np_frac=0.03, ro_frac=0.03, nslots=3,
                        host_base=2 << 20, slot_gap_pages=512, paging=paging)
    img = W.add_ept(img0, seed, **ept)
    pool = W.materialize_pool(img)
    return img0, img, pool


@pytest.mark.parametrize("paging", ["x86_64", "pae"])
def test_ept_equal_to_memslots_walks(paging):
    img0, img, pool = _pair(410 if paging == "x86_64" else 411, paging)
    assert any(int(t[i]) & W.EPT_LARGE for t in img.ept_tables.values() for i in np.nonzero(t)[0])
    a, b = O.Guest.from_image(img0, pool), O.Guest.from_image(img, pool)
    va = W.translate_gvas(img0, 412, 100_000)
    for write in (False, True):
        ra, rb = a.translate(va, write), b.translate(va, write)
        for x, y in zip(ra, rb):
            np.testing.assert_array_equal(x, y)
        assert len(np.unique(ra[2])) >= 3


def test_ept_equal_to_memslots_copies():
    img0, img, pool = _pair(413)
    wl = W.tiny_requests(img0, 413, nreq=200, hi=40000, frame_frac=0.05)
    stg = W.payload_bytes(414, wl.staging_bytes)
    out = []
    for im in (img0, img):
        p, s = pool.copy(), stg.copy()
        out.append((O.copy_batch([O.Guest.from_image(im, p)], wl.reqs, wl.segs, s), p, s))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
    assert (out[0][0]["fault_code"] == 0).any() and (out[0][0]["fault_code"] != 0).any()


def test_ept_faults_follow_generator_record():
    img0 = W.make_guest(64 << 20, 415, huge_frac=0.3, np_frac=0.0, ro_frac=0.0, host_base=2 << 20)
    img = W.add_ept(img0, 415, np_frac=0.05, ro_frac=0.05)
    assert len(img.ept_unmapped) > 100 and len(img.ept_readonly) > 100
    pool = W.materialize_pool(img)
    og = O.Guest.from_image(img, pool)
    unmapped, readonly = set(img.ept_unmapped.tolist()), set(img.ept_readonly.tolist())
    seen = set()
    for p in range(img.data_pages):
        va = img.data_gva + p * PAGE + (p * 41) % PAGE
        g = int(img.page_gfn[p])
        if g < 0:
            g = int(img.huge_gfn[p // 512]) + p % 512
        gpa = (g << 12) + va % PAGE
        h = img.gpa_to_host(gpa)
        if g in unmapped:
            assert og.walk(va) == (5, O.NO_FRAME, O.NO_FRAME) and og.walk(va, True)[0] == 5
            seen.add("unmapped")
        elif g in readonly:
            assert og.walk(va) == (0, gpa, h) and og.walk(va, True)[0] == 10
            seen.add("readonly")
        else:
            assert og.walk(va, True) == (0, gpa, h)
    assert seen == {"unmapped", "readonly"}


def test_ept_copy_faults_per_byte_equals_per_page():
    img0 = W.make_guest(64 << 20, 416, huge_frac=0.3, np_frac=0.01, ro_frac=0.01, nslots=2,
                        host_base=2 << 20)
    img = W.add_ept(img0, 416, np_frac=0.01, ro_frac=0.02)
    pool = W.materialize_pool(img)
    wl = W.tiny_requests(img, 416, nreq=300, hi=60000)
    stg = W.payload_bytes(417, wl.staging_bytes)
    out = []
    for per_byte in (False, True):
        p, s = pool.copy(), stg.copy()
        out.append((O.copy_batch([O.Guest.from_image(img, p)], wl.reqs, wl.segs, s, per_byte=per_byte), p, s))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
    res = out[0][0]
    codes = res["fault_code"]
    assert (codes == 10).any() and (codes == 5).any() and (codes == 0).any()
    # an EPT_VIOLATION only on copy-to (dir 1), at the start of an EPT read-only page
    readonly = set(img.ept_readonly.tolist())
    og = O.Guest.from_image(img, pool)
    for r in np.nonzero(codes == 10)[0]:
        assert wl.reqs["dir"][r] == 1
        va = int(res["fault_gva"][r])
        code, gpa, _ = og.walk(va)
        assert code == 0 and (gpa >> 12) in readonly


def test_ept_hand_copy_prefix():
    """A copy-to across the guest pages at va 0x0 (EPT R|W) and 0x1000 (EPT
    read-only) stops at 0x1000 with EPT_VIOLATION and 4,096 bytes done; the
    same copy-from runs through and reads host frames h12 then h13."""
    g, og = _hand_guest()
    pool = og.pool
    pool[0xC000:0xE000] = np.arange(0x2000, dtype=np.uint32).astype(np.uint8)
    segs = np.array([(0x800, 0x1000), (0x800, 0x1000)], dtype=W.SEG_DTYPE)
    reqs = np.zeros(2, dtype=W.REQ_DTYPE)
    reqs[0] = (0, 1, 0, 0, 0)           # copy_from
    reqs[1] = (1, 1, 1, 0, 0x1000)      # copy_to
    stg = np.full(0x2000, 0xEE, dtype=np.uint8)
    before = pool.copy()
    res = O.copy_batch([og], reqs, segs, stg)
    assert (res["fault_code"][0], res["done"][0]) == (0, 0x1000)
    assert np.array_equal(stg[:0x1000], before[0xC800:0xD800])
    assert (res["fault_code"][1], res["done"][1], res["fault_gva"][1]) == (10, 0x800, 0x1000)
    assert np.array_equal(pool[0xC800:0xD000], stg[0x1000:0x1800])
    assert np.array_equal(pool[0xD000:0xE000], before[0xD000:0xE000])


def test_ept_install_refused_page_by_page():
    img0, img, pool = _pair(418)
    og = O.Guest.from_image(img, pool)
    reqs, hf, _ = W.mmap_requests(img0, 418, 50, window_bytes=64 << 20)
    before = pool.copy()
    st = og.mmap_install(reqs, hf)
    assert len(st) == int(reqs["npages"].astype(np.int64).sum()) and (st == -22).all()
    assert np.array_equal(pool, before) and (og.pt_used, og.rsv_used) == (0, 0)


def test_ept_frame_must_lie_inside_the_pool():
    """With the pool cut 8 bytes short of 0x20000 the host frame 0x1F000 is no
    longer whole inside it: a page there is not backed, even at its first byte;
    the frame below is unaffected."""
    g = parse_golden("walk_ept_hand.txt")
    pool, slots = golden_pool(g)
    rg, rn = g["rsv"]
    p2m = np.full(rn, O.NO_FRAME, dtype=np.uint64)
    og = O.Guest(pool[:0x20000 - 8].copy(), slots, g["cr3"], rsv_gfn=rg, rsv_n=rn, p2m=p2m,
                 ept_root=g["ept_root"])
    assert og.walk(0x21F000)[0] == 5 and og.walk(0x21FFF8)[0] == 5
    assert og.walk(0x21EFF8) == (0, 0x21EFF8, 0x1EFF8)
