"""The oracle's driver-initiated maps (Sec. 6.6: the backend picks the guest
virtual range itself, then installs), pinned without the oracle's own
placement code: closed forms on empty tables, hand-built holes with
hand-derived placements, and a brute-force checker that recomputes free pages
from the walk (a page is free when its walk stops at a non-present entry) and
verifies that every range is free, disjoint from earlier ones and the lowest
that fits (first fit), that ENOSPC is given only when no range fits, and that
the installed pages translate to their host frames."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W

PAGE = 4096
NONE = O.NO_FRAME


def _empty_guest(pt_n=4096, rsv_n=1 << 16, F=8192):
    cr3, tables, low = W.build_tables(F - 1, (np.zeros(0, np.int64), np.zeros(0, np.uint64)))
    slots = np.array([(0, F, 0)], dtype=W.SLOT_DTYPE)
    pool = np.zeros(F * PAGE, dtype=np.uint8)
    return pool, O.Guest(pool, slots, cr3, pt_pool_gfn=16, pt_pool_n=pt_n, rsv_gfn=F + 100, rsv_n=rsv_n)


def _reqs(npages, flags=W.PTE_RW | W.PTE_US):
    r = np.zeros(len(npages), dtype=W.PLACE_DTYPE)
    r["npages"] = npages
    r["flags"] = flags
    r["hf_begin"] = np.concatenate([[0], np.cumsum(npages)[:-1]]) if len(npages) else []
    return r


def test_empty_tables_pack_back_to_back():
    pool, og = _empty_guest()
    n = np.array([3, 1, 512, 7, 600, 2])
    lo = 5 << 30
    reqs = _reqs(n)
    hf = np.arange(int(n.sum()), dtype=np.uint64) + 100
    gva, st = og.mmap_place(lo, lo + (64 << 20), reqs, hf)
    assert gva.tolist() == (lo + np.concatenate([[0], np.cumsum(n)[:-1]]) * PAGE).tolist()
    assert (st == 0).all()
    # closed form: PDPT (new 512 GiB prefix), PD, and one PT per 2 MiB unit touched
    pages = np.arange(int(n.sum()))
    assert og.pt_used == 2 + len(np.unique((lo // PAGE + pages) >> 9))
    for k in (0, 3, 1000, int(n.sum()) - 1):
        code, _, hpa = og.walk(lo + k * PAGE + 5)
        assert code == 0 and hpa == (100 + k) * PAGE + 5


def _hand_holes():
    """Window = the 2 MiB unit at 1 GiB: a PT whose leaves at indexes 2, 3, 7
    and 10..511 are present (taken); free pages 0, 1, 4, 5, 6, 8, 9."""
    pool, og = _empty_guest()
    present = [2, 3, 7] + list(range(10, 512))
    reqs = np.zeros(len(present), dtype=W.MAPREQ_DTYPE)
    reqs["gva"] = (1 << 30) + np.array(present) * PAGE
    reqs["npages"] = 1
    reqs["flags"] = W.PTE_RW | W.PTE_US
    reqs["hf_begin"] = np.arange(len(present))
    assert (og.mmap_install(reqs, np.arange(len(present), dtype=np.uint64) + 1) == 0).all()
    return pool, og


def test_hand_holes_first_fit():
    pool, og = _hand_holes()
    lo, hi = 1 << 30, (1 << 30) + (2 << 20)
    # hand-derived: [2] -> pages 0-1; [3] -> 4-6; [1] -> 8; [2] -> none (9 alone); [1] -> 9; [1] -> none
    reqs = _reqs(np.array([2, 3, 1, 2, 1, 1]))
    hf = np.arange(10, dtype=np.uint64) + 40
    gva, st = og.mmap_place(lo, hi, reqs, hf)
    exp = [lo, lo + 4 * PAGE, lo + 8 * PAGE, NONE, lo + 9 * PAGE, NONE]
    assert gva.tolist() == exp
    assert st.tolist() == [0, 0, 0, 0, 0, 0, -28, -28, 0, -28]
    # the window's second half (pages 256..511) is all taken: a window there has no room
    gva, st = og.mmap_place(lo + 256 * PAGE, hi, _reqs(np.array([1])), hf)
    assert gva.tolist() == [NONE] and st.tolist() == [-28]


def test_malformed_requests_and_bad_window():
    pool, og = _empty_guest()
    lo = 1 << 30
    reqs = _reqs(np.array([0, 2, 3, 1]))
    reqs["flags"][2] |= W.PTE_PS            # PS is not an install flag
    reqs["hf_begin"][3] = 10                # past the 6 frames given
    gva, st = og.mmap_place(lo, lo + (1 << 20), reqs, np.arange(6, dtype=np.uint64) + 3)
    assert gva.tolist() == [NONE, lo, NONE, NONE]
    assert st.tolist() == [0, 0, -22, -22, -22, -22]
    for w in ((lo + 1, lo + PAGE), (lo, lo), (lo + PAGE, lo), (lo, (1 << 47) + PAGE)):
        with pytest.raises(ValueError):
            og.mmap_place(w[0], w[1], reqs, np.arange(6, dtype=np.uint64))


def test_enomem_latch_leaves_enospc_alone():
    pool, og = _empty_guest(pt_n=3, rsv_n=5)
    lo = 1 << 30
    # window of 8 pages: 4 + 3 fit, the 2-page request does not; reserved frames run out at page 6
    reqs = _reqs(np.array([4, 3, 2, 1]))
    gva, st = og.mmap_place(lo, lo + 8 * PAGE, reqs, np.arange(10, dtype=np.uint64) + 1)
    assert gva.tolist() == [lo, lo + 4 * PAGE, NONE, lo + 7 * PAGE]
    assert st.tolist() == [0, 0, 0, 0, 0, -12, -12, -28, -28, -12]


def test_ept_guest_gets_einval():
    img0 = W.make_guest(64 << 20, 450, host_base=2 << 20)
    img = W.add_ept(img0, 450)
    og = O.Guest.from_image(img, W.materialize_pool(img))
    gva, st = og.mmap_place(1 << 40, (1 << 40) + (1 << 30), _reqs(np.array([2, 1])), np.arange(3, dtype=np.uint64))
    assert gva.tolist() == [NONE, NONE] and st.tolist() == [-22, -22, -22]


def _free_at_start(og, lo, hi):
    va = np.arange(lo, hi, PAGE, dtype=np.uint64)
    code = og.translate(va)[2]
    return (code & 0xFF) == 1          # the walk stops at a non-present entry


def _check_first_fit(free0, lo, reqs, gva, nhf):
    """Brute-force check of step 2 against the free-page map at call start."""
    avail = free0.copy()
    for r, q in enumerate(reqs):
        n = int(q["npages"])
        malformed = n == 0 or (int(q["flags"]) & ~(0x11F | (1 << 31))) or int(q["hf_begin"]) + n > nhf
        fits = [a for a in range(len(avail) - n + 1) if n and avail[a:a + n].all()]
        if malformed:
            assert gva[r] == NONE
            continue
        if not fits:
            assert gva[r] == NONE, r
            continue
        a = (int(gva[r]) - lo) // PAGE
        assert a == fits[0], (r, a, fits[:3])
        avail[a:a + n] = False


@pytest.mark.parametrize("paging", ["x86_64", "pae"])
def test_generated_guest_first_fit_and_translation(paging):
    img = W.make_guest(64 << 20, 451, paging=paging, np_frac=0.05, ro_frac=0.02, huge_frac=0.2,
                       pt_pool_n=512, rsv_n=1 << 15)
    pool = W.materialize_pool(img, fill=False)
    og = O.Guest.from_image(img, pool)
    # window: the last 8 MiB of the data region (holes where leaves are not
    # present; 2 MiB leaves taken) and 8 MiB of unmapped space after it
    lo = img.data_gva + img.data_pages * PAGE - (8 << 20)
    hi = lo + (16 << 20)
    free0 = _free_at_start(og, lo, hi)
    assert 0.01 < free0[:2048].mean() < 0.5 and free0[2048:].all()
    reqs, hf = W.place_requests(img, 451, 300, max_pages=24, bad_flag_frac=0.02)
    gva, st = og.mmap_place(lo, hi, reqs, hf)
    _check_first_fit(free0, lo, reqs, gva, len(hf))
    assert (gva != NONE).sum() > 150 and (st == -22).any() and (st == -28).any()
    # holes were filled by small requests
    placed = gva[gva != NONE]
    assert (placed < lo + (8 << 20)).any() and (placed >= lo + (8 << 20)).any()
    # every installed page translates to its host frame
    off = np.concatenate([[0], np.cumsum(reqs["npages"].astype(np.int64))[:-1]])
    for r in np.nonzero(gva != NONE)[0][::7]:
        for k in range(int(reqs["npages"][r])):
            if st[off[r] + k] == 0:
                code, _, hpa = og.walk(int(gva[r]) + k * PAGE + 9)
                assert code == 0 and hpa == int(hf[int(reqs["hf_begin"][r]) + k]) * PAGE + 9


def test_zero_page_request_gets_no_range_in_a_fragmented_window():
    """A request for zero pages is malformed: no range, even where the window
    starts with taken pages (a zero-length run 'fits' anywhere), and it takes
    nothing from the requests after it (Sec. 6.6: the backend picks a range
    for a map of some pages)."""
    pool, og = _hand_holes()
    lo, hi = (1 << 30) + 2 * PAGE, (1 << 30) + (2 << 20)     # the window starts at taken page 2
    gva, st = og.mmap_place(lo, hi, _reqs(np.array([0, 2])), np.arange(4, dtype=np.uint64) + 40)
    assert gva.tolist() == [NONE, (1 << 30) + 4 * PAGE]
    assert st.tolist() == [0, 0]
