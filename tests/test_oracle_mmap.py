"""Pins of the oracle's mmap PTE install (paper Sec. 4.2 second category of
routines; insert_pfn, Sec. 6.2; PT pages from the frontend's pool and
reserved guest frames, Sec. 4.2)."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W
from tests.oracle_fixtures import ALL_ONES, golden_maps, golden_pool, parse_golden, read_entries


def _golden_guest():
    g = parse_golden("mmap_hand.txt")
    pool, slots = golden_pool(g)
    rg, rn = g["rsv"]
    og = O.Guest(pool, slots, g["cr3"], pt_pool_gfn=g["ptpool"][0], pt_pool_n=g["ptpool"][1],
                 rsv_gfn=rg, rsv_n=rn)
    return g, pool, og


def test_hand_computed_install():
    g, pool, og = _golden_guest()
    # dirty the PT-pool frames: the install must zero them
    pool[0x3000 + 8 * 4096:0x3000 + 12 * 4096] = 0xCD
    reqs, hf = golden_maps(g)
    st = og.mmap_install(reqs, hf)
    assert st.tolist() == g["status"]
    got = read_entries(pool, lambda gfn: 0x3000 + gfn * 4096, [8, 9, 10, 11, 15])
    exp = {(gfn, idx): e for gfn, idx, e in g["expect"]}
    assert got == exp
    for i, frame in g["p2m"]:
        assert int(og.p2m[i]) == frame
    assert int(og.p2m[3]) == ALL_ONES
    assert (og.pt_used, og.rsv_used) == g["used"]


def test_translate_after_install_returns_reserved_frames():
    g, pool, og = _golden_guest()
    reqs, hf = golden_maps(g)
    og.mmap_install(reqs, hf)
    assert og.walk(0x40201ABC) == (0, 0x1000ABC, 0x21ABC)
    assert og.walk(0x40202000, True) == (0, 0x1001000, 0x22000)
    # US-only leaf: readable, write-protected
    assert og.walk(0x40400010) == (0, 0x1002010, 0x23010)
    assert og.walk(0x40400010, True)[0] == 2
    assert og.walk(0x80000000)[0] == 0x301        # ENOMEM page left nothing behind


def _empty_guest(pt_n=4096, rsv_n=1 << 16, F=8192):
    cr3, tables, low = W.build_tables(F - 1, (np.zeros(0, np.int64), np.zeros(0, np.uint64)))
    assert list(tables) == [F - 1]
    slots = np.array([(0, F, 0)], dtype=W.SLOT_DTYPE)
    pool = np.zeros(F * 4096, dtype=np.uint8)
    return pool, O.Guest(pool, slots, cr3, pt_pool_gfn=16, pt_pool_n=pt_n, rsv_gfn=F + 100, rsv_n=rsv_n)


def test_table_count_closed_form():
    rng = np.random.default_rng(5)
    pool, og = _empty_guest()
    n = 200
    gva = (rng.integers(0, 1 << 23, n) << 12) + (rng.integers(0, 4, n) << 39)
    npg = rng.integers(1, 40, n)
    reqs = np.zeros(n, dtype=W.MAPREQ_DTYPE)
    reqs["gva"], reqs["npages"], reqs["flags"] = gva, npg, 6
    reqs["hf_begin"] = np.concatenate([[0], np.cumsum(npg)[:-1]])
    hf = rng.integers(0, pool.nbytes // 4096, int(npg.sum())).astype(np.uint64)
    st = og.mmap_install(reqs, hf)
    va = np.concatenate([g + np.arange(k) * 4096 for g, k in zip(gva, npg)])
    # closed form: one PDPT per distinct 512 GiB prefix, one PD per distinct
    # 1 GiB prefix, one PT per distinct 2 MiB prefix; one reserved frame per
    # distinct page (later duplicates are EBUSY).
    exp_tables = len(np.unique(va >> 39)) + len(np.unique(va >> 30)) + len(np.unique(va >> 21))
    assert og.pt_used == exp_tables
    assert og.rsv_used == len(np.unique(va))
    first = np.zeros(len(va), bool)
    first[np.unique(va, return_index=True)[1]] = True
    assert np.array_equal(st == 0, first)
    assert (st[~first] == -16).all()


def test_reinstall_is_ebusy_and_huge_leaf_blocks():
    img = W.make_guest(256 << 20, 31, huge_frac=0.5, np_frac=0, ro_frac=0, rsv_n=64)
    pool = W.materialize_pool(img, fill=False)
    og = O.Guest.from_image(img, pool)
    hu = int(np.nonzero(img.huge_gfn >= 0)[0][0])
    sm = int(np.nonzero(img.huge_gfn < 0)[0][0])
    reqs = np.zeros(2, dtype=W.MAPREQ_DTYPE)
    reqs[0] = (img.data_gva + hu * (2 << 20) + 8 * 4096, 2, 6, 0)   # inside a 2 MiB leaf
    reqs[1] = (img.data_gva + sm * (2 << 20) + 8 * 4096, 2, 6, 2)   # present 4 KiB leaves
    before = pool.copy()
    st = og.mmap_install(reqs, np.arange(4, dtype=np.uint64))
    assert st.tolist() == [-16, -16, -16, -16]
    assert np.array_equal(before, pool)
    assert og.pt_used == 0 and og.rsv_used == 0


def test_enomem_latch_and_einval():
    pool, og = _empty_guest(pt_n=3, rsv_n=3)
    reqs = np.zeros(5, dtype=W.MAPREQ_DTYPE)
    reqs[0] = (1 << 30, 2, 6, 0)          # 3 tables + 2 frames
    reqs[1] = ((1 << 30) + 0x123, 1, 6, 2)  # misaligned -> EINVAL
    reqs[2] = (2 << 30, 1, 6, 3)          # needs 2 tables: pool empty -> ENOMEM, latch
    reqs[3] = ((1 << 30) + 2 * 4096, 1, 6, 4)   # would fit (0 tables, 1 frame) but latched
    reqs[4] = ((1 << 30) + 3 * 4096, 1, 0x40, 5)  # D bit not allowed -> EINVAL
    st = og.mmap_install(reqs, np.arange(6, dtype=np.uint64) + 1)
    assert st.tolist() == [0, 0, -22, -12, -12, -22]
    assert (og.pt_used, og.rsv_used) == (3, 2)
    # host frame outside the pool -> EINVAL for that page only
    pool2, og2 = _empty_guest()
    r = np.array([(1 << 30, 2, 6, 0)], dtype=W.MAPREQ_DTYPE)
    st2 = og2.mmap_install(r, np.array([pool2.nbytes // 4096, 5], dtype=np.uint64))
    assert st2.tolist() == [-22, 0]


def test_nx_and_flag_bits():
    pool, og = _empty_guest()
    r = np.array([(1 << 30, 1, W.MAP_NX | W.PTE_RW | W.PTE_US | W.PTE_G | W.PTE_PCD, 0)],
                 dtype=W.MAPREQ_DTYPE)
    assert og.mmap_install(r, np.array([9], dtype=np.uint64)).tolist() == [0]
    # the PT created for the page is the third pool frame (16 + 2)
    t = pool[18 * 4096:19 * 4096].view(np.uint64)
    rsv = og.s.rsv_gfn
    assert int(t[0]) == (1 << 63) | (rsv << 12) | 0x1 | 0x2 | 0x4 | 0x10 | 0x100


@pytest.mark.parametrize("pool_frames,expect", [(2, -12), (3, 0)])
def test_pt_pool_must_hold_every_missing_table(pool_frames, expect):
    """A page under an empty PML4 slot needs three new tables (PDPT, PD, PT):
    a PT pool of two frames gives ENOMEM and takes nothing; three frames
    install it and use all three (Sec. 4.2: tables come from the frontend's
    pool; the closed form of the table count per missing level)."""
    img = W.make_guest(16 << 20, 531, np_frac=0.0, ro_frac=0.0, pt_pool_n=pool_frames)
    og = O.Guest.from_image(img, W.materialize_pool(img))
    va = next(k << 39 for k in range(1, 256) if og.walk(k << 39)[0] == 0x401)
    before = og.pool.copy()
    reqs = np.zeros(1, dtype=W.MAPREQ_DTYPE)
    reqs[0] = (va, 1, 0x7, 0)
    st = og.mmap_install(reqs, np.array([5], dtype=np.uint64))
    assert st.tolist() == [expect]
    if expect == 0:
        assert (og.pt_used, og.rsv_used) == (3, 1)
        assert og.walk(va)[:2] == (0, img.rsv_gfn * 4096)
    else:
        assert (og.pt_used, og.rsv_used) == (0, 0)
        assert np.array_equal(og.pool, before)


def test_reserved_window_holds_exactly_its_frames():
    """Three pages under an empty PML4 slot with a reserved window of two
    frames: the first two install (the first creating three tables), the
    third finds the window used up -> ENOMEM (Sec. 4.2: each mapped page takes
    a guest frame reserved through the hypervisor; the window's size bounds
    them)."""
    img = W.make_guest(16 << 20, 533, np_frac=0.0, ro_frac=0.0, pt_pool_n=8, rsv_n=2)
    og = O.Guest.from_image(img, W.materialize_pool(img))
    va = next(k << 39 for k in range(1, 256) if og.walk(k << 39)[0] == 0x401)
    reqs = np.zeros(1, dtype=W.MAPREQ_DTYPE)
    reqs[0] = (va, 3, 0x7, 0)
    st = og.mmap_install(reqs, np.array([5, 6, 7], dtype=np.uint64))
    assert st.tolist() == [0, 0, -12]
    assert (og.pt_used, og.rsv_used) == (3, 2)
    assert og.walk(va + 4096)[:2] == (0, (img.rsv_gfn + 1) * 4096)
    assert og.walk(va + 8192)[0] == 0x101


def test_host_frame_range_must_lie_inside_the_array():
    """A request whose host-frame range [hf_begin, hf_begin + npages) runs past
    the given array by one entry is malformed: EINVAL for each of its pages,
    nothing installed (the install's contract: every page names a host frame)."""
    img = W.make_guest(16 << 20, 535, np_frac=0.0, ro_frac=0.0)
    og = O.Guest.from_image(img, W.materialize_pool(img))
    va = next(k << 39 for k in range(1, 256) if og.walk(k << 39)[0] == 0x401)
    reqs = np.zeros(2, dtype=W.MAPREQ_DTYPE)
    reqs[0] = (va, 2, 0x7, 2)            # frames 2, 3 of a 3-frame array: one past its end
    reqs[1] = (va + (4 << 20), 2, 0x7, 1)   # frames 1, 2: inside
    st = og.mmap_install(reqs, np.array([5, 6, 7], dtype=np.uint64))
    assert st.tolist() == [-22, -22, 0, 0]
    assert og.walk(va)[0] != 0 and og.rsv_used == 2
