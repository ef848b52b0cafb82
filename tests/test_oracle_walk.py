"""Pins of the oracle's page walk and memslot step (paper Sec. 4.2: software
walk gVA->gPA, then KVM's gPA->host map) against values fixed outside the
oracle: hand-encoded tables, closed forms and the generator's own record of
the mapping it built."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W
from tests.oracle_fixtures import ALL_ONES, golden_pool, identity_guest, parse_golden


def test_hand_encoded_tables():
    g = parse_golden("walk_hand.txt")
    pool, slots = golden_pool(g)
    og = O.Guest(pool, slots, g["cr3"])
    assert len(g["cases"]) >= 20
    for va, write, code, gpa, hpa in g["cases"]:
        got = og.walk(va, bool(write))
        assert got == (code, gpa, hpa), (hex(va), write, got)


def test_walk_is_read_only():
    g = parse_golden("walk_hand.txt")
    pool, slots = golden_pool(g)
    before = pool.copy()
    og = O.Guest(pool, slots, g["cr3"])
    for va, write, *_ in g["cases"]:
        og.walk(va, bool(write))
    assert np.array_equal(before, pool)


def test_identity_map_closed_form():
    base = 5 << 30
    pool, slots, cr3 = identity_guest(1024, base_gva=base, host_off=0x7000)
    og = O.Guest(pool, slots, cr3)
    rng = np.random.default_rng(1)
    va = base + rng.integers(0, 1024 * 4096, 5000).astype(np.uint64)
    gpa, hpa, code = og.translate(va)
    assert (code == 0).all()
    assert np.array_equal(gpa, va - np.uint64(base))
    assert np.array_equal(hpa, va - np.uint64(base) + np.uint64(0x7000))


def test_permutation_brute_force_every_page():
    img = W.make_guest(64 << 20, 11)
    pool = W.materialize_pool(img, fill=False)
    og = O.Guest.from_image(img, pool)
    vpages = np.arange(img.data_pages)
    offs = np.random.default_rng(2).integers(0, 4096, img.data_pages)
    va = (img.data_gva + vpages * 4096 + offs).astype(np.uint64)
    for write in (False, True):
        gpa, hpa, code = og.translate(va, write)
        fl = img.page_flags
        present = (fl & np.uint64(W.PTE_P)) != 0
        writable = (fl & np.uint64(W.PTE_RW)) != 0
        exp_code = np.where(~present, 0x101, np.where(write & ~writable, 2, 0))
        assert np.array_equal(code, exp_code.astype(np.uint32))
        ok = exp_code == 0
        exp_gpa = img.page_gfn * 4096 + offs
        assert np.array_equal(gpa[ok], exp_gpa[ok].astype(np.uint64))
        assert np.array_equal(hpa[ok], (exp_gpa[ok] + int(img.slots[0]["host_off"])).astype(np.uint64))
        assert (gpa[~ok] == np.uint64(ALL_ONES)).all()


def test_huge_leaf_is_512_consecutive_frames():
    img = W.make_guest(256 << 20, 12, huge_frac=0.5, np_frac=0, ro_frac=0, nslots=3)
    pool = W.materialize_pool(img, fill=False)
    og = O.Guest.from_image(img, pool)
    units = np.nonzero(img.huge_gfn >= 0)[0]
    assert len(units) > 10
    for u in units[:40]:
        va = (img.data_gva + u * (2 << 20) + np.arange(512) * 4096 + 17).astype(np.uint64)
        gpa, hpa, code = og.translate(va)
        assert (code == 0).all()
        exp = img.huge_gfn[u] * 4096 + np.arange(512) * 4096 + 17
        assert np.array_equal(gpa, exp.astype(np.uint64))
        # memslot closed form: host = host_off + gpa - base_gfn*4096 of the containing slot
        for a, h in zip(exp[::64], hpa[::64]):
            gfn = a >> 12
            s = [s for s in img.slots if s["base_gfn"] <= gfn < s["base_gfn"] + s["npages"]][0]
            assert int(h) == int(s["host_off"]) + int(a) - int(s["base_gfn"]) * 4096


def test_multi_slot_and_missing_slot():
    # 4 KiB identity map over 64 frames; slots cover gfn 0..31 and 40..63 at
    # different host offsets; gfn 32..39 has no slot.
    base = 1 << 30
    F = 512
    vpn = (base >> 12) + np.arange(64)
    leaves = (vpn, (np.arange(64, dtype=np.uint64) << np.uint64(12)) | np.uint64(7))
    cr3, tables, low = W.build_tables(F - 1, leaves)
    slots = np.array([(0, 32, 0x100000), (40, F - 40, 0x2000)], dtype=W.SLOT_DTYPE)
    pool = np.zeros(0x200000, dtype=np.uint8)
    for gfn, t in tables.items():
        h = 0x2000 + (gfn - 40) * 4096
        pool[h:h + 4096] = t.view(np.uint8)
    og = O.Guest(pool, slots, cr3)
    for i in range(64):
        code, gpa, hpa = og.walk(base + i * 4096 + 5)
        if i < 32:
            assert (code, gpa, hpa) == (0, i * 4096 + 5, 0x100000 + i * 4096 + 5)
        elif i < 40:
            assert code == 5 and gpa == ALL_ONES
        else:
            assert (code, gpa, hpa) == (0, i * 4096 + 5, 0x2000 + (i - 40) * 4096 + 5)


def test_reserved_window_goes_through_p2m():
    g = parse_golden("walk_hand.txt")
    pool, slots = golden_pool(g)
    # map VA 0x7000 (PT[7]) to reserved gfn 0x1000 + 2
    h = 0x3000 + 12 * 4096 + 7 * 8
    pool[h:h + 8] = np.frombuffer(((0x1002 << 12) | 7).to_bytes(8, "little"), np.uint8)
    p2m = np.full(4, ALL_ONES, dtype=np.uint64)
    og = O.Guest(pool, slots, g["cr3"], rsv_gfn=0x1000, rsv_n=4, p2m=p2m)
    assert og.walk(0x7ABC)[0] == 5          # unmapped reserved frame
    p2m[2] = 0x11
    assert og.walk(0x7ABC) == (0, 0x1002ABC, 0x11ABC)
    p2m[2] = pool.nbytes // 4096           # host frame outside the pool
    assert og.walk(0x7ABC)[0] == 5


@pytest.mark.parametrize("va,code", [(0x0000800000000000, 3), (0x8000000000000000, 3),
                                     (0xFFFF800000000000, 4), (0xFFFFFFFFFFFFFFFF, 4)])
def test_canonical_and_user_half(va, code):
    g = parse_golden("walk_hand.txt")
    pool, slots = golden_pool(g)
    og = O.Guest(pool, slots, g["cr3"])
    assert og.walk(va)[0] == code


def test_1gib_leaf_offsets_reach_a_backed_frame():
    """The hand tables' 1 GiB leaf (PDPT entry 2 -> gPA 0x40000000, P|RW|US|PS)
    with a second memslot over guest frames 0x40200-0x4020F at host offset
    0x14000: the leaf keeps va bits 29:0, so an offset past 2 MiB inside the
    leaf reaches that slot (hand-derived from the SDM Vol. 3 ch. 4 format)."""
    g = parse_golden("walk_hand.txt")
    pool, slots = golden_pool(g)
    pool = np.concatenate([pool, np.zeros(16 * 4096, np.uint8)])
    slots = np.concatenate([slots, np.array([(0x40200, 16, 0x14000)], dtype=W.SLOT_DTYPE)])
    og = O.Guest(pool, slots, g["cr3"])
    assert og.walk(0x80200010) == (0, 0x40200010, 0x14010)
    assert og.walk(0x8020F123, True) == (0, 0x4020F123, 0x23123)
    assert og.walk(0x80210000)[0] == 0x005          # past the slot: NOSLOT
    assert og.walk(0x80000005)[0] == 0x005          # below it: NOSLOT
