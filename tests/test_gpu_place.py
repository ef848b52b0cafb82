"""GPU parity for driver-initiated maps (Sec. 6.6: the backend picks the
guest virtual range, then installs): chosen ranges, per-page statuses, the
page tables, the p2m and the allocator state against the oracle, on hand-built
holes, generated guests (x86-64 and PAE, malformed requests, ENOSPC, the
ENOMEM latch), a window with more free extents than the shared-memory tree
holds, and an EPT guest."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W

pytestmark = pytest.mark.gpu
PAGE = 4096
NONE = O.NO_FRAME


def _place_both(pool, og_kw, lo, hi, reqs, hf):
    import torch
    from paper_1304_3771_b300 import cvd
    o_pool = pool.copy()
    og = O.Guest(o_pool, **og_kw)
    o_gva, o_st = og.mmap_place(lo, hi, reqs, hf)
    pool_d = torch.from_numpy(pool.copy()).cuda()
    kw = dict(og_kw)
    p2m = torch.full((max(kw.get("rsv_n", 0), 1),), -1, dtype=torch.int64, device="cuda")
    dg = cvd.Guest(pool_d, kw.pop("slots"), kw.pop("cr3_gpa"), p2m=p2m, **kw)
    npg = int(reqs["npages"].astype(np.int64).sum())
    st = torch.zeros(max(npg, 1), dtype=torch.int32, device="cuda")
    gva = torch.zeros(max(len(reqs), 1), dtype=torch.int64, device="cuda")
    dg.mmap_place(lo, hi, cvd.records_to_device(reqs), len(reqs), cvd.u64_to_device(hf), len(hf), gva, st)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cvd.u64_from_device(gva)[:len(reqs)], o_gva)
    np.testing.assert_array_equal(st.cpu().numpy()[:npg], o_st)
    assert np.array_equal(pool_d.cpu().numpy(), o_pool), "page tables differ"
    rn = og_kw.get("rsv_n", 0)
    np.testing.assert_array_equal(cvd.u64_from_device(p2m)[:rn], og.p2m[:rn])
    assert dg.alloc_state() == (og.pt_used, og.rsv_used)
    dg.close()
    return o_gva, o_st


def _empty(F=8192, pt_n=4096, rsv_n=1 << 16):
    cr3, tables, low = W.build_tables(F - 1, (np.zeros(0, np.int64), np.zeros(0, np.uint64)))
    pool = np.zeros(F * PAGE, dtype=np.uint8)
    for gfn, t in tables.items():
        pool[gfn * PAGE:(gfn + 1) * PAGE] = t.view(np.uint8)
    kw = dict(slots=np.array([(0, F, 0)], dtype=W.SLOT_DTYPE), cr3_gpa=cr3, pt_pool_gfn=16, pt_pool_n=pt_n,
              rsv_gfn=F + 100, rsv_n=rsv_n)
    return pool, kw


def _reqs(npages, flags=W.PTE_RW | W.PTE_US):
    r = np.zeros(len(npages), dtype=W.PLACE_DTYPE)
    r["npages"] = npages
    r["flags"] = flags
    r["hf_begin"] = np.concatenate([[0], np.cumsum(npages)[:-1]])
    return r


def test_place_empty_and_hand_holes():
    pool, kw = _empty()
    lo = 5 << 30
    n = np.array([3, 1, 512, 7, 600, 2])
    gva, st = _place_both(pool, kw, lo, lo + (64 << 20), _reqs(n), np.arange(int(n.sum()), dtype=np.uint64) + 100)
    assert gva.tolist() == (lo + np.concatenate([[0], np.cumsum(n)[:-1]]) * PAGE).tolist()
    # holes: present leaves at 2, 3, 7 and 10..511 of the unit at 1 GiB (installed by the oracle)
    og = O.Guest(pool, **kw)
    present = [2, 3, 7] + list(range(10, 512))
    m = np.zeros(len(present), dtype=W.MAPREQ_DTYPE)
    m["gva"] = (1 << 30) + np.array(present) * PAGE
    m["npages"], m["flags"], m["hf_begin"] = 1, 6, np.arange(len(present))
    assert (og.mmap_install(m, np.arange(len(present), dtype=np.uint64) + 1) == 0).all()
    kw2 = dict(kw, pt_pool_gfn=16 + og.pt_used, pt_pool_n=4096 - og.pt_used, rsv_gfn=kw["rsv_gfn"] + og.rsv_used,
               rsv_n=kw["rsv_n"] - og.rsv_used)
    gva, st = _place_both(pool, kw2, 1 << 30, (1 << 30) + (2 << 20), _reqs(np.array([2, 3, 1, 2, 1, 1])),
                          np.arange(10, dtype=np.uint64) + 40)
    b = 1 << 30
    assert gva.tolist() == [b, b + 4 * PAGE, b + 8 * PAGE, NONE, b + 9 * PAGE, NONE]


def test_place_bad_window_rejected():
    import torch
    from paper_1304_3771_b300 import cvd
    pool, kw = _empty()
    kw = dict(kw)
    g = cvd.Guest(torch.from_numpy(pool).cuda(), kw.pop("slots"), kw.pop("cr3_gpa"), **kw)
    reqs = cvd.records_to_device(_reqs(np.array([1])))
    hf = cvd.u64_to_device(np.array([5], dtype=np.uint64))
    gva = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    lo = 1 << 30
    for w in ((lo + 1, lo + PAGE), (lo, lo), (lo + PAGE, lo), (lo, (1 << 47) + PAGE)):
        assert cvd.lib().cvd_mmap_place(g.handle, w[0], w[1], cvd._ptr(reqs), 1, cvd._ptr(hf), 1, cvd._ptr(gva),
                                        cvd._ptr(st), None) == cvd.EINVAL
    g.close()


@pytest.mark.parametrize("paging", ["x86_64", "pae"])
def test_place_generated(paging):
    img = W.make_guest(64 << 20, 452, paging=paging, np_frac=0.05, ro_frac=0.02, huge_frac=0.2, pt_pool_n=512,
                       rsv_n=1 << 15)
    pool = W.materialize_pool(img, fill=False)
    kw = dict(slots=img.slots, cr3_gpa=img.cr3_gpa, pt_pool_gfn=img.pt_pool_gfn, pt_pool_n=img.pt_pool_n,
              rsv_gfn=img.rsv_gfn, rsv_n=img.rsv_n, paging=img.paging)
    lo = img.data_gva + img.data_pages * PAGE - (8 << 20)
    reqs, hf = W.place_requests(img, 452, 400, max_pages=24, bad_flag_frac=0.02)
    gva, st = _place_both(pool, kw, lo, lo + (16 << 20), reqs, hf)
    assert (gva != NONE).sum() > 150 and (st == -28).any() and (st == -22).any() and (st == 0).any()


def test_place_enomem_latch():
    pool, kw = _empty(pt_n=3, rsv_n=5)
    lo = 1 << 30
    gva, st = _place_both(pool, kw, lo, lo + 8 * PAGE, _reqs(np.array([4, 3, 2, 1])),
                          np.arange(10, dtype=np.uint64) + 1)
    assert st.tolist() == [0, 0, 0, 0, 0, -12, -12, -28, -28, -12]


@pytest.mark.parametrize("arena_mib", [256, 384, 1024])
def test_place_many_extents(arena_mib):
    """Half the 4 KiB leaves not present: single free runs by the thousand --
    ~15K and ~22K (the 64-ary tree with a middle level in shared memory) and
    ~57K (the 32-ary tree through L2)."""
    img = W.make_guest(arena_mib << 20, 453, np_frac=0.5, ro_frac=0.0, huge_frac=0.0, pt_pool_n=256, rsv_n=1 << 16)
    pool = W.materialize_pool(img, fill=False)
    kw = dict(slots=img.slots, cr3_gpa=img.cr3_gpa, pt_pool_gfn=img.pt_pool_gfn, pt_pool_n=img.pt_pool_n,
              rsv_gfn=img.rsv_gfn, rsv_n=img.rsv_n)
    lo = img.data_gva
    hi = lo + img.data_pages * PAGE
    reqs, hf = W.place_requests(img, 453, 3000, max_pages=3)
    gva, st = _place_both(pool, kw, lo, hi, reqs, hf)
    assert (gva != NONE).all() and (st == 0).all()


def test_place_ept_guest_einval():
    import torch
    from paper_1304_3771_b300 import cvd
    img0 = W.make_guest(64 << 20, 454, host_base=2 << 20)
    img = W.add_ept(img0, 454)
    pool = W.materialize_pool(img)
    g = cvd.Guest.from_image(img, torch.from_numpy(pool.copy()).cuda())
    reqs = _reqs(np.array([2, 1]))
    gva = torch.zeros(2, dtype=torch.int64, device="cuda")
    st = torch.zeros(3, dtype=torch.int32, device="cuda")
    g.mmap_place(1 << 40, (1 << 40) + (1 << 30), cvd.records_to_device(reqs), 2,
                 cvd.u64_to_device(np.arange(3, dtype=np.uint64)), 3, gva, st)
    torch.cuda.synchronize()
    assert cvd.u64_from_device(gva).tolist() == [NONE, NONE] and st.cpu().tolist() == [-22, -22, -22]
    g.close()


def test_place_edges_of_the_space():
    """Windows ending at the top of the user range (2^47; 2^32 for PAE), a
    window with no free page (every request ENOSPC), and no requests."""
    import torch
    from paper_1304_3771_b300 import cvd
    pool, kw = _empty()
    top = 1 << 47
    _place_both(pool, kw, top - (4 << 20), top, _reqs(np.array([1, 512, 600, 3])),
                np.arange(1116, dtype=np.uint64) + 9)
    # PAE: a fresh 4-entry PDPT; the last 8 MiB below 4 GiB
    ppool = np.zeros(0x800000, dtype=np.uint8)
    pkw = dict(slots=np.array([(0, 0x800, 0)], dtype=W.SLOT_DTYPE), cr3_gpa=0x1000, pt_pool_gfn=16, pt_pool_n=64,
               rsv_gfn=0x1000, rsv_n=4096, paging=1)
    gva, st = _place_both(ppool, pkw, (1 << 32) - (8 << 20), 1 << 32, _reqs(np.array([1, 1024, 2])),
                          np.arange(1027, dtype=np.uint64) + 5)
    assert (st == 0).all()
    # a window whose pages are all taken: the first 2 MiB of the identity-mapped hand guest
    hpool, hkw = _empty()
    og = O.Guest(hpool, **hkw)
    m = np.zeros(1, dtype=W.MAPREQ_DTYPE)
    m[0] = (1 << 30, 512, 6, 0)
    assert (og.mmap_install(m, np.arange(512, dtype=np.uint64) + 1) == 0).all()
    hkw2 = dict(hkw, pt_pool_gfn=16 + og.pt_used, pt_pool_n=4096 - og.pt_used, rsv_gfn=hkw["rsv_gfn"] + og.rsv_used,
                rsv_n=hkw["rsv_n"] - og.rsv_used)
    gva, st = _place_both(hpool, hkw2, 1 << 30, (1 << 30) + (2 << 20), _reqs(np.array([1, 2])),
                          np.arange(3, dtype=np.uint64))
    assert (st == -28).all() and (gva == NONE).all()
    # no requests
    kw3 = dict(kw)
    g = cvd.Guest(torch.from_numpy(pool.copy()).cuda(), kw3.pop("slots"), kw3.pop("cr3_gpa"), **kw3)
    z = torch.zeros(8, dtype=torch.int64, device="cuda")
    g.mmap_place(1 << 30, 2 << 30, z, 0, z, 0, z, z)
    torch.cuda.synchronize()
    g.close()
