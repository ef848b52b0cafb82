"""GPU parity for 32-bit PAE guests (the paging mode of the paper's own
implementation, Sec. 6.2): translation, copies through the levelled and the
hazard-free paths (long segments included) and mmap installs, compared with
the oracle element by element; the hand-encoded tables also against their
hand-derived results."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W
from tests.gpu_helpers import assert_same, run_both
from tests.oracle_fixtures import golden_pool, parse_golden

pytestmark = pytest.mark.gpu


def _pae_guest(seed, arena=64 << 20, **kw):
    args = dict(np_frac=0.03, ro_frac=0.03, huge_frac=0.3)
    args.update(kw)
    img = W.make_guest(arena, seed, paging="pae", **args)
    return img, W.materialize_pool(img)


@pytest.mark.parametrize("pdpt_off", [0, 0x60])
def test_pae_hand_tables_translate(pdpt_off):
    """The hand tables, with the PDPT also at offset 0x60 inside its frame
    (cr3 is 32-byte aligned, not page aligned)."""
    import torch
    from paper_1304_3771_b300 import cvd
    gd = parse_golden("walk_pae_hand.txt")
    pool, slots = golden_pool(gd)
    if pdpt_off:
        base = 0x3000 + 15 * 4096
        pdpt = pool[base:base + 32].copy()
        pool[base:base + 32] = 0
        pool[base + pdpt_off:base + pdpt_off + 32] = pdpt
    cr3 = gd["cr3"] + pdpt_off
    g = cvd.Guest(torch.from_numpy(pool).cuda(), slots, cr3, paging=1)
    og = O.Guest(pool, slots, cr3, paging=1)
    for write in (0, 1):
        cases = [c for c in gd["cases"] if c[1] == write]
        va = np.array([c[0] for c in cases], dtype=np.uint64)
        gpa, hpa, code = g.translate(cvd.u64_to_device(va), write=bool(write))
        torch.cuda.synchronize()
        got = list(zip(code.cpu().numpy().view(np.uint32).tolist(), cvd.u64_from_device(gpa).tolist(),
                       cvd.u64_from_device(hpa).tolist()))
        assert got == [(c[2], c[3], c[4]) for c in cases]
        o = og.translate(va, bool(write))
        assert got == list(zip(o[2].tolist(), o[0].tolist(), o[1].tolist()))
    g.close()


@pytest.mark.parametrize("write", [False, True])
def test_pae_translate_generated(write):
    import torch
    from paper_1304_3771_b300 import cvd
    img, pool = _pae_guest(320)
    g = cvd.Guest.from_image(img, torch.from_numpy(pool).cuda())
    va = W.translate_gvas(img, 320, 100_003)
    gpa, hpa, code = g.translate(cvd.u64_to_device(va), write=write)
    torch.cuda.synchronize()
    exp = O.Guest.from_image(img, pool).translate(va, write)
    np.testing.assert_array_equal(cvd.u64_from_device(gpa), exp[0])
    np.testing.assert_array_equal(cvd.u64_from_device(hpa), exp[1])
    np.testing.assert_array_equal(code.cpu().numpy().view(np.uint32), exp[2])
    assert len(np.unique(exp[2])) >= 4
    g.close()


def test_pae_levelled_copies_with_range_faults():
    img, pool = _pae_guest(321)
    wl = W.tiny_requests(img, 321, nreq=300, hi=30000, frame_frac=0.05)
    segs = wl.segs.copy()
    segs[0] = ((1 << 32) - 100, 200)      # crosses 2^32 -> RANGE at the segment start
    segs[-1] = ((1 << 32) + 8, 16)
    stg = W.payload_bytes(322, wl.staging_bytes)
    out = run_both(img, pool, wl.reqs, segs, stg)
    assert_same(out)
    codes = out["o_res"]["fault_code"]
    assert (codes == 4).any() and (codes == 0x101).any() and (codes == 0).any()


@pytest.mark.parametrize("flags", ["hazard_free", "levelled"])
def test_pae_batches_and_long_segments(flags):
    from paper_1304_3771_b300 import cvd
    img, pool = _pae_guest(323, arena=512 << 20, np_frac=0.002, ro_frac=0.002)
    rng = np.random.default_rng(323)
    sizes = np.concatenate([W.batching_sizes(323, 600), W.log_uniform(rng, 2 << 20, 16 << 20, 12)])
    sizes = sizes[rng.permutation(len(sizes))]
    wl = W.batched_requests(img, 323, sizes, 8)
    lo, hi = wl.batches[0]
    stg = W.payload_bytes(324, wl.staging_bytes)
    f = cvd.BATCH_HAZARD_FREE if flags == "hazard_free" else 0
    out = run_both(img, pool, wl.reqs[lo:hi], wl.segs, stg, flags=f)
    assert_same(out)
    codes = out["o_res"]["fault_code"]
    assert (codes != 0).any() and (codes == 0).any()


def _install_both(img_or_pool, reqs, hf, **g):
    import torch
    from paper_1304_3771_b300 import cvd
    pool = img_or_pool
    o_pool = pool.copy()
    og = O.Guest(o_pool, g["slots"], g["cr3"], pt_pool_gfn=g["pt_pool_gfn"], pt_pool_n=g["pt_pool_n"],
                 rsv_gfn=g["rsv_gfn"], rsv_n=g["rsv_n"], paging=1)
    pool_d = torch.from_numpy(pool.copy()).cuda()
    dg = cvd.Guest(pool_d, g["slots"], g["cr3"], pt_pool_gfn=g["pt_pool_gfn"], pt_pool_n=g["pt_pool_n"],
                   rsv_gfn=g["rsv_gfn"], rsv_n=g["rsv_n"], paging=1)
    o_st = og.mmap_install(reqs, hf)
    npg = int(reqs["npages"].astype(np.int64).sum())
    st = torch.zeros(max(npg, 1), dtype=torch.int32, device="cuda")
    dg.mmap_install(cvd.records_to_device(reqs), len(reqs), cvd.u64_to_device(hf), len(hf), st)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(st.cpu().numpy()[:npg], o_st)
    assert np.array_equal(pool_d.cpu().numpy(), o_pool), "page tables differ"
    np.testing.assert_array_equal(cvd.u64_from_device(dg.p2m)[:g["rsv_n"]], og.p2m[:g["rsv_n"]])
    assert dg.alloc_state() == (og.pt_used, og.rsv_used)
    return og, dg, o_st


def test_pae_hand_install_on_gpu():
    pool = np.zeros(0x40000, dtype=np.uint8)
    pool[16 * 4096:19 * 4096] = 0xCD                # new tables must be zeroed
    slots = np.array([(0, 0x40, 0)], dtype=W.SLOT_DTYPE)
    reqs = np.zeros(3, dtype=W.MAPREQ_DTYPE)
    reqs[0] = (0x40000000, 1, W.PTE_RW | W.PTE_US, 0)
    reqs[1] = (0x40201000, 1, W.PTE_US, 1)
    reqs[2] = (0x40000000, 1, W.PTE_RW | W.PTE_US, 2)   # duplicate -> EBUSY
    hf = np.array([0x21, 0x22, 0x23], dtype=np.uint64)
    og, dg, st = _install_both(pool, reqs, hf, slots=slots, cr3=0x1000, pt_pool_gfn=16, pt_pool_n=16,
                               rsv_gfn=0x100, rsv_n=8)
    assert st.tolist() == [0, 0, -16]
    dg.close()


def test_pae_generated_install_and_translate_after():
    import torch
    from paper_1304_3771_b300 import cvd
    img, _ = _pae_guest(325, pt_pool_n=4096, rsv_n=1 << 18)
    pool = W.materialize_pool(img, fill=False)
    reqs, hf, win = W.mmap_requests(img, 325, 1500, window_bytes=512 << 20, busy_frac=0.03, bad_flag_frac=0.01)
    og, dg, st = _install_both(pool, reqs, hf, slots=img.slots, cr3=img.cr3_gpa, pt_pool_gfn=img.pt_pool_gfn,
                               pt_pool_n=img.pt_pool_n, rsv_gfn=img.rsv_gfn, rsv_n=img.rsv_n)
    assert (st == 0).sum() > 100_000 and (st == -16).any() and (st == -22).any()
    va = (win + np.arange(0, 512 << 20, 4096 * 7, dtype=np.uint64)).astype(np.uint64)
    gpa, hpa, code = dg.translate(cvd.u64_to_device(va))
    torch.cuda.synchronize()
    exp = og.translate(va)
    np.testing.assert_array_equal(code.cpu().numpy().view(np.uint32), exp[2])
    np.testing.assert_array_equal(cvd.u64_from_device(hpa), exp[1])
    dg.close()
