"""GPU parity of cvd_mmap_install (insert_pfn, Sec. 6.2; guest PTE to a
reserved frame plus second-dimension map, new tables from the frontend's
pool, Sec. 4.2) against the sequential oracle: every page status, every byte
of the host pool (so every page-table entry), the p2m array and the
allocation counters, bit-exact."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W
from tests.oracle_fixtures import golden_maps, golden_pool, parse_golden

pytestmark = pytest.mark.gpu


def _install_both(pool, slots, cr3, reqs, hf, *, pt_pool_gfn, pt_pool_n, rsv_gfn, rsv_n, calls=1):
    import torch
    from paper_1304_3771_b300 import cvd
    o_pool = pool.copy()
    og = O.Guest(o_pool, slots, cr3, pt_pool_gfn=pt_pool_gfn, pt_pool_n=pt_pool_n, rsv_gfn=rsv_gfn, rsv_n=rsv_n)
    pool_d = torch.from_numpy(pool.copy()).cuda()
    g = cvd.Guest(pool_d, slots, cr3, pt_pool_gfn=pt_pool_gfn, pt_pool_n=pt_pool_n, rsv_gfn=rsv_gfn, rsv_n=rsv_n)
    parts = np.array_split(np.arange(len(reqs)), calls)
    hf_d = cvd.u64_to_device(hf)
    for idx in parts:
        r = reqs[idx]
        o_st = og.mmap_install(r, hf)
        npg = int(r["npages"].astype(np.int64).sum())
        st_d = torch.zeros(max(npg, 1), dtype=torch.int32, device="cuda")
        g.mmap_install(cvd.records_to_device(r), len(r), hf_d, len(hf), st_d)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(st_d.cpu().numpy()[:npg], o_st)
    assert np.array_equal(pool_d.cpu().numpy(), o_pool), "page tables differ"
    np.testing.assert_array_equal(cvd.u64_from_device(g.p2m)[:rsv_n], og.p2m[:rsv_n])
    assert g.alloc_state() == (og.pt_used, og.rsv_used)
    return og, g, o_st


def test_hand_computed_install_on_gpu():
    gd = parse_golden("mmap_hand.txt")
    pool, slots = golden_pool(gd)
    pool[0x3000 + 8 * 4096:0x3000 + 12 * 4096] = 0xCD     # the install must zero new tables
    reqs, hf = golden_maps(gd)
    rg, rn = gd["rsv"]
    og, g, st = _install_both(pool, slots, gd["cr3"], reqs, hf, pt_pool_gfn=gd["ptpool"][0],
                              pt_pool_n=gd["ptpool"][1], rsv_gfn=rg, rsv_n=rn)
    assert st.tolist() == gd["status"]
    g.close()


@pytest.mark.parametrize("calls", [1, 3])
def test_translate_mmap_shape_install(calls):
    img = W.make_guest(256 << 20, 301, pt_pool_n=8192, rsv_n=1 << 20)
    pool = W.materialize_pool(img, fill=False)
    reqs, hf, win = W.mmap_requests(img, 301, 3000, window_bytes=16 << 30, busy_frac=0.02, bad_flag_frac=0.01)
    og, g, _ = _install_both(pool, img.slots, img.cr3_gpa, reqs, hf, pt_pool_gfn=img.pt_pool_gfn,
                             pt_pool_n=img.pt_pool_n, rsv_gfn=img.rsv_gfn, rsv_n=img.rsv_n, calls=calls)
    assert og.rsv_used > 100_000 and og.pt_used > 100
    # translate after install: GPU walk through the new tables and the p2m
    import torch
    from paper_1304_3771_b300 import cvd
    rng = np.random.default_rng(3)
    k = rng.integers(0, len(reqs), 20_000)
    va = (reqs["gva"][k] + rng.integers(0, 1 << 20, 20_000).astype(np.uint64)).astype(np.uint64)
    exp = og.translate(va)
    out = g.translate(cvd.u64_to_device(va))
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cvd.u64_from_device(out[0]), exp[0])
    np.testing.assert_array_equal(cvd.u64_from_device(out[1]), exp[1])
    np.testing.assert_array_equal(out[2].cpu().numpy().view(np.uint32), exp[2])
    assert (exp[2] == 0).sum() > 1000
    g.close()


def test_enomem_latch_small_pools():
    img = W.make_guest(64 << 20, 302, pt_pool_n=40, rsv_n=5000)
    pool = W.materialize_pool(img, fill=False)
    reqs, hf, win = W.mmap_requests(img, 302, 400, window_bytes=64 << 30, busy_frac=0.05, bad_flag_frac=0.02)
    og, g, st = _install_both(pool, img.slots, img.cr3_gpa, reqs, hf, pt_pool_gfn=img.pt_pool_gfn,
                              pt_pool_n=img.pt_pool_n, rsv_gfn=img.rsv_gfn, rsv_n=img.rsv_n)
    assert (st == -12).sum() > 1000 and (st == 0).sum() > 100
    g.close()
