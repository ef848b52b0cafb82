"""GPU parity for guests behind a software EPT (the second dimension without
KVM, Sec. 4.2; EPT format per the Intel SDM Vol. 3 sec. 28.3.2): translation
on hand-encoded and generated tables, copies through the levelled and the
hazard-free paths (long segments and EPT faults included), batches that mix
EPT and memslot guests, and installs refused page by page -- each compared
with the oracle element by element."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W
from tests.gpu_helpers import assert_same, run_both
from tests.oracle_fixtures import golden_pool, parse_golden

pytestmark = pytest.mark.gpu


def _hand():
    import torch
    from paper_1304_3771_b300 import cvd
    gd = parse_golden("walk_ept_hand.txt")
    pool, slots = golden_pool(gd)
    rg, rn = gd["rsv"]
    p2m = np.full(rn, O.NO_FRAME, dtype=np.uint64)
    for i, f in gd["p2m_set"]:
        p2m[i] = f
    p2m_d = torch.from_numpy(p2m.view(np.int64).copy()).cuda()
    g = cvd.Guest(torch.from_numpy(pool).cuda(), slots[:0], gd["cr3"], rsv_gfn=rg, rsv_n=rn, p2m=p2m_d,
                  ept_root=gd["ept_root"])
    og = O.Guest(pool, slots, gd["cr3"], rsv_gfn=rg, rsv_n=rn, p2m=p2m, ept_root=gd["ept_root"])
    return gd, g, og


def test_ept_hand_tables_translate():
    import torch
    from paper_1304_3771_b300 import cvd
    gd, g, og = _hand()
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


def _ept_guest(seed, arena=64 << 20, paging="x86_64", np_frac=0.01, ro_frac=0.02, **kw):
    args = dict(np_frac=0.02, ro_frac=0.02, huge_frac=0.3, nslots=3, host_base=2 << 20, slot_gap_pages=512)
    args.update(kw)
    img0 = W.make_guest(arena, seed, paging=paging, **args)
    img = W.add_ept(img0, seed, np_frac=np_frac, ro_frac=ro_frac)
    return img, W.materialize_pool(img)


@pytest.mark.parametrize("paging,write", [("x86_64", False), ("x86_64", True), ("pae", True)])
def test_ept_translate_generated(paging, write):
    import torch
    from paper_1304_3771_b300 import cvd
    img, pool = _ept_guest(430, paging=paging)
    g = cvd.Guest.from_image(img, torch.from_numpy(pool).cuda())
    va = W.translate_gvas(img, 430, 100_003)
    gpa, hpa, code = g.translate(cvd.u64_to_device(va), write=write)
    torch.cuda.synchronize()
    exp = O.Guest.from_image(img, pool).translate(va, write)
    np.testing.assert_array_equal(code.cpu().numpy().view(np.uint32), exp[2])
    np.testing.assert_array_equal(cvd.u64_from_device(gpa), exp[0])
    np.testing.assert_array_equal(cvd.u64_from_device(hpa), exp[1])
    assert (exp[2] == 5).any() and (exp[2] == 0).any()
    if write:
        assert (exp[2] == 10).any()
    g.close()


@pytest.mark.parametrize("basic", [None, "from", "to"])
def test_ept_copies_small(basic):
    img, pool = _ept_guest(431)
    wl = W.tiny_requests(img, 431, nreq=400, hi=60000, frame_frac=0.05)
    stg = W.payload_bytes(432, wl.staging_bytes)
    if basic:
        wl.reqs["dir"] = 0 if basic == "from" else 1
    out = run_both(img, pool, wl.reqs, wl.segs, stg, basic=basic)
    assert_same(out)
    codes = out["o_res"]["fault_code"]
    assert (codes == 0).any() and (codes == 5).any()
    if basic != "from":
        assert (codes == 10).any()


@pytest.mark.parametrize("flags", ["hazard_free", "levelled"])
def test_ept_batches_and_long_segments(flags):
    from paper_1304_3771_b300 import cvd
    img, pool = _ept_guest(433, arena=512 << 20, np_frac=0.0005, ro_frac=0.001)
    rng = np.random.default_rng(433)
    sizes = np.concatenate([W.batching_sizes(433, 600), W.log_uniform(rng, 2 << 20, 16 << 20, 12)])
    sizes = sizes[rng.permutation(len(sizes))]
    wl = W.batched_requests(img, 433, sizes, 8)
    lo, hi = wl.batches[0]
    stg = W.payload_bytes(434, wl.staging_bytes)
    f = cvd.BATCH_HAZARD_FREE if flags == "hazard_free" else 0
    out = run_both(img, pool, wl.reqs[lo:hi], wl.segs, stg, flags=f)
    assert_same(out)
    codes = out["o_res"]["fault_code"]
    assert (codes != 0).any() and (codes == 0).any()


def test_ept_and_memslot_guests_in_one_batch():
    """Requests for an EPT guest and a memslot guest interleaved in one call
    (the per-walk second dimension), each guest's result against the oracle
    running the same call over both guests."""
    import torch
    from paper_1304_3771_b300 import cvd
    img_e, pool_e = _ept_guest(435)
    img_m = W.make_guest(64 << 20, 436, huge_frac=0.3, np_frac=0.02, ro_frac=0.02)
    pool_m = W.materialize_pool(img_m)
    a = W.tiny_requests(img_e, 435, nreq=200, hi=40000, guest=0)
    b = W.tiny_requests(img_m, 436, nreq=200, hi=40000, guest=1)
    segs = np.concatenate([a.segs, b.segs])
    reqs = np.concatenate([a.reqs, b.reqs])
    reqs["seg_begin"][len(a.reqs):] += len(a.segs)
    reqs["host_off"][len(a.reqs):] += a.staging_bytes
    order = np.random.default_rng(437).permutation(len(reqs))
    reqs = reqs[order]
    stg = W.payload_bytes(438, a.staging_bytes + b.staging_bytes)
    o_pe, o_pm, o_stg = pool_e.copy(), pool_m.copy(), stg.copy()
    o_res = O.copy_batch([O.Guest.from_image(img_e, o_pe), O.Guest.from_image(img_m, o_pm)], reqs, segs, o_stg)
    pe_d, pm_d = torch.from_numpy(pool_e.copy()).cuda(), torch.from_numpy(pool_m.copy()).cuda()
    ge, gm = cvd.Guest.from_image(img_e, pe_d), cvd.Guest.from_image(img_m, pm_d)
    stg_d = torch.from_numpy(stg.copy()).cuda()
    res_d = torch.zeros(len(reqs) * W.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cvd.copy_batch([ge, gm], cvd.records_to_device(reqs), len(reqs), cvd.records_to_device(segs), len(segs),
                   stg_d, res_d)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(cvd.records_from_device(res_d, W.RESULT_DTYPE, len(reqs)), o_res)
    assert np.array_equal(stg_d.cpu().numpy(), o_stg)
    assert np.array_equal(pe_d.cpu().numpy(), o_pe) and np.array_equal(pm_d.cpu().numpy(), o_pm)
    assert (o_res["fault_code"] == 0).any() and (o_res["fault_code"] != 0).any()
    ge.close()
    gm.close()


def test_ept_install_refused_on_gpu():
    import torch
    from paper_1304_3771_b300 import cvd
    img, pool = _ept_guest(439)
    reqs, hf, _ = W.mmap_requests(img, 439, 40, window_bytes=64 << 20)
    pool_d = torch.from_numpy(pool.copy()).cuda()
    g = cvd.Guest.from_image(img, pool_d)
    npg = int(reqs["npages"].astype(np.int64).sum())
    st = torch.zeros(npg, dtype=torch.int32, device="cuda")
    g.mmap_install(cvd.records_to_device(reqs), len(reqs), cvd.u64_to_device(hf), len(hf), st)
    torch.cuda.synchronize()
    o_st = O.Guest.from_image(img, pool.copy()).mmap_install(reqs, hf)
    np.testing.assert_array_equal(st.cpu().numpy(), o_st)
    assert (o_st == -22).all()
    assert np.array_equal(pool_d.cpu().numpy(), pool) and g.alloc_state() == (0, 0)
    g.close()
