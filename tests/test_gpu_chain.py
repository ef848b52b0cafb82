"""GPU parity for dependent second-level gathers (a command submission whose
structure names further guest buffers; generic class drivers, Sec. 6.1):
results, descriptor buffer and payload buffer against the oracle, byte for
byte, on hand-built identity maps, generated guests with faults at both
levels (x86-64, PAE, an EPT guest, two guests in one call), HOSTBUF and
malformed requests, and long buffers that take the planner's long-segment
path."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W
from tests.oracle_fixtures import identity_guest

pytestmark = pytest.mark.gpu
PAGE = 4096


def _run_both(imgs_pools, reqs, desc_bytes, payload_bytes, flags=0, guests_kw=None):
    """imgs_pools: list of (image or None, pool, oracle-guest kwargs or None)."""
    import torch
    from paper_1304_3771_b300 import cvd
    o_guests, d_guests, pools_d = [], [], []
    o_pools = [p.copy() for _, p, _ in imgs_pools]
    for (img, pool, kw), op in zip(imgs_pools, o_pools):
        pd = torch.from_numpy(pool.copy()).cuda()
        pools_d.append(pd)
        if img is not None:
            o_guests.append(O.Guest.from_image(img, op))
            d_guests.append(cvd.Guest.from_image(img, pd))
        else:
            o_guests.append(O.Guest(op, kw["slots"], kw["cr3"]))
            d_guests.append(cvd.Guest(pd, kw["slots"], kw["cr3"]))
    o_desc = np.full(desc_bytes, 0xEE, np.uint8)
    o_pay = np.full(payload_bytes, 0xEE, np.uint8)
    o_res = O.gather_chained(o_guests, reqs, o_desc, o_pay)
    desc = torch.full((max(desc_bytes, 1),), 0xEE, dtype=torch.uint8, device="cuda")[:desc_bytes]
    pay = torch.full((max(payload_bytes, 1),), 0xEE, dtype=torch.uint8, device="cuda")[:payload_bytes]
    res = torch.zeros(max(len(reqs), 1) * W.CHAIN_RES_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cvd.gather_chained(d_guests, cvd.records_to_device(reqs), len(reqs), desc, pay, res, flags=flags)
    torch.cuda.synchronize()
    g_res = cvd.records_from_device(res, W.CHAIN_RES_DTYPE, len(reqs))
    np.testing.assert_array_equal(g_res, o_res)
    assert np.array_equal(desc.cpu().numpy(), o_desc), "descriptor bytes differ"
    assert np.array_equal(pay.cpu().numpy(), o_pay), "payload bytes differ"
    for pd, op in zip(pools_d, o_pools):
        assert np.array_equal(pd.cpu().numpy(), op)
    for g in d_guests:
        g.close()
    return o_res


def _table(entries):
    t = np.zeros(2 * len(entries), dtype=np.uint64)
    for k, (g, n) in enumerate(entries):
        t[2 * k], t[2 * k + 1] = g, n
    return t.view(np.uint8)


def test_chain_identity_and_hostbuf():
    base, host = 1 << 30, 0x5000
    pool, slots, cr3 = identity_guest(64, base_gva=base, host_off=host)

    def put(g, d):
        pool[host + g - base:host + g - base + len(d)] = d

    put(base + 0x100, _table([(base + 0x9000, 100), (base + 0x1FFF0, 5000)]))
    put(base + 0x0FF8, _table([]))
    put(base + 0x2000 - 16, _table([(base + 0x300, 1), (base + 0x20000, 4096)]))
    put(base + 0x400, _table([(base + 0x1000, 50), (base, (1 << 64) - 10)]))
    reqs = np.zeros(7, dtype=W.CHAIN_REQ_DTYPE)
    reqs[0] = (base + 0x100, 2, 0, 0)
    reqs[1] = (base + 0x0FF8, 0, 0, 32)
    reqs[2] = (base + 0x2000 - 16, 2, 0, 32)
    reqs[3] = (base + 0x400, 2, 0, 64)              # saturated length: HOSTBUF
    reqs[4] = (base + 0x100, 70000, 0, 96)          # BADREQ
    reqs[5] = (base + 0x100, 1, 0, 100)             # desc_off not a multiple of 16: BADREQ
    reqs[6] = (base + 0x100, 1, 5, 112)             # no guest 5: BADREQ
    res = _run_both([(None, pool, dict(slots=slots, cr3=cr3))], reqs, 128, 12000)
    assert res["level"].tolist() == [0, 0, 0, 2, 1, 1, 1]
    assert res["fault_code"].tolist() == [0, 0, 0, 8, 9, 9, 9]


@pytest.mark.parametrize("paging", ["x86_64", "pae"])
def test_chain_generated_faults(paging):
    img = W.make_guest(64 << 20, 470, paging=paging, huge_frac=0.3, np_frac=0.01, ro_frac=0.0, nslots=3)
    pool = W.materialize_pool(img)
    wl = W.chained_requests(img, 470, 800, max_count=16, hi=30000)
    for g, t in wl.tables:
        W.write_gva(img, pool, g, t)
    # tables moved onto (or running into) pages whose leaf is not present
    absent = np.nonzero((img.page_gfn >= 0) & ((img.page_flags & np.uint64(W.PTE_P)) == 0))[0]
    reqs = wl.reqs.copy()
    for k, r in enumerate(range(0, len(reqs), 50)):
        p = int(absent[k % len(absent)])
        reqs["table_gva"][r] = img.data_gva + p * PAGE - (16 if k % 2 else 0)
    res = _run_both([(img, pool, None)], reqs, wl.desc_bytes, wl.payload_bytes, flags=1)
    lv = res["level"]
    assert (lv == 0).sum() > 400 and (lv == 2).any() and (lv == 1).any()


def test_chain_two_guests_and_ept():
    img_a = W.make_guest(64 << 20, 471, huge_frac=0.3, np_frac=0.01, host_base=2 << 20)
    img_b = W.add_ept(W.make_guest(64 << 20, 472, huge_frac=0.3, np_frac=0.0, host_base=2 << 20), 472,
                      np_frac=0.01)
    pa, pb = W.materialize_pool(img_a), W.materialize_pool(img_b)
    wa = W.chained_requests(img_a, 471, 300, max_count=12, hi=20000)
    wb = W.chained_requests(img_b, 472, 300, max_count=12, hi=20000)
    for g, t in wa.tables:
        W.write_gva(img_a, pa, g, t)
    for g, t in wb.tables:
        W.write_gva(img_b, pb, g, t)
    rb = wb.reqs.copy()
    rb["guest"] = 1
    rb["desc_off"] += wa.desc_bytes
    reqs = np.concatenate([wa.reqs, rb])[np.random.default_rng(473).permutation(600)]
    res = _run_both([(img_a, pa, None), (img_b, pb, None)], reqs, wa.desc_bytes + wb.desc_bytes,
                    wa.payload_bytes + wb.payload_bytes)
    assert (res["level"] == 0).sum() > 300 and (res["level"] != 0).any()


def test_chain_long_buffers_and_small_payload_buffer():
    """Entries up to 8 MiB (the planner's long-segment list) and a payload
    buffer that holds only part of the requests (HOSTBUF for the rest)."""
    img = W.make_guest(512 << 20, 474, huge_frac=0.5, np_frac=0.002, ro_frac=0.0)
    pool = W.materialize_pool(img)
    wl = W.chained_requests(img, 474, 200, max_count=6, lo=4096, hi=8 << 20, table_area=0.01)
    for g, t in wl.tables:
        W.write_gva(img, pool, g, t)
    res = _run_both([(img, pool, None)], wl.reqs, wl.desc_bytes, wl.payload_bytes // 2, flags=1)
    assert (res["fault_code"] == 8).any() and (res["level"] == 0).sum() > 50


def test_chain_edge_cases():
    """Empty tables, overlapping descriptor ranges (level 1 levelled: the later
    table's bytes win, as in sequential order), a request whose table is in no
    mapped page, and a call with no requests."""
    import torch
    from paper_1304_3771_b300 import cvd
    base, host = 1 << 30, 0x5000
    pool, slots, cr3 = identity_guest(64, base_gva=base, host_off=host)

    def put(g, d):
        pool[host + g - base:host + g - base + len(d)] = d

    put(base + 0x100, _table([(base + 0x9000, 100), (base + 0x3000, 50)]))
    put(base + 0x200, _table([(base + 0x4000, 70)]))
    reqs = np.zeros(5, dtype=W.CHAIN_REQ_DTYPE)
    reqs[0] = (base + 0x100, 2, 0, 0)
    reqs[1] = (base + 0x200, 1, 0, 16)      # overlaps request 0's second entry
    reqs[2] = (base + 0x100, 0, 0, 48)      # empty table
    reqs[3] = (base + (70 << 12), 1, 0, 48)  # beyond the mapped pages: level 1
    reqs[4] = (base + 0x200, 1, 0, 64)
    res = _run_both([(None, pool, dict(slots=slots, cr3=cr3))], reqs, 96, 1000)
    assert res["level"].tolist()[2:4] == [0, 1] and res["payload_len"][2] == 0
    # no requests at all
    from paper_1304_3771_b300 import cvd as _c
    g = _c.Guest(torch.from_numpy(pool.copy()).cuda(), slots, cr3)
    e = torch.zeros(16, dtype=torch.uint8, device="cuda")
    _c.gather_chained([g], e, 0, e, e, e)
    torch.cuda.synchronize()
    g.close()


def test_chain_hazard_free_table_reads_edge_cases():
    """Level 1 of a hazard-free call (one warp per table on the device) gives
    the batch rules' results: an empty table, count above the maximum,
    desc_off not a multiple of 16, a guest index out of range, a table that
    passes the end of the descriptor buffer, a non-canonical and an
    out-of-range table address, and a table running into an unmapped page
    (prefix copied, rest zero-filled)."""
    base, host = 1 << 30, 0x5000
    pool, slots, cr3 = identity_guest(64, base_gva=base, host_off=host)

    def put(g, d):
        pool[host + g - base:host + g - base + len(d)] = d

    put(base + 0x100, _table([(base + 0x9000, 100), (base + 0x3000, 50)]))
    put(base + (64 << 12) - 16, _table([(base + 0x4000, 70)]))   # 16 B before the end of the mapping
    reqs = np.zeros(9, dtype=W.CHAIN_REQ_DTYPE)
    reqs[0] = (base + 0x100, 2, 0, 0)
    reqs[1] = (base + 0x100, 0, 0, 32)                   # empty table
    reqs[2] = (base + 0x100, 70000, 0, 32)               # count above the maximum: BADREQ
    reqs[3] = (base + 0x100, 1, 0, 40)                   # desc_off not a multiple of 16: BADREQ
    reqs[4] = (base + 0x100, 1, 3, 48)                   # no guest 3: BADREQ
    reqs[5] = (base + 0x100, 8, 0, 224)                  # 128 B at 224 of a 256 B buffer: HOSTBUF
    reqs[6] = ((1 << 63) | 0x1000, 1, 0, 64)             # non-canonical
    reqs[7] = ((1 << 47) - 16, 2, 0, 80)                 # passes the user range
    reqs[8] = (base + (64 << 12) - 16, 3, 0, 112)        # first entry mapped, the rest in no page
    res = _run_both([(None, pool, dict(slots=slots, cr3=cr3))], reqs, 256, 1000, flags=1)
    codes = res["fault_code"].tolist()
    assert codes[:8] == [0, 0, 9, 9, 9, 8, 3, 4]
    assert res["level"].tolist() == [0, 0, 1, 1, 1, 1, 1, 1, 1]
    assert res["done"][8] == 16 and codes[8] != 0
