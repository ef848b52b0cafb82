"""The oracle's dependent second-level gathers (a command submission whose
structure holds further guest pointers: the host driver reads the structure, then
gathers what it names -- generic class drivers, Sec. 6.1; copy_from_user per
page, Sec. 4.2), pinned without the oracle's own composition: on an identity
map the tables and payloads must equal bytes read straight from the pool at
gva - base (closed form); on a generated guest every payload byte is
re-derived page by page through the walk; hand-placed faults at both levels
give hand-derived done / fault_gva / level; payload offsets are prefix sums;
HOSTBUF, saturation and malformed requests follow the stated rules."""
import numpy as np

import oracle as O
from paper_1304_3771_b300 import workload as W
from tests.oracle_fixtures import identity_guest

PAGE = 4096
BASE = 1 << 30
HOST = 0x5000


def _table(entries):
    t = np.zeros(2 * len(entries), dtype=np.uint64)
    for k, (g, n) in enumerate(entries):
        t[2 * k], t[2 * k + 1] = g, n
    return t.view(np.uint8)


def _ident(npages=64):
    pool, slots, cr3 = identity_guest(npages, base_gva=BASE, host_off=HOST)
    return pool, O.Guest(pool, slots, cr3)


def _put(pool, gva, data):
    h = HOST + (gva - BASE)
    pool[h:h + len(data)] = data


def test_identity_closed_form():
    pool, og = _ident()
    specs = [[(BASE + 0x9000, 100), (BASE + 0x1FFF0, 5000)], [], [(BASE + 0x300, 1), (BASE + 0x20000, 4096)]]
    reqs = np.zeros(3, dtype=W.CHAIN_REQ_DTYPE)
    tg = [BASE + 0x100, BASE + 0x0FF8, BASE + 0x2000 - 16]     # the second is empty, the third crosses a page
    off = 0
    for r, (sp, g) in enumerate(zip(specs, tg)):
        _put(pool, g, _table(sp))
        reqs[r] = (g, len(sp), 0, off)
        off += 16 * len(sp)
    desc = np.full(off + 32, 0xEE, np.uint8)
    payload = np.full(20000, 0xEE, np.uint8)
    snap = pool.copy()
    res = O.gather_chained([og], reqs, desc, payload)
    assert np.array_equal(pool, snap)                          # gathers never write guest memory
    lens = [sum(n for _, n in sp) for sp in specs]
    assert res["payload_len"].tolist() == lens
    assert res["payload_off"].tolist() == [0, lens[0], lens[0]]
    assert (res["fault_code"] == 0).all() and (res["level"] == 0).all() and res["done"].tolist() == lens
    for r, sp in enumerate(specs):
        assert np.array_equal(desc[reqs["desc_off"][r]:reqs["desc_off"][r] + 16 * len(sp)], _table(sp))
        p = int(res["payload_off"][r])
        for g, n in sp:
            h = HOST + (g - BASE)
            assert np.array_equal(payload[p:p + n], snap[h:h + n])
            p += n
    assert (payload[sum(lens):] == 0xEE).all() and (desc[off:] == 0xEE).all()


def test_faults_at_both_levels_hand_derived():
    pool, slots, cr3 = identity_guest(64, base_gva=BASE, host_off=HOST)
    # page 40 of the identity map not present: clear P of its PTE in the pool
    og0 = O.Guest(pool, slots, cr3)
    _, gpa_pt, _ = og0.walk(BASE + 40 * PAGE)
    # find the PTE: scan the table frames for the entry mapping gfn 40
    tab = pool[HOST:].view(np.uint64)
    idx = np.nonzero((tab & np.uint64(0x000FFFFFFFFFF001)) == np.uint64((40 << 12) | 1))[0]
    assert len(idx) == 1
    tab[idx[0]] &= ~np.uint64(1)
    og = O.Guest(pool, slots, cr3)
    assert og.walk(BASE + 40 * PAGE + 8)[0] == 0x101
    reqs = np.zeros(3, dtype=W.CHAIN_REQ_DTYPE)
    # request 0: table of 3 entries starting 16 bytes before the hole -> level 1, 16 bytes read
    t0 = BASE + 40 * PAGE - 16
    _put(pool, t0, _table([(BASE, 8)]))
    reqs[0] = (t0, 3, 0, 0)
    # request 1: entries 100 B, then a buffer running into the hole -> level 2
    t1 = BASE + 0x100
    _put(pool, t1, _table([(BASE + 0x3000, 100), (BASE + 40 * PAGE - 50, 200)]))
    reqs[1] = (t1, 2, 0, 48)
    # request 2: fine
    t2 = BASE + 0x200
    _put(pool, t2, _table([(BASE + 0x5000, 30)]))
    reqs[2] = (t2, 1, 0, 80)
    desc = np.full(96, 0xEE, np.uint8)
    payload = np.full(400, 0xEE, np.uint8)
    res = O.gather_chained([og], reqs, desc, payload)
    r0, r1, r2 = res
    assert (r0["level"], r0["fault_code"], r0["done"], r0["fault_gva"]) == (1, 0x101, 16, BASE + 40 * PAGE)
    assert r0["payload_len"] == 0 and (desc[16:48] == 0).all()            # rest of the table zero-filled
    assert (r1["level"], r1["fault_code"], r1["done"], r1["fault_gva"]) == (2, 0x101, 150, BASE + 40 * PAGE)
    assert (r1["payload_off"], r1["payload_len"]) == (0, 300)
    assert (payload[150:300] == 0).all()                                  # zero-filled after the fault
    assert (r2["level"], r2["fault_code"], r2["done"], r2["payload_off"]) == (0, 0, 30, 300)


def test_hostbuf_saturation_and_malformed():
    pool, og = _ident()
    reqs = np.zeros(6, dtype=W.CHAIN_REQ_DTYPE)
    _put(pool, BASE + 0x100, _table([(BASE + 0x1000, 60)]))
    _put(pool, BASE + 0x200, _table([(BASE + 0x1000, 50), (BASE, (1 << 64) - 10)]))    # L saturates
    _put(pool, BASE + 0x300, _table([(BASE + 0x2000, 30)]))
    reqs[0] = (BASE + 0x100, 1, 0, 0)
    reqs[1] = (BASE + 0x200, 2, 0, 16)          # HOSTBUF (saturated length)
    reqs[2] = (BASE + 0x300, 1, 0, 48)          # after a saturated one: no room either
    reqs[3] = (BASE + 0x300, 65537, 0, 64)      # count above 65,536 (the first past it): BADREQ
    reqs[4] = (BASE + 0x300, 1, 0, 72)          # desc_off not a multiple of 16: BADREQ
    reqs[5] = (BASE + 0x300, 1, 3, 80)          # no guest 3: BADREQ
    desc = np.zeros(96, np.uint8)
    payload = np.full(100, 0xEE, np.uint8)
    res = O.gather_chained([og], reqs, desc, payload)
    assert res["fault_code"].tolist() == [0, 8, 8, 9, 9, 9]
    assert res["level"].tolist() == [0, 2, 2, 1, 1, 1]
    assert res["payload_len"].tolist()[:3] == [60, (1 << 64) - 1, 30]
    assert res["payload_off"].tolist() == [0, 0, 0, 0, 0, 0]
    assert (payload[60:] == 0xEE).all()


def test_generated_guest_payload_rederived_through_the_walk():
    img = W.make_guest(64 << 20, 460, huge_frac=0.3, np_frac=0.01, ro_frac=0.0, nslots=2)
    pool = W.materialize_pool(img)
    wl = W.chained_requests(img, 460, 150, max_count=12, hi=20000)
    for g, t in wl.tables:
        W.write_gva(img, pool, g, t)
    og = O.Guest.from_image(img, pool)
    desc = np.zeros(wl.desc_bytes, np.uint8)
    payload = np.full(wl.payload_bytes, 0xEE, np.uint8)
    res = O.gather_chained([og], wl.reqs, desc, payload)
    assert (res["level"] == 0).sum() > 80 and (res["level"] == 2).any()
    cursor = 0
    for r, q in enumerate(wl.reqs):
        g0, t = wl.tables[r]
        if res["level"][r] == 1:
            assert res["payload_len"][r] == 0
            continue
        assert np.array_equal(desc[q["desc_off"]:q["desc_off"] + len(t)], t)
        ent = t.view(np.uint64).reshape(-1, 2)
        assert res["payload_len"][r] == ent[:, 1].sum() and res["payload_off"][r] == cursor
        # every payload byte up to `done` re-read page by page through the walk
        done, p = int(res["done"][r]), cursor
        for gva, n in ent:
            gva, n = int(gva), int(n)
            k = 0
            while k < n and p < cursor + done:
                va = gva + k
                m = min(n - k, PAGE - va % PAGE, cursor + done - p)
                code, _, h = og.walk(va)
                assert code == 0
                assert np.array_equal(payload[p:p + m], pool[h:h + m])
                p += m
                k += m
        assert (payload[cursor + done:cursor + int(res["payload_len"][r])] == 0).all()
        cursor += int(res["payload_len"][r])


def test_entry_list_bounded_by_the_descriptor_buffer():
    """Tables that overlap in the descriptor buffer: the payload entry list
    holds desc_bytes / 16 entries, places are running sums of the counts of
    the requests whose table was read whole, and a request whose entries pass
    the capacity gets HOSTBUF at level 2 (hand-derived: capacity 4 entries)."""
    pool, og = _ident()
    _put(pool, BASE + 0x100, _table([(BASE + 0x1000, 10), (BASE + 0x1100, 20)]))
    _put(pool, BASE + 0x200, _table([(BASE + 0x2000, 5)]))
    reqs = np.zeros(4, dtype=W.CHAIN_REQ_DTYPE)
    reqs[0] = (BASE + 0x100, 2, 0, 0)     # entries 0-1
    reqs[1] = (BASE + 0x100, 2, 0, 0)     # the same table bytes again: entries 2-3 (fits exactly)
    reqs[2] = (BASE + 0x200, 1, 0, 32)    # entries 4: past the 4-entry capacity -> HOSTBUF
    reqs[3] = (BASE + 0x200, 1, 0, 48)    # entry 5: past it as well (places keep counting)
    desc = np.zeros(64, np.uint8)
    payload = np.full(200, 0xEE, np.uint8)
    res = O.gather_chained([og], reqs, desc, payload)
    assert res["fault_code"].tolist() == [0, 0, 8, 8]
    assert res["level"].tolist() == [0, 0, 2, 2]
    assert res["payload_len"].tolist() == [30, 30, 5, 5]
    assert res["payload_off"].tolist() == [0, 30, 0, 0]
    assert res["done"].tolist() == [30, 30, 0, 0]
    h = HOST + 0x1000
    exp = np.concatenate([pool[h:h + 10], pool[h + 0x100:h + 0x100 + 20]])
    assert np.array_equal(payload[:30], exp) and np.array_equal(payload[30:60], exp)
    assert (payload[60:] == 0xEE).all()
