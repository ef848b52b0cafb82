"""Host-side fault injection through the C ABI, without a GPU: corrupt memslot
tables, reserved windows and PT pools, malformed copy parameters and batch
arguments.  Every one must come back as a status (CVD_EINVAL) from the
library's host-side checks, before any CUDA call is made."""
import ctypes as C

import pytest

EINVAL = -22
POOL = 64 << 20


def _lib():
    from paper_1304_3771_b300 import build, cvd
    build.build()
    return cvd, cvd.lib()


def _desc(cvd, slots, **kw):
    arr = (cvd.Memslot * max(len(slots), 1))(*[cvd.Memslot(*s) for s in slots])
    d = cvd.GuestDesc()
    d.d_host_pool = kw.get("pool", 0x10000000)      # never dereferenced by the host checks
    d.host_pool_bytes = kw.get("pool_bytes", POOL)
    d.slots = C.cast(arr, C.c_void_p) if kw.get("slots_ptr", True) else None
    d.nslots = kw.get("nslots", len(slots))
    d.cr3_gpa = kw.get("cr3", 10 << 12)
    d.paging = kw.get("paging", 0)
    d.pt_pool_gfn, d.pt_pool_n = kw.get("pt", (100, 10))
    d.rsv_gfn, d.rsv_n = kw.get("rsv", (1 << 20, 16))
    d.d_p2m = kw.get("p2m", 0x20000000)
    d.second = kw.get("second", 0)
    d.reserved1 = kw.get("reserved1", 0)
    d.ept_root = kw.get("ept_root", 0)
    return d, arr


GOOD = [(0, POOL >> 12, 0)]

CASES = {
    "no slots": dict(slots=GOOD, nslots=0),
    "more than 64 slots": dict(slots=[(i * 16, 16, i * 65536) for i in range(65)]),
    "null slot array": dict(slots=GOOD, slots_ptr=False),
    "null host pool": dict(slots=GOOD, pool=None),
    "slot host offset not page aligned": dict(slots=[(0, 1024, 100)]),
    "empty slot": dict(slots=[(0, 0, 0)]),
    "slot past the pool end": dict(slots=[(0, (POOL >> 12) + 1, 0)]),
    "slot starting past the pool": dict(slots=[(0, 16, POOL + 4096)]),
    "overlapping slots": dict(slots=[(0, 2048, 0), (1024, 2048, 16 << 20)]),
    "guest frame numbers wrap": dict(slots=[((1 << 64) - 8, 16, 0)]),
    "reserved window over a slot": dict(slots=GOOD, rsv=(100, 16)),
    "reserved window wraps": dict(slots=GOOD, rsv=((1 << 64) - 4, 16)),
    "reserved window without p2m": dict(slots=GOOD, p2m=None),
    "PT pool outside every slot": dict(slots=[(0, 1024, 0)], pt=(5000, 10)),
    "PT pool running past its slot": dict(slots=[(0, 1024, 0)], pt=(1020, 10)),
    "unknown paging format": dict(slots=GOOD, paging=2),
    "PAE cr3 not 32-byte aligned": dict(slots=GOOD, paging=1, cr3=0x1010),
    "PAE cr3 above 4 GiB": dict(slots=GOOD, paging=1, cr3=1 << 32),
    "unknown second dimension": dict(slots=GOOD, second=2),
    "reserved word set": dict(slots=GOOD, reserved1=1),
    "EPT guest with memslots": dict(slots=GOOD, second=1, pt=(0, 0)),
    "EPT guest with a PT pool": dict(slots=[], second=1, pt=(100, 10)),
    "EPT root not 4 KiB aligned": dict(slots=[], second=1, pt=(0, 0), ept_root=0x1008),
    "EPT root table past the pool": dict(slots=[], second=1, pt=(0, 0), ept_root=POOL - 2048),
    "EPT root outside the pool": dict(slots=[], second=1, pt=(0, 0), ept_root=POOL),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_guest_create_rejects_corrupt_descriptor(name):
    cvd, lib = _lib()
    kw = dict(CASES[name])
    d, keep = _desc(cvd, kw.pop("slots"), **kw)
    out = C.c_void_p()
    assert lib.cvd_guest_create(C.byref(d), C.byref(out)) == EINVAL
    assert not out.value


def test_guest_create_rejects_null_arguments():
    cvd, lib = _lib()
    d, keep = _desc(cvd, GOOD)
    out = C.c_void_p()
    assert lib.cvd_guest_create(None, C.byref(out)) == EINVAL
    assert lib.cvd_guest_create(C.byref(d), None) == EINVAL


@pytest.mark.parametrize("bad", [dict(chunk_bytes=1000), dict(chunk_bytes=2048), dict(blocks_per_sm=0),
                                 dict(small_bytes=8192), dict(engine=2), dict(engine=1, warps_per_block=0),
                                 dict(engine=1, warps_per_block=33), dict(engine=1, stages=0),
                                 dict(engine=1, stage_bytes=100), dict(engine=1, ring_bytes=4096),
                                 dict(engine=1, warps_per_block=32, ring_bytes=16512),
                                 dict(engine=0, warps_per_block=32), dict(engine=0, vec_bytes=2)])
def test_copy_params_rejected(bad):
    cvd, lib = _lib()
    p = cvd.CopyParams(vec_bytes=16, unroll=4, chunk_bytes=256 << 10, blocks_per_sm=1, warps_per_block=16,
                       small_bytes=256, engine=1, stages=8, stage_bytes=4096, ring_bytes=8320)
    for k, v in bad.items():
        setattr(p, k, v)
    assert lib.cvd_set_copy_params(C.byref(p)) == EINVAL


def test_batch_calls_reject_bad_arguments_before_cuda():
    cvd, lib = _lib()
    g = (C.c_void_p * 1)(0x1234)
    # no guests
    assert lib.cvd_copy_batch(C.cast(g, C.c_void_p), 0, None, 0, None, 0, None, 0, None, 0, None) == EINVAL
    # more guests than CVD_MAX_GUESTS_PER_BATCH
    g65 = (C.c_void_p * 65)(*([0x1234] * 65))
    assert lib.cvd_copy_batch(C.cast(g65, C.c_void_p), 65, None, 0, None, 0, None, 0, None, 0, None) == EINVAL
    # unknown flag bits on the host-buffer paths
    assert lib.cvd_copy_batch_host(C.cast(g, C.c_void_p), 1, None, 0, None, 0, None, 0, None, 1 << 7, None) == EINVAL
    assert lib.cvd_copy_batches_host(C.cast(g, C.c_void_p), 1, None, 1, 0, None) == EINVAL
    # requests without a results buffer
    hb = cvd.HostBatch(0x1000, 5, 0, 0x2000, 5, 0x3000, 4096, None)
    assert lib.cvd_copy_batches_host(C.cast(g, C.c_void_p), 1, C.byref(hb), 1, 0, None) == EINVAL


def test_probe_and_selftest_reject_bad_arguments():
    cvd, lib = _lib()
    v = C.c_double()
    b = C.c_uint32()
    assert lib.cvd_probe_latency(None, 1 << 20, 10, None, C.byref(v)) == EINVAL
    assert lib.cvd_probe_latency(C.c_void_p(0x1001), 1 << 20, 10, None, C.byref(v)) == EINVAL   # misaligned
    assert lib.cvd_probe_latency(C.c_void_p(0x1000), 128, 10, None, C.byref(v)) == EINVAL       # < 2 slots
    assert lib.cvd_probe_latency(C.c_void_p(0x1000), 1 << 20, 0, None, C.byref(v)) == EINVAL
    assert lib.cvd_selftest_wait_timeout(None, 0, C.byref(b)) == EINVAL
    assert lib.cvd_selftest_wait_timeout(None, (1 << 22) + 1, C.byref(b)) == EINVAL
    assert lib.cvd_selftest_wait_timeout(None, 16, None) == EINVAL


def test_every_status_has_a_message():
    cvd, lib = _lib()
    for code in (0, cvd.EINVAL, cvd.ENOMEM, cvd.ECUDA, cvd.ETIMEDOUT, cvd.EHAZARD, cvd.E2BIG, -9999):
        msg = lib.cvd_strerror(code)
        assert msg and len(msg.decode()) >= 2


def test_multi_batch_and_chained_calls_reject_bad_arguments_before_cuda():
    cvd, lib = _lib()
    g = (C.c_void_p * 1)(0x1234)
    gp = C.cast(g, C.c_void_p)
    b = cvd.DevBatch(0x1000, 1, 0, 0x2000, 1, 0x3000)
    # planned-ahead batches: flags must be exactly HAZARD_FREE; batches required
    assert lib.cvd_copy_batches(gp, 1, C.byref(b), 1, None, 0, 0, None) == EINVAL
    assert lib.cvd_copy_batches(gp, 1, C.byref(b), 1, None, 0, cvd.BATCH_HAZARD_FREE | cvd.BATCH_CHECK, None) == EINVAL
    assert lib.cvd_copy_batches(gp, 1, None, 2, None, 0, cvd.BATCH_HAZARD_FREE, None) == EINVAL
    # chained gathers: flags, missing buffers, a misaligned descriptor buffer, oversized payload
    assert lib.cvd_gather_chained(gp, 1, C.c_void_p(0x1000), 1, C.c_void_p(0x2000), 64, C.c_void_p(0x3000), 64,
                                  C.c_void_p(0x4000), cvd.BATCH_GRAPH, None) == EINVAL
    assert lib.cvd_gather_chained(gp, 1, None, 1, C.c_void_p(0x2000), 64, C.c_void_p(0x3000), 64,
                                  C.c_void_p(0x4000), 0, None) == EINVAL
    assert lib.cvd_gather_chained(gp, 1, C.c_void_p(0x1000), 1, C.c_void_p(0x2008), 64, C.c_void_p(0x3000), 64,
                                  C.c_void_p(0x4000), 0, None) == EINVAL
    assert lib.cvd_gather_chained(gp, 1, C.c_void_p(0x1000), 1, C.c_void_p(0x2000), 64, C.c_void_p(0x3000),
                                  1 << 52, C.c_void_p(0x4000), 0, None) == EINVAL
    assert lib.cvd_gather_chained(gp, 1, C.c_void_p(0x1000), 1, C.c_void_p(0x2000), 64, None, 64,
                                  C.c_void_p(0x4000), 0, None) == EINVAL
    # placement: no guest
    assert lib.cvd_mmap_place(None, 0, 4096, None, 0, None, 0, None, None, None) == EINVAL
