"""Repro files (guest state dump and reload): a saved guest, re-created from
its file, walks, copies and installs exactly as the saved one would have
(the oracle runs both sides; Sec. 4.2 installs take PT-pool and reserved
frames in order, so the allocation counters must travel too)."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import repro
from paper_1304_3771_b300 import workload as W


def _oracle_guest(st: repro.GuestState) -> O.Guest:
    g = O.Guest(st.pool, st.slot_records(W.SLOT_DTYPE), st.cr3_gpa, pt_pool_gfn=st.pt_pool_gfn,
                pt_pool_n=st.pt_pool_n, rsv_gfn=st.rsv_gfn, rsv_n=st.rsv_n,
                p2m=st.p2m if st.p2m is not None else None, paging=st.paging, ept_root=st.ept_root)
    g.s.pt_used = st.pt_used
    g.s.rsv_used = st.rsv_used
    return g


def test_round_trip_keeps_every_field_and_array(tmp_path):
    img = W.make_guest(32 << 20, 501, np_frac=0.05, ro_frac=0.05)
    pool = W.materialize_pool(img)
    p2m = np.arange(img.rsv_n, dtype=np.uint64) * 3
    st = repro.state_from_image(img, pool, p2m=p2m, pt_used=2, rsv_used=7)
    wl = W.tiny_requests(img, 502, nreq=50)
    path = tmp_path / "case.npz"
    repro.save(path, st, reqs=wl.reqs, segs=wl.segs, gva=np.arange(5, dtype=np.uint64))
    got, arrays = repro.load(path)
    for f in ("cr3_gpa", "paging", "pt_pool_gfn", "pt_pool_n", "rsv_gfn", "rsv_n", "ept_root", "pt_used",
              "rsv_used"):
        assert getattr(got, f) == getattr(st, f), f
    assert np.array_equal(got.pool, pool) and np.array_equal(got.slots, st.slots)
    assert np.array_equal(got.p2m, p2m)
    assert got.ept_root is None
    assert set(arrays) == {"reqs", "segs", "gva"}
    assert arrays["reqs"].dtype == W.REQ_DTYPE and np.array_equal(arrays["reqs"], wl.reqs)
    assert arrays["segs"].dtype == W.SEG_DTYPE and np.array_equal(arrays["segs"], wl.segs)
    assert np.array_equal(got.slot_records(W.SLOT_DTYPE), img.slots)


def test_reloaded_guest_walks_and_copies_like_the_saved_one(tmp_path):
    img = W.make_guest(32 << 20, 503, np_frac=0.05, ro_frac=0.05)
    pool = W.materialize_pool(img)
    wl = W.tiny_requests(img, 504, nreq=200)
    path = tmp_path / "case.npz"
    repro.save(path, repro.state_from_image(img, pool), reqs=wl.reqs, segs=wl.segs)
    st, arrays = repro.load(path)
    a, b = O.Guest.from_image(img, pool.copy()), _oracle_guest(st)
    gva = W.translate_gvas(img, 505, 4000)
    for write in (False, True):
        for x, y in zip(a.translate(gva, write), b.translate(gva, write)):
            assert np.array_equal(x, y)
    nbytes = int(wl.reqs["host_off"].max() + 2 * 65536 * 8)
    sa, sb = W.payload_bytes(506, nbytes), W.payload_bytes(506, nbytes)
    ra = O.copy_batch([a], wl.reqs, wl.segs, sa)
    rb = O.copy_batch([b], arrays["reqs"], arrays["segs"], sb)
    assert np.array_equal(ra, rb) and np.array_equal(sa, sb) and np.array_equal(a.pool, b.pool)


def test_installs_continue_from_the_saved_counters(tmp_path):
    """Install a batch, save, reload, install a second batch on both sides:
    statuses, p2m and every pool byte agree; a reload that dropped the
    counters would hand out the same frames again."""
    img = W.make_guest(32 << 20, 507, np_frac=0.0, ro_frac=0.0)
    a = O.Guest.from_image(img, W.materialize_pool(img))
    r1, hf1, _ = W.mmap_requests(img, 508, 30, max_pages=64, window_bytes=256 << 20)
    a.mmap_install(r1, hf1)
    assert a.pt_used > 0 and a.rsv_used > 0
    st = repro.state_from_image(img, a.pool.copy(), p2m=a.p2m.copy(), pt_used=a.pt_used, rsv_used=a.rsv_used)
    path = tmp_path / "after_first.npz"
    repro.save(path, st)
    loaded, _ = repro.load(path)
    b = _oracle_guest(loaded)
    fresh = _oracle_guest(repro.GuestState(**{**loaded.__dict__, "pool": loaded.pool.copy(),
                                              "p2m": loaded.p2m.copy(), "pt_used": 0, "rsv_used": 0}))
    r2, hf2, _ = W.mmap_requests(img, 509, 30, max_pages=64, window_bytes=256 << 20, purpose=1)
    sa, sb, sf = a.mmap_install(r2, hf2), b.mmap_install(r2, hf2), fresh.mmap_install(r2, hf2)
    assert np.array_equal(sa, sb)
    assert np.array_equal(a.pool, b.pool) and np.array_equal(a.p2m, b.p2m)
    assert (a.pt_used, a.rsv_used) == (b.pt_used, b.rsv_used)
    assert not np.array_equal(a.p2m, fresh.p2m)


def test_ept_guest_round_trip(tmp_path):
    img = W.add_ept(W.make_guest(32 << 20, 511, np_frac=0.0, ro_frac=0.0), 512)
    pool = W.materialize_pool(img)
    path = tmp_path / "ept.npz"
    repro.save(path, repro.state_from_image(img, pool))
    st, _ = repro.load(path)
    assert st.ept_root == img.ept_root and len(st.slots) == 0
    gva = W.translate_gvas(img, 513, 2000)
    for x, y in zip(O.Guest.from_image(img, pool).translate(gva), _oracle_guest(st).translate(gva)):
        assert np.array_equal(x, y)


def test_bad_files_and_states_are_refused(tmp_path):
    img = W.make_guest(16 << 20, 515, np_frac=0.0, ro_frac=0.0)
    pool = W.materialize_pool(img)
    st = repro.state_from_image(img, pool)
    with pytest.raises(ValueError):
        repro.save(tmp_path / "x.npz", st, pool=np.zeros(1, np.uint8))    # a reserved name
    with pytest.raises(ValueError):
        repro.save(tmp_path / "x.npz", repro.GuestState(**{**st.__dict__, "pt_used": st.pt_pool_n + 1}))
    with pytest.raises(ValueError):
        repro.save(tmp_path / "x.npz", repro.GuestState(**{**st.__dict__, "paging": 2}))
    np.savez(tmp_path / "old.npz", version=np.array([99], np.uint64), pool=pool)
    with pytest.raises(ValueError):
        repro.load(tmp_path / "old.npz")
