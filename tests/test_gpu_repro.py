"""A device guest saved to a repro file and re-created from it continues
exactly where the saved one stopped: after one mmap install call, a second
call on the re-created guest gives the oracle's statuses, pool bytes, p2m
and allocation counters (Sec. 4.2 insert_pfn takes PT-pool and reserved
frames in order), and its walks equal the saved guest's."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import repro
from paper_1304_3771_b300 import workload as W

pytestmark = pytest.mark.gpu


def test_guest_state_round_trip_continues_installs(tmp_path):
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(64 << 20, 521, np_frac=0.02, ro_frac=0.0)
    pool = W.materialize_pool(img)
    og = O.Guest.from_image(img, pool.copy())
    g = cvd.Guest.from_image(img, torch.from_numpy(pool.copy()).cuda())
    r1, hf1, _ = W.mmap_requests(img, 522, 200, max_pages=64, window_bytes=1 << 30)
    r2, hf2, _ = W.mmap_requests(img, 523, 200, max_pages=64, window_bytes=1 << 30, purpose=1)

    def install(guest, reqs, hf):
        npg = int(reqs["npages"].astype(np.int64).sum())
        st = torch.zeros(npg, dtype=torch.int32, device="cuda")
        guest.mmap_install(cvd.records_to_device(reqs), len(reqs), cvd.u64_to_device(hf), len(hf), st)
        torch.cuda.synchronize()
        return st.cpu().numpy()

    np.testing.assert_array_equal(install(g, r1, hf1), og.mmap_install(r1, hf1))
    path = tmp_path / "guest.npz"
    repro.save(path, g.state())
    st, _ = repro.load(path)
    assert (st.pt_used, st.rsv_used) == (og.pt_used, og.rsv_used) and og.rsv_used > 0
    g2 = cvd.Guest.from_state(st)
    assert g2.alloc_state() == (og.pt_used, og.rsv_used)
    gva = torch.from_numpy(W.translate_gvas(img, 524, 20000).view(np.int64)).cuda()
    for a, b in zip(g.translate(gva), g2.translate(gva)):
        assert torch.equal(a, b)
    np.testing.assert_array_equal(install(g2, r2, hf2), og.mmap_install(r2, hf2))
    assert np.array_equal(g2.pool.cpu().numpy(), og.pool)
    np.testing.assert_array_equal(cvd.u64_from_device(g2.p2m)[:img.rsv_n], og.p2m[:img.rsv_n])
    assert g2.alloc_state() == (og.pt_used, og.rsv_used)
    with pytest.raises(cvd.CvdError):
        g2.set_alloc_state(img.pt_pool_n + 1, 0)
    g.close()
    g2.close()
