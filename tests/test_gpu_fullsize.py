"""Parity at the full workload sizes, compared exhaustively.

* Batching (16 GiB guest, 1,000,000 requests in 6 hazard-free batches,
  58.8 GB payload) and frames (32 GiB guest, 4 KiB pages permuted, 4,096
  page-aligned frames of 8,294,400 or 33,177,600 B, 85 GB payload): the
  oracle runs every batch in order on a host copy of the initial guest pool
  and staging buffer.  The GPU runs the same batches twice from the same
  initial state: once as the step bench.py times (one planned-ahead
  cvd_copy_batches call over all batches), once as one hazard-free
  cvd_copy_batch call per batch in lockstep with the oracle.  Every result
  of every batch is compared, and after every batch of the lockstep run and
  at the end of the planned-ahead run the whole staging buffer and the whole
  guest pool are compared byte for byte, streamed to the device in 1 GiB
  chunks (staging ranges are reused by every batch, so a wrong byte that a
  later batch overwrites is still caught).
* Translation (8 GiB guest, 2^26 gVAs): every output compared.
* mmap install (8 GiB guest, 10,000 requests, 2.55 M pages): every page
  status, the whole p2m array and every page-table frame compared."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W
from tests.fullsize_helpers import exhaustive_batches, table_shadow, upload_guest

pytestmark = pytest.mark.gpu

SEED = W.DEFAULT_SEED


def test_batching_full_size_every_batch_every_byte():
    import torch
    img = W.make_guest(16 << 30, SEED, huge_frac=0.7, np_frac=0.0, ro_frac=0.0, nslots=4, slot_gap_pages=512)
    wl = W.batched_requests(img, SEED, W.batching_sizes(SEED, 1_000_000), 32)
    assert len(wl.batches) == 6
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1)
    assert exhaustive_batches(img, wl, gen) == 1_000_000


def test_frames_full_size_every_batch_every_byte():
    import torch
    seed = SEED + 4
    img = W.make_guest(32 << 30, seed, np_frac=0.0, ro_frac=0.0)
    wl = W.batched_requests(img, seed, W.frame_sizes(seed, 4096), 1, page_aligned=True)
    assert (wl.reqs["seg_count"] == 1).all() and img.pool_bytes % 4096 == 0 and len(wl.batches) >= 3
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    assert exhaustive_batches(img, wl, gen) == 4096


def test_translate_full_size_all_outputs():
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(8 << 30, SEED + 3, np_frac=0.05, ro_frac=0.05)
    gen = torch.Generator(device="cuda")
    g, pool_d = upload_guest(img, gen, fill=False)
    gva = W.translate_gvas(img, SEED + 3, 1 << 26)
    out = g.translate(cvd.u64_to_device(gva))
    torch.cuda.synchronize()
    og = O.Guest.from_image(img, table_shadow(img))
    for write in (False,):
        exp = og.translate(gva, write)
        np.testing.assert_array_equal(cvd.u64_from_device(out[0]), exp[0])
        np.testing.assert_array_equal(cvd.u64_from_device(out[1]), exp[1])
        np.testing.assert_array_equal(out[2].cpu().numpy().view(np.uint32), exp[2])
    g.close()


def test_mmap_full_size_all_outputs():
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(8 << 30, SEED + 3, np_frac=0.05, ro_frac=0.05, pt_pool_n=40000, rsv_n=3 << 20)
    reqs, hf, _ = W.mmap_requests(img, SEED + 3, 10000)
    npg = int(reqs["npages"].astype(np.int64).sum())
    gen = torch.Generator(device="cuda")
    g, pool_d = upload_guest(img, gen, fill=False)
    st = torch.zeros(npg, dtype=torch.int32, device="cuda")
    g.mmap_install(cvd.records_to_device(reqs), len(reqs), cvd.u64_to_device(hf), len(hf), st)
    shadow = table_shadow(img)
    og = O.Guest.from_image(img, shadow)
    o_st = og.mmap_install(reqs, hf)
    np.testing.assert_array_equal(st.cpu().numpy(), o_st)
    np.testing.assert_array_equal(cvd.u64_from_device(g.p2m), og.p2m)
    assert g.alloc_state() == (og.pt_used, og.rsv_used)
    # every table frame: the generator's tables and the PT pool
    frames = sorted(set(img.tables) | set(range(img.pt_pool_gfn, img.pt_pool_gfn + img.pt_pool_n)))
    host = np.array([img.gpa_to_host(f << 12) for f in frames], dtype=np.int64)
    runs = np.split(host, np.nonzero(np.diff(host) != 4096)[0] + 1)
    for run in runs:
        a, b = int(run[0]), int(run[-1]) + 4096
        assert np.array_equal(pool_d[a:b].cpu().numpy(), shadow[a:b]), hex(a)
    assert (o_st == 0).sum() > 1_000_000
    g.close()
