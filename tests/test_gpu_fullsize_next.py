"""Parity at the measured sizes of the rows beyond the base path, in the
launch configuration bench.py times.

* Software EPT and PAE guests (2 GiB guests of the ept / pae arms, 2^26
  gVAs): every translation output compared with the oracle.
* The batching mix on the same EPT and PAE guests (200,000 requests in
  hazard-free batches): every batch on the oracle beside the GPU (planned-
  ahead and per-batch), every result, the whole staging buffer and guest
  pool compared after every batch (tests/fullsize_helpers.py).
* Chained gathers (8 GiB guest, 50,000 descriptor tables, 7.75 GB payload):
  the whole call on the oracle from a copy of the initial pool; every
  result, the whole descriptor and payload buffers and the pool compared.
* Driver-initiated maps (the place arm: 64 GiB window fragmented by 2,000
  installs, 10,000 requests): the GPU result is checked against properties
  that hold at any size -- every range inside the window, ranges pairwise
  disjoint and clear of the fragmenting installs, every page installed and
  translating to its host frame (sampled), and first fit for a sample of
  requests against the exact free map below their range.  The oracle itself
  runs the same call on smaller windows in test_gpu_place.py."""
import numpy as np
import pytest

import oracle as O
from paper_1304_3771_b300 import workload as W
from tests.fullsize_helpers import assert_equal_streamed, exhaustive_batches, to_host_pinned

pytestmark = pytest.mark.gpu

SEED = W.DEFAULT_SEED


def _upload(img, fill_seed=None):
    import torch
    from paper_1304_3771_b300 import cvd
    pool = torch.zeros(img.pool_bytes, dtype=torch.uint8, device="cuda")
    if fill_seed is not None:
        gen = torch.Generator(device="cuda")
        gen.manual_seed(fill_seed)
        n = pool.numel()
        for a in range(0, n, 1 << 30):
            b = min(n, a + (1 << 30))
            pool[a:b] = torch.randint(0, 256, (b - a,), dtype=torch.uint8, device="cuda", generator=gen)
    offs, data = W.table_blob(img)
    idx = torch.from_numpy((offs[:, None] + np.arange(4096)[None, :]).reshape(-1)).cuda()
    pool[idx] = torch.from_numpy(data.reshape(-1)).cuda()
    p2m = torch.full((max(img.rsv_n, 1),), -1, dtype=torch.int64, device="cuda")
    return cvd.Guest.from_image(img, pool, p2m=p2m), pool, p2m


def _shadow(img):
    pool = np.zeros(img.pool_bytes, dtype=np.uint8)
    W.write_tables(img, pool)
    return pool


def _arm_image(kind):
    """The 2 GiB guest of the ept or pae arm, and its seed."""
    if kind == "ept":
        img0 = W.make_guest(2 << 30, SEED + 12, huge_frac=0.3, np_frac=0.0, ro_frac=0.0, nslots=4,
                            slot_gap_pages=512, host_base=2 << 20)
        return W.add_ept(img0, SEED + 12, huge_frac=0.5), SEED + 12
    return W.make_guest(2 << 30, SEED + 8, paging="pae", huge_frac=0.3, np_frac=0.0, ro_frac=0.0, nslots=4,
                        slot_gap_pages=512), SEED + 8


@pytest.mark.parametrize("kind", ["ept", "pae"])
def test_translate_bench_size_ept_and_pae(kind):
    import torch
    from paper_1304_3771_b300 import cvd
    img, _ = _arm_image(kind)
    g, pool, _ = _upload(img)
    gva = W.translate_gvas(img, SEED + 12, 1 << 26)
    out = g.translate(cvd.u64_to_device(gva), write=True)
    torch.cuda.synchronize()
    exp = O.Guest.from_image(img, _shadow(img)).translate(gva, True)
    np.testing.assert_array_equal(out[2].cpu().numpy().view(np.uint32), exp[2])
    np.testing.assert_array_equal(cvd.u64_from_device(out[0]), exp[0])
    np.testing.assert_array_equal(cvd.u64_from_device(out[1]), exp[1])
    assert (exp[2] == 0).sum() > (1 << 24)
    g.close()


@pytest.mark.parametrize("kind", ["ept", "pae"])
def test_batching_bench_size_ept_and_pae_every_batch_every_byte(kind):
    import torch
    img, seed = _arm_image(kind)
    wl = W.batched_requests(img, seed, W.batching_sizes(seed, 200_000), 32)
    assert len(wl.batches) >= 5
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed + 2)
    assert exhaustive_batches(img, wl, gen) == 200_000


def test_chain_bench_size_every_byte():
    """The whole 50,000-request call on the oracle from a pinned copy of the
    guest pool: every result, the whole descriptor buffer and the whole
    payload buffer compared."""
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(8 << 30, SEED + 15, huge_frac=0.7, np_frac=0.0, ro_frac=0.0, nslots=4, slot_gap_pages=512)
    wl = W.chained_requests(img, SEED + 15, 50_000)
    g, pool, _ = _upload(img, fill_seed=5)
    offs = W.host_of_gva_array(img, wl.entry_gvas())
    idx = torch.from_numpy((offs[:, None] + np.arange(16)[None, :]).reshape(-1)).cuda()
    pool[idx] = torch.from_numpy(wl.entries.reshape(-1).view(np.uint8)).cuda()
    del idx
    pool_ht, pool_h = to_host_pinned(pool)
    desc = torch.full((wl.desc_bytes,), 0xEE, dtype=torch.uint8, device="cuda")
    pay = torch.full((wl.payload_bytes,), 0xEE, dtype=torch.uint8, device="cuda")
    res = torch.zeros(len(wl.reqs) * W.CHAIN_RES_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    cvd.gather_chained([g], cvd.records_to_device(wl.reqs), len(wl.reqs), desc, pay, res,
                       flags=cvd.BATCH_HAZARD_FREE)
    torch.cuda.synchronize()
    assert cvd.stream_check() == 0
    g_res = cvd.records_from_device(res, W.CHAIN_RES_DTYPE, len(wl.reqs))
    og = O.Guest.from_image(img, pool_h)
    o_desc = np.full(wl.desc_bytes, 0xEE, np.uint8)
    o_pay_t = torch.full((wl.payload_bytes,), 0xEE, dtype=torch.uint8, pin_memory=True)
    o_res = O.gather_chained([og], wl.reqs, o_desc, o_pay_t.numpy())
    np.testing.assert_array_equal(g_res, o_res)
    L = np.add.reduceat(wl.entries[:, 1].astype(np.int64), wl.first[:-1])
    assert (o_res["level"] == 0).all() and (o_res["payload_len"] == L.astype(np.uint64)).all()
    assert np.array_equal(desc.cpu().numpy(), o_desc)
    assert_equal_streamed(pay, o_pay_t, "payload buffer")
    assert_equal_streamed(pool, pool_ht, "guest pool")        # gathers never write guest memory
    g.close()


def test_place_bench_size_properties():
    import torch
    from paper_1304_3771_b300 import cvd
    img = W.make_guest(8 << 30, SEED + 3, np_frac=0.05, ro_frac=0.05, pt_pool_n=60000, rsv_n=3 << 20)
    frag, fhf, win = W.mmap_requests(img, SEED + 13, 2000, max_pages=64, window_bytes=16 << 30, busy_frac=0.0)
    reqs, hf = W.place_requests(img, SEED + 14, 10000)
    g, pool, p2m = _upload(img)
    fst = torch.zeros(int(frag["npages"].astype(np.int64).sum()), dtype=torch.int32, device="cuda")
    g.mmap_install(cvd.records_to_device(frag), len(frag), cvd.u64_to_device(fhf), len(fhf), fst)
    # the free map of the window's first 16 GiB before the call: the fragmenting installs take their pages
    npg_w = (16 << 30) // 4096
    taken = np.zeros(npg_w, dtype=bool)
    ok = fst.cpu().numpy() == 0
    off = 0
    for q in frag:
        k = int(q["npages"])
        p0 = (int(q["gva"]) - win) // 4096
        taken[p0:p0 + k] |= ok[off:off + k]
        off += k
    npg = int(reqs["npages"].astype(np.int64).sum())
    st = torch.zeros(npg, dtype=torch.int32, device="cuda")
    gva = torch.zeros(len(reqs), dtype=torch.int64, device="cuda")
    g.mmap_place(win, win + (64 << 30), cvd.records_to_device(reqs), len(reqs), cvd.u64_to_device(hf), len(hf),
                 gva, st)
    torch.cuda.synchronize()
    gv = cvd.u64_from_device(gva)
    assert (st.cpu().numpy() == 0).all() and (gv != O.NO_FRAME).all()
    start = (gv.astype(np.int64) - win) // 4096
    n = reqs["npages"].astype(np.int64)
    assert (gv % 4096 == 0).all() and (start >= 0).all() and (start + n <= (64 << 30) // 4096).all()
    order = np.argsort(start)
    assert (start[order][1:] >= (start + n)[order][:-1]).all(), "ranges overlap"
    # clear of the fragmenting installs; first fit for a sample against the exact free map
    used = taken.copy()
    for r in range(len(reqs)):
        a, k = int(start[r]), int(n[r])
        if a < npg_w:
            assert not used[a:min(a + k, npg_w)].any(), r
        if r % 97 == 0:   # no lower start fits: every earlier run of free pages is shorter than k
            free = ~used[:min(a, npg_w)]
            if len(free):
                edges = np.flatnonzero(np.diff(np.concatenate([[0], free.astype(np.int8), [0]])))
                assert ((edges[1::2] - edges[0::2]) < k).all(), r
        used[a:min(a + k, npg_w)] = True
    # translation after the install: a sample of pages reaches its host frame
    og_pool = np.zeros(img.pool_bytes, dtype=np.uint8)
    frames = sorted(set(img.tables) | set(range(img.pt_pool_gfn, img.pt_pool_gfn + img.pt_pool_n)))
    host = np.array([img.gpa_to_host(f << 12) for f in frames], dtype=np.int64)
    for run in np.split(host, np.nonzero(np.diff(host) != 4096)[0] + 1):   # every table frame, as the GPU left it
        a, b = int(run[0]), int(run[-1]) + 4096
        og_pool[a:b] = pool[a:b].cpu().numpy()
    og = O.Guest.from_image(img, og_pool, p2m=cvd.u64_from_device(p2m).copy())
    hf_off = reqs["hf_begin"].astype(np.int64)
    rng = np.random.default_rng(4)
    for r in rng.choice(len(reqs), 200, replace=False):
        k = int(rng.integers(0, n[r]))
        code, _, hpa = og.walk(int(gv[r]) + 4096 * k + 7)
        assert code == 0 and hpa == int(hf[hf_off[r] + k]) * 4096 + 7, r
    g.close()
