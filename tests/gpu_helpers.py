"""Shared set-up for the GPU parity tests: the same seeded inputs go to the
oracle (numpy) and to the CUDA library (torch device tensors)."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1304_3771_b300 import workload as W


def device_guest(img, pool_np):
    import torch
    from paper_1304_3771_b300 import cvd
    pool_d = torch.from_numpy(pool_np.copy()).cuda()
    p2m = torch.full((max(img.rsv_n, 1),), -1, dtype=torch.int64, device="cuda")
    g = cvd.Guest.from_image(img, pool_d, p2m=p2m)
    return g, pool_d


def run_both(img, pool_np, reqs, segs, stg_np, flags=0, params=None, basic=None):
    """Run one call on the oracle and on the GPU; return both outcomes."""
    import torch
    from paper_1304_3771_b300 import cvd
    o_pool = pool_np.copy()
    o_stg = stg_np.copy()
    o_res = O.copy_batch([O.Guest.from_image(img, o_pool)], reqs, segs, o_stg)
    g, pool_d = device_guest(img, pool_np)
    req_d = cvd.records_to_device(reqs)
    seg_d = cvd.records_to_device(segs)
    stg_d = torch.from_numpy(stg_np.copy()).cuda()
    res_d = torch.zeros(max(len(reqs), 1) * W.RESULT_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    if params:
        cvd.set_copy_params(**params)
    if basic == "from":
        g.copy_from(req_d, len(reqs), seg_d, len(segs), stg_d, res_d)
    elif basic == "to":
        g.copy_to(req_d, len(reqs), seg_d, len(segs), stg_d, res_d)
    else:
        cvd.copy_batch([g], req_d, len(reqs), seg_d, len(segs), stg_d, res_d, flags=flags)
    torch.cuda.synchronize()
    g_res = cvd.records_from_device(res_d, W.RESULT_DTYPE, len(reqs))
    out = dict(o_res=o_res, o_pool=o_pool, o_stg=o_stg, g_res=g_res, g_pool=pool_d.cpu().numpy(),
               g_stg=stg_d.cpu().numpy())
    g.close()
    return out


def assert_same(out):
    np.testing.assert_array_equal(out["g_res"], out["o_res"])
    assert np.array_equal(out["g_stg"], out["o_stg"]), "staging bytes differ"
    assert np.array_equal(out["g_pool"], out["o_pool"]), "guest memory differs"
