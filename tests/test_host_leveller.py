"""The levelled calls' byte-exact host leveller (cvd_level_runs, no CUDA
call) against its definition written out by brute force: a run's level is 1
+ the highest level of an earlier run sharing a byte with it, one of the two
writing it (0 when none); the marked runs are those with a range in a
cluster of overlapping ranges that holds two or more ranges and a writer.
Executing the levels in order then gives the sequential result, checked on
bytes for small cases."""
import numpy as np
import pytest

from paper_1304_3771_b300 import cvd


def _ranges(r):
    out = []
    if r["len"]:
        out.append((int(r["dst"]), int(r["dst"]) + int(r["len"]), 1))
        if r["src"]:
            out.append((int(r["src"]), int(r["src"]) + int(r["len"]), 0))
    return out


def _brute_levels(runs):
    rs = [_ranges(r) for r in runs]
    lev = []
    for i, ri in enumerate(rs):
        L = 0
        for j in range(i):
            if any(a < d and c < b and (w or x) for a, b, w in ri for c, d, x in rs[j]):
                L = max(L, lev[j] + 1)
        lev.append(L)
    return lev


def _brute_marked(runs):
    iv = sorted(((a, b, w, i) for i, r in enumerate(runs) for a, b, w in _ranges(r)), key=lambda t: t[0])
    marked, k = set(), 0
    while k < len(iv):
        end, m, w = iv[k][1], k + 1, iv[k][2]
        while m < len(iv) and iv[m][0] < end:
            end, w = max(end, iv[m][1]), w | iv[m][2]
            m += 1
        if m - k >= 2 and w:
            marked.update(t[3] for t in iv[k:m])
        k = m
    return len(marked)


def _random_runs(rng, n, span, maxlen, zero_frac=0.2):
    runs = np.zeros(n, dtype=cvd.RUN_DTYPE)
    # two disjoint windows, as staging and guest memory are: dst and src each in either
    base = np.array([1 << 20, 1 << 30], dtype=np.uint64)
    runs["len"] = rng.integers(0, maxlen + 1, n)
    runs["dst"] = base[rng.integers(0, 2, n)] + rng.integers(0, span, n).astype(np.uint64)
    src = base[rng.integers(0, 2, n)] + rng.integers(0, span, n).astype(np.uint64)
    runs["src"] = np.where(rng.random(n) < zero_frac, 0, src)
    return runs


@pytest.mark.parametrize("seed,n,span,maxlen", [(1, 40, 400, 40), (2, 200, 5000, 64), (3, 300, 100000, 4096),
                                                 (4, 120, 64, 16), (5, 1, 10, 10)])
def test_levels_and_marks_equal_the_definition(seed, n, span, maxlen):
    runs = _random_runs(np.random.default_rng(seed), n, span, maxlen)
    lev, top, marked = cvd.level_runs(runs)
    want = _brute_levels(runs)
    assert lev.tolist() == want
    assert top == max(want)
    assert marked == _brute_marked(runs)


def _loc(addr):
    base = (1 << 30) if addr >= (1 << 30) else (1 << 20)
    return base, addr - base


def _apply(r, dst_mem, src_mem):
    """One run: len bytes from src (or zeros) to dst."""
    L = int(r["len"])
    if not L:
        return
    db, od = _loc(int(r["dst"]))
    if r["src"]:
        sb, os_ = _loc(int(r["src"]))
        dst_mem[db][od:od + L] = src_mem[sb][os_:os_ + L]
    else:
        dst_mem[db][od:od + L] = 0


def test_levels_run_in_order_give_the_sequential_bytes():
    rng = np.random.default_rng(7)
    runs = _random_runs(rng, 150, 3000, 80)
    mem0 = {b: rng.integers(0, 256, 3100, dtype=np.uint8) for b in (1 << 20, 1 << 30)}
    seq = {b: m.copy() for b, m in mem0.items()}
    for r in runs:
        _apply(r, seq, {b: m.copy() for b, m in seq.items()})
    lev, top, _ = cvd.level_runs(runs)
    par = {b: m.copy() for b, m in mem0.items()}
    for level in range(top + 1):
        snap = {b: m.copy() for b, m in par.items()}   # a level's runs all read memory as it was before the level
        for i in np.nonzero(lev == level)[0]:
            _apply(runs[i], par, snap)
    for b in mem0:
        assert np.array_equal(par[b], seq[b])


def test_bad_arguments():
    runs = np.zeros(1, dtype=cvd.RUN_DTYPE)
    runs["dst"] = np.uint64(2**64 - 8)
    runs["len"] = 16
    with pytest.raises(cvd.CvdError):
        cvd.level_runs(runs)
    lev, top, marked = cvd.level_runs(np.zeros(0, dtype=cvd.RUN_DTYPE))
    assert len(lev) == 0 and top == 0 and marked == 0
