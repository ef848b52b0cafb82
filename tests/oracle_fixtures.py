"""Helpers shared by the tests: parse the hand-written golden fixtures and build
small guests.  Nothing here computes a walk, a copy or an install."""
from __future__ import annotations

import os

import numpy as np

from paper_1304_3771_b300 import workload as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
ALL_ONES = (1 << 64) - 1


def _int(tok: str) -> int:
    return int(tok, 0)


def parse_golden(name: str) -> dict:
    out = {"slots": [], "entries": [], "cases": [], "maps": [], "expect": [], "p2m": [], "hentries": [],
           "p2m_set": []}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            t = line.split()
            k = t[0]
            if k == "slot":
                out["slots"].append(tuple(_int(x) for x in t[1:4]))
            elif k in ("pool", "cr3", "paging", "ept_root"):
                out[k] = _int(t[1])
            elif k == "ptpool":
                out["ptpool"] = (_int(t[1]), _int(t[2]))
            elif k == "rsv":
                out["rsv"] = (_int(t[1]), _int(t[2]))
            elif k == "entry" or k == "expect":
                out["entries" if k == "entry" else "expect"].append(
                    (_int(t[1]), _int(t[2]), _int(t[3])))
            elif k == "case":
                gpa = ALL_ONES if t[4] == "-" else _int(t[4])
                hpa = ALL_ONES if t[5] == "-" else _int(t[5])
                out["cases"].append((_int(t[1]), _int(t[2]), _int(t[3]), gpa, hpa))
            elif k == "map":
                out["maps"].append((_int(t[1]), _int(t[2]), _int(t[3]), [_int(x) for x in t[4:]]))
            elif k == "status":
                out["status"] = [_int(x) for x in t[1:]]
            elif k == "p2m" or k == "p2m_set":
                out[k].append((_int(t[1]), _int(t[2])))
            elif k == "hentry":
                out["hentries"].append((_int(t[1]), _int(t[2]), _int(t[3])))
            elif k == "used":
                out["used"] = (_int(t[1]), _int(t[2]))
            else:
                raise ValueError(line)
    return out


def golden_pool(g: dict) -> tuple[np.ndarray, np.ndarray]:
    """Host pool image with the golden entries written little-endian: `entry`
    lines at a guest frame of the first memslot, `hentry` lines at a host-pool
    byte offset."""
    pool = np.zeros(g["pool"], dtype=np.uint8)
    slots = np.array(g["slots"], dtype=W.SLOT_DTYPE)
    for gfn, idx, e in g["entries"]:
        base, n, host = g["slots"][0]
        assert base <= gfn < base + n
        off = host + (gfn - base) * 4096 + idx * 8
        pool[off:off + 8] = np.frombuffer(int(e).to_bytes(8, "little"), dtype=np.uint8)
    for hoff, idx, e in g["hentries"]:
        assert hoff % 4096 == 0 and hoff + 4096 <= len(pool)
        off = hoff + idx * 8
        pool[off:off + 8] = np.frombuffer(int(e).to_bytes(8, "little"), dtype=np.uint8)
    return pool, slots


def golden_maps(g: dict):
    maps = g["maps"]
    reqs = np.zeros(len(maps), dtype=W.MAPREQ_DTYPE)
    hf = []
    for i, (gva, npg, flags, frames) in enumerate(maps):
        assert len(frames) == npg
        reqs[i] = (gva, npg, flags, len(hf))
        hf.extend(frames)
    return reqs, np.array(hf, dtype=np.uint64)


def read_entries(pool: np.ndarray, host_of_gfn, gfns) -> dict:
    """{(gfn, idx): entry} for every non-zero entry of the given table frames."""
    out = {}
    for gfn in gfns:
        h = host_of_gfn(gfn)
        t = pool[h:h + 4096].view(np.uint64)
        for idx in np.nonzero(t)[0]:
            out[(gfn, int(idx))] = int(t[idx])
    return out


def identity_guest(npages: int, base_gva: int = 1 << 30, host_off: int = 0x5000, flags=7):
    """gVA page base_gva/4096 + i -> gfn i (closed form gpa = gva - base_gva)."""
    F = npages + 64
    F = ((F + 511) // 512) * 512
    vpn = (base_gva >> 12) + np.arange(npages)
    leaves = (vpn, (np.arange(npages, dtype=np.uint64) << np.uint64(12)) | np.uint64(flags))
    cr3, tables, low = W.build_tables(F - 1, leaves)
    assert low > npages
    slots = np.array([(0, F, host_off)], dtype=W.SLOT_DTYPE)
    pool = np.zeros(host_off + F * 4096 + 4096, dtype=np.uint8)
    pool[host_off:host_off + npages * 4096] = W.payload_bytes(7, npages * 4096)
    for gfn, t in tables.items():
        pool[host_off + gfn * 4096: host_off + gfn * 4096 + 4096] = t.view(np.uint8)
    return pool, slots, cr3
