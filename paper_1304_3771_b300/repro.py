"""Repro files: one guest's state saved with whatever requests reproduce a case.

A file holds the guest's host pool (page tables and data), its second
dimension (memslots, or the host-pool offset of its EPT), its cr3, the PT
pool and reserved window that installs take frames from (Sec. 4.2,
insert_pfn), the p2m array of that window, and the two allocation counters,
so a guest re-created from it walks, copies and installs exactly as the saved
one would have.  Any further named arrays (requests, segments, gVAs) travel
beside the state.  The format is a numpy ``.npz`` archive read without
pickle; ``Guest.state`` / ``Guest.from_state`` in the binding move a state
between a file and the device.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np

VERSION = 1
# the descriptor's scalars, in their order in the file's "desc" array
_FIELDS = ("cr3_gpa", "paging", "pt_pool_gfn", "pt_pool_n", "rsv_gfn", "rsv_n", "ept_root", "pt_used", "rsv_used")
_NONE = np.uint64(0xFFFFFFFFFFFFFFFF)   # ept_root of a memslot guest
_RESERVED = ("version", "pool", "slots", "desc", "p2m")


@dataclass
class GuestState:
    pool: np.ndarray                # uint8, the whole host pool
    slots: np.ndarray               # (n, 3) uint64: base_gfn, npages, host_off
    cr3_gpa: int
    paging: int = 0                 # 0: x86-64 4-level, 1: 32-bit PAE
    pt_pool_gfn: int = 0
    pt_pool_n: int = 0
    rsv_gfn: int = 0
    rsv_n: int = 0
    ept_root: Optional[int] = None  # host-pool offset of the EPT, or None (memslots)
    pt_used: int = 0                # PT-pool frames installs have taken
    rsv_used: int = 0               # reserved frames installs have taken
    p2m: Optional[np.ndarray] = None   # uint64 per reserved frame (all ones: unmapped)

    def check(self) -> None:
        """The consistency a guest descriptor needs (ValueError otherwise)."""
        if self.pool.dtype != np.uint8 or self.pool.ndim != 1:
            raise ValueError("pool must be a 1-D uint8 array")
        if self.slots.dtype != np.uint64 or self.slots.ndim != 2 or self.slots.shape[1] != 3:
            raise ValueError("slots must be an (n, 3) uint64 array")
        if self.paging not in (0, 1):
            raise ValueError("paging must be 0 (x86-64) or 1 (PAE)")
        if self.pt_used > self.pt_pool_n or self.rsv_used > self.rsv_n:
            raise ValueError("allocation counters pass their pools")
        if self.p2m is not None and (self.p2m.dtype != np.uint64 or len(self.p2m) < self.rsv_n):
            raise ValueError("p2m must be uint64 with an entry per reserved frame")

    def slot_records(self, dtype: np.dtype) -> np.ndarray:
        """The memslots as records of `dtype` (fields base_gfn, npages, host_off)."""
        out = np.zeros(len(self.slots), dtype=dtype)
        for k, name in enumerate(("base_gfn", "npages", "host_off")):
            out[name] = self.slots[:, k]
        return out


def state_from_image(img, pool: np.ndarray, p2m: Optional[np.ndarray] = None, pt_used: int = 0,
                     rsv_used: int = 0) -> GuestState:
    """A GuestState from a generated guest image and its pool (a copy of neither)."""
    slots = img.slots
    s = np.stack([slots["base_gfn"], slots["npages"], slots["host_off"]], axis=1).astype(np.uint64) \
        if len(slots) else np.zeros((0, 3), np.uint64)
    ept_root = getattr(img, "ept_root", None)
    return GuestState(pool=pool, slots=s if ept_root is None else s[:0], cr3_gpa=int(img.cr3_gpa),
                      paging=int(getattr(img, "paging", 0)),
                      pt_pool_gfn=int(img.pt_pool_gfn) if ept_root is None else 0,
                      pt_pool_n=int(img.pt_pool_n) if ept_root is None else 0,
                      rsv_gfn=int(img.rsv_gfn), rsv_n=int(img.rsv_n), ept_root=ept_root, pt_used=pt_used,
                      rsv_used=rsv_used, p2m=p2m)


def save(path, state: GuestState, **arrays: np.ndarray) -> None:
    """Write `state` and the named arrays (plain or structured dtypes) to `path`."""
    state.check()
    bad = set(arrays) & set(_RESERVED)
    if bad:
        raise ValueError(f"array names reserved by the format: {sorted(bad)}")
    desc = np.array([_NONE if (f == "ept_root" and state.ept_root is None) else getattr(state, f)
                     for f in _FIELDS], dtype=np.uint64)
    extra = {"p2m": state.p2m} if state.p2m is not None else {}
    with open(path, "wb") as fh:
        np.savez(fh, version=np.array([VERSION], np.uint64), pool=state.pool, slots=state.slots, desc=desc,
                 **extra, **arrays)


def load(path) -> tuple[GuestState, dict]:
    """Read a file written by `save`: (state, the other named arrays)."""
    with np.load(path, allow_pickle=False) as z:
        names = set(z.files)
        if "version" not in names or int(z["version"][0]) != VERSION:
            raise ValueError(f"{path}: not a version-{VERSION} repro file")
        desc = z["desc"]
        if len(desc) != len(_FIELDS):
            raise ValueError(f"{path}: descriptor has {len(desc)} fields, expected {len(_FIELDS)}")
        kv = {f: int(v) for f, v in zip(_FIELDS, desc)}
        if kv["ept_root"] == int(_NONE):
            kv["ept_root"] = None
        st = GuestState(pool=z["pool"], slots=z["slots"], p2m=z["p2m"] if "p2m" in names else None, **kv)
        arrays = {k: z[k] for k in names - set(_RESERVED)}
    st.check()
    return st, arrays
