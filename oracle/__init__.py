"""CPU oracle for the CVD memory operations -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``cvd_oracle.c`` (plain,
single-threaded C compiled with gcc) through ctypes; see that file for the
definitions it restates (Sec. 4.2 and Sec. 6.2-6.3 of the paper) and the
readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cvd_oracle.c")
_LIB = os.path.join(_HERE, "libcvd_oracle.so")

NO_FRAME = (1 << 64) - 1


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O2, no vectorisation tricks, single thread)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared", "-fPIC",
                               "-o", _LIB, _SRC])
    return _LIB


class OGuest(C.Structure):
    _fields_ = [("pool", C.c_void_p), ("pool_bytes", C.c_uint64),
                ("slots", C.c_void_p), ("nslots", C.c_uint32), ("paging", C.c_uint32),
                ("cr3_gpa", C.c_uint64),
                ("pt_pool_gfn", C.c_uint64), ("pt_pool_n", C.c_uint64), ("pt_used", C.c_uint64),
                ("rsv_gfn", C.c_uint64), ("rsv_n", C.c_uint64), ("rsv_used", C.c_uint64),
                ("p2m", C.c_void_p), ("ept", C.c_uint32), ("pad2", C.c_uint32), ("ept_root", C.c_uint64)]


_lib = None


def lib():
    """The compiled oracle; CVD_ORACLE_LIB names another build of it (the
    mutation check in ``mutants.py`` loads deliberately broken copies)."""
    global _lib
    if _lib is None:
        _lib = C.CDLL(os.environ.get("CVD_ORACLE_LIB") or build())
        _lib.oracle_walk.restype = C.c_uint32
        _lib.oracle_walk.argtypes = [C.POINTER(OGuest), C.c_uint64, C.c_int,
                                     C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
        _lib.oracle_translate.restype = None
        _lib.oracle_translate.argtypes = [C.POINTER(OGuest), C.c_void_p, C.c_uint64, C.c_int,
                                          C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.oracle_copy_batch.restype = C.c_int
        _lib.oracle_copy_batch.argtypes = [C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32,
                                           C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint64,
                                           C.c_void_p, C.c_int]
        _lib.oracle_mmap_install.restype = C.c_int
        _lib.oracle_mmap_install.argtypes = [C.POINTER(OGuest), C.c_void_p, C.c_uint32,
                                             C.c_void_p, C.c_uint64, C.c_void_p]
        _lib.oracle_gather_chained.restype = C.c_int
        _lib.oracle_gather_chained.argtypes = [C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint32, C.c_void_p,
                                               C.c_uint64, C.c_void_p, C.c_uint64, C.c_void_p]
        _lib.oracle_mmap_place.restype = C.c_int
        _lib.oracle_mmap_place.argtypes = [C.POINTER(OGuest), C.c_uint64, C.c_uint64, C.c_void_p, C.c_uint32,
                                           C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


class Guest:
    """Oracle view of one guest: a host pool (numpy uint8), memslots, cr3,
    PT pool, reserved window and p2m.  Keeps the numpy arrays alive."""

    def __init__(self, pool: np.ndarray, slots: np.ndarray, cr3_gpa: int, *, pt_pool_gfn=0,
                 pt_pool_n=0, rsv_gfn=0, rsv_n=0, p2m: np.ndarray | None = None, paging: int = 0,
                 ept_root: int | None = None):
        self.pool = pool
        self.slots = np.ascontiguousarray(slots)
        if p2m is None:
            p2m = np.full(max(rsv_n, 1), NO_FRAME, dtype=np.uint64)
        self.p2m = p2m
        self.s = OGuest(_ptr(pool), pool.nbytes, _ptr(self.slots), len(self.slots), paging, cr3_gpa,
                        pt_pool_gfn, pt_pool_n, 0, rsv_gfn, rsv_n, 0, _ptr(self.p2m),
                        0 if ept_root is None else 1, 0, 0 if ept_root is None else ept_root)

    @classmethod
    def from_image(cls, img, pool: np.ndarray, p2m: np.ndarray | None = None):
        return cls(pool, img.slots, img.cr3_gpa, pt_pool_gfn=img.pt_pool_gfn,
                   pt_pool_n=img.pt_pool_n, rsv_gfn=img.rsv_gfn, rsv_n=img.rsv_n, p2m=p2m,
                   paging=getattr(img, "paging", 0), ept_root=getattr(img, "ept_root", None))

    @property
    def pt_used(self):
        return self.s.pt_used

    @property
    def rsv_used(self):
        return self.s.rsv_used

    def walk(self, va: int, write: bool = False):
        gpa, hpa = C.c_uint64(), C.c_uint64()
        code = lib().oracle_walk(C.byref(self.s), va & NO_FRAME, int(write), C.byref(gpa), C.byref(hpa))
        return code, gpa.value, hpa.value

    def translate(self, va: np.ndarray, write: bool = False):
        va = np.ascontiguousarray(va, dtype=np.uint64)
        n = len(va)
        gpa = np.empty(n, np.uint64)
        hpa = np.empty(n, np.uint64)
        code = np.empty(n, np.uint32)
        lib().oracle_translate(C.byref(self.s), _ptr(va), n, int(write), _ptr(gpa), _ptr(hpa), _ptr(code))
        return gpa, hpa, code

    def mmap_install(self, reqs: np.ndarray, hf: np.ndarray):
        reqs = np.ascontiguousarray(reqs)
        hf = np.ascontiguousarray(hf, dtype=np.uint64)
        npg = int(reqs["npages"].astype(np.int64).sum()) if len(reqs) else 0
        status = np.zeros(max(npg, 1), np.int32)
        rc = lib().oracle_mmap_install(C.byref(self.s), _ptr(reqs), len(reqs), _ptr(hf), len(hf), _ptr(status))
        if rc != 0:
            raise RuntimeError(f"oracle_mmap_install failed: {rc}")
        return status[:npg]

    def mmap_place(self, va_lo: int, va_hi: int, reqs: np.ndarray, hf: np.ndarray):
        """Driver-initiated maps (Sec. 6.6): first-fit ranges in [va_lo, va_hi)
        for requests without an address, then the install.  Returns (gva per
        request, all ones for none; per-page status); raises ValueError when
        the call itself is refused (bad window)."""
        reqs = np.ascontiguousarray(reqs)
        hf = np.ascontiguousarray(hf, dtype=np.uint64)
        npg = int(reqs["npages"].astype(np.int64).sum()) if len(reqs) else 0
        status = np.zeros(max(npg, 1), np.int32)
        gva = np.zeros(max(len(reqs), 1), np.uint64)
        rc = lib().oracle_mmap_place(C.byref(self.s), va_lo, va_hi, _ptr(reqs), len(reqs), _ptr(hf), len(hf),
                                     _ptr(gva), _ptr(status))
        if rc == -22:
            raise ValueError("oracle_mmap_place: bad window")
        if rc != 0:
            raise RuntimeError(f"oracle_mmap_place failed: {rc}")
        return gva[:len(reqs)], status[:npg]


def gather_chained(guests, reqs: np.ndarray, desc: np.ndarray, payload: np.ndarray):
    """Dependent second-level gathers: every request's descriptor table into
    ``desc``, then the buffers it names into ``payload`` (both updated in
    place).  Returns CHAIN_RES records."""
    from paper_1304_3771_b300.workload import CHAIN_RES_DTYPE
    reqs = np.ascontiguousarray(reqs)
    res = np.zeros(max(len(reqs), 1), dtype=CHAIN_RES_DTYPE)
    arr = (C.POINTER(OGuest) * max(len(guests), 1))(*[C.pointer(g.s) for g in guests])
    rc = lib().oracle_gather_chained(C.cast(arr, C.c_void_p), len(guests), _ptr(reqs), len(reqs), _ptr(desc),
                                     desc.nbytes, _ptr(payload), payload.nbytes, _ptr(res))
    if rc != 0:
        raise MemoryError("oracle_gather_chained: out of host memory")
    return res[:len(reqs)]


def copy_batch(guests, reqs: np.ndarray, segs: np.ndarray, staging: np.ndarray, per_byte: bool = False):
    """Run one call's requests in index order; returns RESULT records.
    ``guests`` is a list of ``Guest``; ``staging`` (uint8) is updated in place,
    as are the guests' pools."""
    from paper_1304_3771_b300.workload import RESULT_DTYPE
    reqs = np.ascontiguousarray(reqs)
    segs = np.ascontiguousarray(segs)
    res = np.zeros(max(len(reqs), 1), dtype=RESULT_DTYPE)
    arr = (C.POINTER(OGuest) * max(len(guests), 1))(*[C.pointer(g.s) for g in guests])
    rc = lib().oracle_copy_batch(C.cast(arr, C.c_void_p), len(guests), _ptr(reqs), len(reqs), _ptr(segs),
                                 len(segs), _ptr(staging), staging.nbytes, _ptr(res), int(per_byte))
    if rc != 0:
        raise MemoryError("oracle_copy_batch: out of host memory")
    return res[:len(reqs)]
