"""ctypes binding of libcvd.so (the C ABI in include/cvd.h).

Argument marshalling only: every step of translation, planning, copying and
installing runs in the library's CUDA kernels.  PyTorch provides device
memory and streams.  There is no CPU fallback: if the library is missing,
loading it fails loudly.

Record arrays (requests, segments, results, map requests, memslots) are numpy
structured arrays with the dtypes of ``paper_1304_3771_b300.workload``; on the
device they live in torch ``uint8`` tensors holding the same bytes.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import workload as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcvd.so")

OK = 0
EINVAL, ENOMEM, ECUDA, ETIMEDOUT, EHAZARD, E2BIG = -22, -12, -5, -110, -11, -7
SECOND_MEMSLOTS, SECOND_EPT = 0, 1
BATCH_HAZARD_FREE, BATCH_GRAPH, BATCH_CHECK = 1, 2, 4

# Every function the header declares, with (restype, argtypes).
_vp, _u32, _u64 = C.c_void_p, C.c_uint32, C.c_uint64
SIGNATURES = {
    "cvd_guest_create": (C.c_int, [_vp, _vp]),
    "cvd_guest_destroy": (C.c_int, [_vp]),
    "cvd_guest_alloc_state": (C.c_int, [_vp, _vp, _vp]),
    "cvd_guest_set_alloc_state": (C.c_int, [_vp, C.c_uint64, C.c_uint64]),
    "cvd_level_runs": (C.c_int, [_vp, C.c_uint64, _vp, _vp]),
    "cvd_translate": (C.c_int, [_vp, _vp, _u64, _u32, _vp, _vp, _vp, _vp]),
    "cvd_copy_from_guest": (C.c_int, [_vp, _vp, _u32, _vp, _u64, _vp, _u64, _vp, _vp]),
    "cvd_copy_to_guest": (C.c_int, [_vp, _vp, _u32, _vp, _u64, _vp, _u64, _vp, _vp]),
    "cvd_mmap_install": (C.c_int, [_vp, _vp, _u32, _vp, _u64, _vp, _vp]),
    "cvd_mmap_place": (C.c_int, [_vp, _u64, _u64, _vp, _u32, _vp, _u64, _vp, _vp, _vp]),
    "cvd_gather_chained": (C.c_int, [_vp, _u32, _vp, _u32, _vp, _u64, _vp, _u64, _vp, _u32, _vp]),
    "cvd_copy_batches": (C.c_int, [_vp, _u32, _vp, _u32, _vp, _u64, _u32, _vp]),
    "cvd_copy_batch": (C.c_int, [_vp, _u32, _vp, _u32, _vp, _u64, _vp, _u64, _vp, _u32, _vp]),
    "cvd_copy_batch_host": (C.c_int, [_vp, _u32, _vp, _u32, _vp, _u64, _vp, _u64, _vp, _u32, _vp]),
    "cvd_copy_batches_host": (C.c_int, [_vp, _u32, _vp, _u32, _u32, _vp]),
    "cvd_copy_batch_noalloc": (C.c_int, [_vp, _vp, _u32, _vp, _u64, _vp, _u64, _vp, _vp]),
    "cvd_server_create": (C.c_int, [_vp, _u32, _vp, _u64, _u32, _u32, _u32, _vp]),
    "cvd_server_now_ns": (C.c_uint64, [_vp]),
    "cvd_server_submit": (C.c_int, [_vp, _vp, _u32, _vp]),
    "cvd_server_poll": (C.c_int, [_vp, _vp, _u32, _vp, _u32]),
    "cvd_server_release": (C.c_int, [_vp, C.c_uint64]),
    "cvd_server_destroy": (C.c_int, [_vp]),
    "cvd_get_copy_params": (C.c_int, [_vp]),
    "cvd_set_copy_params": (C.c_int, [_vp]),
    "cvd_tune": (C.c_int, [_vp, _u32, _vp, _u32, _vp, _u64, _vp, _u64, _vp, _u32, _vp, _vp, _vp]),
    "cvd_tune_batches": (C.c_int, [_vp, _u32, _vp, _u32, _vp, _u64, _u32, _vp, _vp, _vp, _vp]),
    "cvd_profile_enable": (C.c_int, [C.c_int]),
    "cvd_profile_read": (C.c_int, [_vp]),
    "cvd_stream_check": (C.c_int, [_vp, _vp]),
    "cvd_last_levels": (C.c_int, [_vp, _vp]),
    "cvd_selftest_wait_timeout": (C.c_int, [_vp, _u32, _vp]),
    "cvd_launch_count": (C.c_uint64, []),
    "cvd_probe_latency": (C.c_int, [_vp, _u64, _u32, _vp, _vp]),
    "cvd_translate_shape": (C.c_int, [_vp, _vp, _vp]),
    "cvd_strerror": (C.c_char_p, [C.c_int]),
    "cvd_last_cuda_error": (C.c_int, []),
}


class CvdError(RuntimeError):
    def __init__(self, fn, status):
        msg = lib().cvd_strerror(status).decode()
        if status == ECUDA:
            msg += f" (cuda error {lib().cvd_last_cuda_error()})"
        super().__init__(f"{fn}: {msg} [{status}]")
        self.status = status


class Memslot(C.Structure):
    _fields_ = [("base_gfn", C.c_uint64), ("npages", C.c_uint64), ("host_off", C.c_uint64)]


class GuestDesc(C.Structure):
    _fields_ = [("d_host_pool", C.c_void_p), ("host_pool_bytes", C.c_uint64),
                ("slots", C.c_void_p), ("nslots", C.c_uint32), ("paging", C.c_uint32),
                ("cr3_gpa", C.c_uint64), ("pt_pool_gfn", C.c_uint64), ("pt_pool_n", C.c_uint64),
                ("rsv_gfn", C.c_uint64), ("rsv_n", C.c_uint64), ("d_p2m", C.c_void_p),
                ("second", C.c_uint32), ("reserved1", C.c_uint32), ("ept_root", C.c_uint64)]


class CopyParams(C.Structure):
    _fields_ = [("vec_bytes", C.c_uint32), ("unroll", C.c_uint32), ("chunk_bytes", C.c_uint32),
                ("blocks_per_sm", C.c_uint32), ("warps_per_block", C.c_uint32), ("small_bytes", C.c_uint32),
                ("engine", C.c_uint32), ("stages", C.c_uint32), ("stage_bytes", C.c_uint32),
                ("ring_bytes", C.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """Load libcvd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1304_3771_b300.build`")
        handle = C.CDLL(LIB_PATH)
        for name, (rt, at) in SIGNATURES.items():
            f = getattr(handle, name)
            f.restype, f.argtypes = rt, at
        _lib = handle
    return _lib


def _check(fn, status):
    if status != OK:
        raise CvdError(fn, status)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def records_to_device(arr: np.ndarray, device="cuda") -> torch.Tensor:
    """Raw bytes of a structured array as a device uint8 tensor."""
    b = np.ascontiguousarray(arr).view(np.uint8).reshape(-1)
    if b.size == 0:
        return torch.zeros(16, dtype=torch.uint8, device=device)
    return torch.from_numpy(b.copy()).to(device)


def records_from_device(t: torch.Tensor, dtype: np.dtype, n: int) -> np.ndarray:
    return t[: n * dtype.itemsize].cpu().numpy().view(dtype)[:n].copy()


def u64_to_device(a: np.ndarray, device="cuda") -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to(device)


def u64_from_device(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


class Guest:
    """A cvd_guest handle over a device host pool (torch uint8 tensor).  With
    ``ept_root`` (host-pool offset of an EPT in the pool) the second dimension
    is that EPT and ``slots`` must be empty."""

    def __init__(self, pool: torch.Tensor, slots: np.ndarray, cr3_gpa: int, *, pt_pool_gfn=0, pt_pool_n=0,
                 rsv_gfn=0, rsv_n=0, p2m: torch.Tensor | None = None, paging: int = 0,
                 ept_root: int | None = None):
        assert pool.is_cuda and pool.dtype == torch.uint8
        self.handle = None
        self.pool = pool
        self.desc = dict(slots=np.array([(int(s["base_gfn"]), int(s["npages"]), int(s["host_off"])) for s in slots],
                                        dtype=np.uint64).reshape(-1, 3),
                         cr3_gpa=int(cr3_gpa), paging=int(paging), pt_pool_gfn=int(pt_pool_gfn),
                         pt_pool_n=int(pt_pool_n), rsv_gfn=int(rsv_gfn), rsv_n=int(rsv_n), ept_root=ept_root)
        if p2m is None and rsv_n:
            p2m = torch.full((rsv_n,), -1, dtype=torch.int64, device=pool.device)
        self.p2m = p2m
        self._slots = (Memslot * max(len(slots), 1))(*[Memslot(int(s["base_gfn"]), int(s["npages"]),
                                                               int(s["host_off"])) for s in slots])
        d = GuestDesc(pool.data_ptr(), pool.numel(), C.cast(self._slots, C.c_void_p), len(slots), paging, cr3_gpa,
                      pt_pool_gfn, pt_pool_n, rsv_gfn, rsv_n, p2m.data_ptr() if p2m is not None else None,
                      SECOND_MEMSLOTS if ept_root is None else SECOND_EPT, 0, ept_root or 0)
        h = C.c_void_p()
        _check("cvd_guest_create", lib().cvd_guest_create(C.byref(d), C.byref(h)))
        self.handle = h

    @classmethod
    def from_image(cls, img, pool: torch.Tensor, p2m: torch.Tensor | None = None):
        """Memslot guest, or (an image with an EPT) the same guest behind its
        EPT: no slots, no PT pool."""
        ept_root = getattr(img, "ept_root", None)
        if ept_root is not None:
            return cls(pool, img.slots[:0], img.cr3_gpa, rsv_gfn=img.rsv_gfn, rsv_n=img.rsv_n, p2m=p2m,
                       paging=getattr(img, "paging", 0), ept_root=ept_root)
        return cls(pool, img.slots, img.cr3_gpa, pt_pool_gfn=img.pt_pool_gfn, pt_pool_n=img.pt_pool_n,
                   rsv_gfn=img.rsv_gfn, rsv_n=img.rsv_n, p2m=p2m, paging=getattr(img, "paging", 0))

    def state(self):
        """The guest's state as a repro.GuestState (pool, p2m and counters
        copied to the host after a device synchronisation)."""
        from . import repro
        pt_used, rsv_used = self.alloc_state()
        p2m = self.p2m.cpu().numpy().view(np.uint64).copy() if self.p2m is not None else None
        return repro.GuestState(pool=self.pool.cpu().numpy().copy(), p2m=p2m, pt_used=pt_used, rsv_used=rsv_used,
                                **self.desc)

    @classmethod
    def from_state(cls, st, device="cuda"):
        """A new guest on `device` from a repro.GuestState: its pool and p2m
        copied to the device, its allocation counters restored."""
        st.check()
        pool = torch.from_numpy(np.ascontiguousarray(st.pool)).to(device)
        p2m = torch.from_numpy(st.p2m.view(np.int64).copy()).to(device) if st.p2m is not None else None
        slots = st.slot_records(np.dtype([("base_gfn", "<u8"), ("npages", "<u8"), ("host_off", "<u8")]))
        g = cls(pool, slots, st.cr3_gpa, pt_pool_gfn=st.pt_pool_gfn, pt_pool_n=st.pt_pool_n, rsv_gfn=st.rsv_gfn,
                rsv_n=st.rsv_n, p2m=p2m, paging=st.paging, ept_root=st.ept_root)
        g.set_alloc_state(st.pt_used, st.rsv_used)
        return g

    def set_alloc_state(self, pt_used: int, rsv_used: int):
        _check("cvd_guest_set_alloc_state", lib().cvd_guest_set_alloc_state(self.handle, pt_used, rsv_used))

    def close(self):
        if self.handle:
            _check("cvd_guest_destroy", lib().cvd_guest_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alloc_state(self):
        a, b = C.c_uint64(), C.c_uint64()
        _check("cvd_guest_alloc_state", lib().cvd_guest_alloc_state(self.handle, C.byref(a), C.byref(b)))
        return a.value, b.value

    def translate(self, gva: torch.Tensor, write: bool = False, out=None, stream=None):
        n = gva.numel()
        if out is None:
            out = (torch.empty(n, dtype=torch.int64, device=gva.device),
                   torch.empty(n, dtype=torch.int64, device=gva.device),
                   torch.empty(n, dtype=torch.int32, device=gva.device))
        gpa, hpa, code = out
        _check("cvd_translate", lib().cvd_translate(self.handle, _ptr(gva), n, int(write), _ptr(gpa), _ptr(hpa),
                                                    _ptr(code), _stream(stream)))
        return gpa, hpa, code

    def copy_from(self, req, nreq, seg, nseg, stg, res, stream=None):
        _check("cvd_copy_from_guest", lib().cvd_copy_from_guest(self.handle, _ptr(req), nreq, _ptr(seg), nseg,
                                                                _ptr(stg), stg.numel(), _ptr(res), _stream(stream)))

    def copy_to(self, req, nreq, seg, nseg, stg, res, stream=None):
        _check("cvd_copy_to_guest", lib().cvd_copy_to_guest(self.handle, _ptr(req), nreq, _ptr(seg), nseg,
                                                            _ptr(stg), stg.numel(), _ptr(res), _stream(stream)))

    def mmap_install(self, req, nreq, hf, nhf, status, stream=None):
        _check("cvd_mmap_install", lib().cvd_mmap_install(self.handle, _ptr(req), nreq, _ptr(hf), nhf,
                                                          _ptr(status), _stream(stream)))

    def mmap_place(self, va_lo, va_hi, req, nreq, hf, nhf, gva, status, stream=None):
        """Driver-initiated maps: the library picks each range in [va_lo, va_hi)."""
        _check("cvd_mmap_place", lib().cvd_mmap_place(self.handle, va_lo, va_hi, _ptr(req), nreq, _ptr(hf), nhf,
                                                      _ptr(gva), _ptr(status), _stream(stream)))


def _guest_array(guests):
    return (C.c_void_p * len(guests))(*[g.handle.value for g in guests])


class DevBatch(C.Structure):
    _fields_ = [("d_req", C.c_void_p), ("nreq", C.c_uint32), ("pad", C.c_uint32), ("d_seg", C.c_void_p),
                ("nseg", C.c_uint64), ("d_res", C.c_void_p)]


def copy_batches(guests, batches, stg, stream=None):
    """Hazard-free batches in order, each batch planned while the previous one
    copies.  ``batches``: (req, nreq, seg, nseg, res) device tensors."""
    arr = _guest_array(guests)
    items = (DevBatch * max(len(batches), 1))(*[DevBatch(r.data_ptr(), n, 0, s.data_ptr(), ns, o.data_ptr())
                                               for r, n, s, ns, o in batches])
    _check("cvd_copy_batches", lib().cvd_copy_batches(C.cast(arr, C.c_void_p), len(guests), items, len(batches),
                                                      _ptr(stg), stg.numel(), BATCH_HAZARD_FREE, _stream(stream)))


def gather_chained(guests, req, nreq, desc, payload, res, flags=0, stream=None):
    """Dependent second-level gathers: descriptor tables into ``desc``, then
    the buffers they name into ``payload`` (device uint8 tensors)."""
    arr = _guest_array(guests)
    _check("cvd_gather_chained", lib().cvd_gather_chained(C.cast(arr, C.c_void_p), len(guests), _ptr(req), nreq,
                                                          _ptr(desc), desc.numel(), _ptr(payload), payload.numel(),
                                                          _ptr(res), flags, _stream(stream)))


def copy_batch(guests, req, nreq, seg, nseg, stg, res, flags=0, stream=None):
    arr = _guest_array(guests)
    _check("cvd_copy_batch", lib().cvd_copy_batch(C.cast(arr, C.c_void_p), len(guests), _ptr(req), nreq, _ptr(seg),
                                                  nseg, _ptr(stg), stg.numel(), _ptr(res), flags, _stream(stream)))


def copy_batch_host(guests, req: torch.Tensor, nreq, seg: torch.Tensor, nseg, stg: torch.Tensor, res: torch.Tensor,
                    flags=0, stream=None):
    """Host-buffer batch: req/seg/stg/res are CPU tensors (pinned for full speed)."""
    arr = _guest_array(guests)
    _check("cvd_copy_batch_host", lib().cvd_copy_batch_host(C.cast(arr, C.c_void_p), len(guests), _ptr(req), nreq,
                                                            _ptr(seg), nseg, _ptr(stg), stg.numel(), _ptr(res),
                                                            flags, _stream(stream)))


class HostBatch(C.Structure):
    _fields_ = [("h_req", C.c_void_p), ("nreq", C.c_uint32), ("pad", C.c_uint32), ("h_seg", C.c_void_p),
                ("nseg", C.c_uint64), ("h_host_buf", C.c_void_p), ("host_buf_bytes", C.c_uint64),
                ("h_res", C.c_void_p)]


def copy_batches_host(guests, batches, flags=0, stream=None):
    """cvd_copy_batches_host: batches = [(req, nreq, seg, nseg, stg, res), ...]
    of CPU tensors (pinned for full speed), run in order with the transfers
    of consecutive batches overlapped."""
    arr = _guest_array(guests)
    hb = (HostBatch * max(len(batches), 1))()
    for i, (req, nreq, seg, nseg, stg, res) in enumerate(batches):
        hb[i] = HostBatch(_ptr(req), nreq, 0, _ptr(seg), nseg, _ptr(stg), stg.numel(), _ptr(res))
    _check("cvd_copy_batches_host", lib().cvd_copy_batches_host(C.cast(arr, C.c_void_p), len(guests), C.byref(hb),
                                                                len(batches), flags, _stream(stream)))


def copy_batch_noalloc(guest, req, nreq, seg, nseg, stg, res, stream=None):
    """cvd_copy_batch_noalloc: hazard-free single-guest batch on the library's
    fixed scratch (no device allocation in the call)."""
    _check("cvd_copy_batch_noalloc", lib().cvd_copy_batch_noalloc(guest.handle, _ptr(req), nreq, _ptr(seg), nseg,
                                                                  _ptr(stg), stg.numel(), _ptr(res),
                                                                  _stream(stream)))


class ServerReq(C.Structure):
    _fields_ = [("guest", C.c_uint32), ("dir", C.c_uint32), ("nseg", C.c_uint32), ("pad", C.c_uint32),
                ("segs", C.c_void_p), ("d_src", C.c_void_p), ("arrival_ns", C.c_uint64), ("tag", C.c_uint64)]


class Result(C.Structure):
    _fields_ = [("done", C.c_uint64), ("fault_gva", C.c_uint64), ("fault_code", C.c_uint32), ("pad", C.c_uint32)]


class ServerDone(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("tag", C.c_uint64), ("res", Result), ("staging_off", C.c_uint64),
                ("len", C.c_uint64), ("arrival_ns", C.c_uint64), ("admit_ns", C.c_uint64),
                ("launch_ns", C.c_uint64), ("complete_ns", C.c_uint64), ("guest", C.c_uint32), ("dir", C.c_uint32),
                ("wave_device_ns", C.c_uint64)]


# cvd_server_req / cvd_server_done as numpy records (the array forms of
# Server.submit_array / Server.poll_array)
SERVER_REQ_DTYPE = np.dtype([("guest", "<u4"), ("dir", "<u4"), ("nseg", "<u4"), ("pad", "<u4"), ("segs", "<u8"),
                             ("d_src", "<u8"), ("arrival_ns", "<u8"), ("tag", "<u8")])
SERVER_DONE_DTYPE = np.dtype([("ticket", "<u8"), ("tag", "<u8"), ("done", "<u8"), ("fault_gva", "<u8"),
                              ("fault_code", "<u4"), ("res_pad", "<u4"), ("staging_off", "<u8"), ("len", "<u8"),
                              ("arrival_ns", "<u8"), ("admit_ns", "<u8"), ("launch_ns", "<u8"),
                              ("complete_ns", "<u8"), ("guest", "<u4"), ("dir", "<u4"), ("wave_device_ns", "<u8")])


class Server:
    """cvd_server: continuous batching of forwarded copies from several guests."""

    def __init__(self, guests, staging: torch.Tensor, max_batch=256, max_inflight=4096, auto_release=False,
                 two_streams=False):
        self.guests = list(guests)
        self.staging = staging
        arr = _guest_array(self.guests)
        h = C.c_void_p()
        _check("cvd_server_create", lib().cvd_server_create(C.cast(arr, C.c_void_p), len(self.guests),
                                                            staging.data_ptr(), staging.numel(), max_batch,
                                                            max_inflight, (1 if auto_release else 0) |
                                                            (2 if two_streams else 0), C.byref(h)))
        self.handle = h
        self._keep = []

    def now_ns(self) -> int:
        return lib().cvd_server_now_ns(self.handle)

    def submit(self, items):
        """items: list of (guest, dir, segs ndarray[SEG_DTYPE], d_src ptr or 0, arrival_ns, tag)."""
        n = len(items)
        reqs = (ServerReq * n)()
        keep = []
        for i, (guest, d, segs, src, arrival, tag) in enumerate(items):
            segs = np.ascontiguousarray(segs)
            keep.append(segs)
            reqs[i] = ServerReq(guest, d, len(segs), 0, segs.ctypes.data if len(segs) else None, src or None,
                                arrival, tag)
        tickets = (C.c_uint64 * max(n, 1))()
        _check("cvd_server_submit", lib().cvd_server_submit(self.handle, C.cast(reqs, C.c_void_p), n,
                                                            C.cast(tickets, C.c_void_p)))
        return list(tickets)[:n]

    def poll(self, max_n=4096, timeout_us=100000):
        out = (ServerDone * max_n)()
        k = C.c_uint32()
        st = lib().cvd_server_poll(self.handle, C.cast(out, C.c_void_p), max_n, C.byref(k), timeout_us)
        if st == ETIMEDOUT:
            return []
        _check("cvd_server_poll", st)
        return [out[i] for i in range(k.value)]

    def submit_array(self, reqs: np.ndarray):
        """Queue SERVER_REQ_DTYPE records (segs: address of each request's
        SEG_DTYPE array, which the caller keeps alive until this returns)."""
        reqs = np.ascontiguousarray(reqs, dtype=SERVER_REQ_DTYPE)
        _check("cvd_server_submit", lib().cvd_server_submit(self.handle, reqs.ctypes.data, len(reqs), None))

    def poll_array(self, max_n=65536, timeout_us=100000) -> np.ndarray:
        """Completions as SERVER_DONE_DTYPE records (empty on a timeout)."""
        if not hasattr(self, "_done_buf") or len(self._done_buf) < max_n:
            self._done_buf = np.zeros(max_n, dtype=SERVER_DONE_DTYPE)
        k = C.c_uint32()
        st = lib().cvd_server_poll(self.handle, self._done_buf.ctypes.data, max_n, C.byref(k), timeout_us)
        if st == ETIMEDOUT:
            return self._done_buf[:0].copy()
        _check("cvd_server_poll", st)
        return self._done_buf[:k.value].copy()

    def release(self, ticket):
        _check("cvd_server_release", lib().cvd_server_release(self.handle, ticket))

    def close(self):
        if self.handle:
            _check("cvd_server_destroy", lib().cvd_server_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def get_copy_params() -> CopyParams:
    p = CopyParams()
    _check("cvd_get_copy_params", lib().cvd_get_copy_params(C.byref(p)))
    return p


def set_copy_params(**kw):
    p = get_copy_params()
    for k, v in kw.items():
        setattr(p, k, v)
    _check("cvd_set_copy_params", lib().cvd_set_copy_params(C.byref(p)))


def tune(guests, req, nreq, seg, nseg, stg, res, reps=3, stream=None):
    arr = _guest_array(guests)
    p = CopyParams()
    ms = C.c_float()
    _check("cvd_tune", lib().cvd_tune(C.cast(arr, C.c_void_p), len(guests), _ptr(req), nreq, _ptr(seg), nseg,
                                      _ptr(stg), stg.numel(), _ptr(res), reps, _stream(stream), C.byref(p),
                                      C.byref(ms)))
    return p, ms.value


def tune_batches(guests, batches, stg, reps=2, stream=None):
    """cvd_tune_batches: autotune the planned-ahead step over ``batches``
    ((req, nreq, seg, nseg, res) device tensors).  Returns (params, ms per
    step, whether the choice came from the tuning cache)."""
    arr = _guest_array(guests)
    items = (DevBatch * max(len(batches), 1))(*[DevBatch(r.data_ptr(), n, 0, s.data_ptr(), ns, o.data_ptr())
                                               for r, n, s, ns, o in batches])
    p = CopyParams()
    ms = C.c_float()
    cached = C.c_int()
    _check("cvd_tune_batches", lib().cvd_tune_batches(C.cast(arr, C.c_void_p), len(guests), items, len(batches),
                                                      _ptr(stg), stg.numel(), reps, _stream(stream), C.byref(p),
                                                      C.byref(ms), C.byref(cached)))
    return p, ms.value, bool(cached.value)


class Profile(C.Structure):
    _fields_ = [("plan_ms", C.c_double), ("copy_ms", C.c_double), ("plan_calls", C.c_uint64),
                ("copy_calls", C.c_uint64), ("map_probe_ms", C.c_double), ("place_fit_ms", C.c_double),
                ("map_probe_calls", C.c_uint64), ("place_fit_calls", C.c_uint64)]


def profile_enable(on: bool = True):
    _check("cvd_profile_enable", lib().cvd_profile_enable(int(on)))


def profile_read() -> dict:
    p = Profile()
    _check("cvd_profile_read", lib().cvd_profile_read(C.byref(p)))
    return {f: getattr(p, f) for f, _ in p._fields_}


def stream_check(stream=None) -> int:
    """Synchronise the stream; return and clear the device error bits."""
    v = C.c_uint32()
    _check("cvd_stream_check", lib().cvd_stream_check(_stream(stream), C.byref(v)))
    return v.value


def selftest_wait_timeout(tries=1 << 12, stream=None) -> int:
    """Run the bounded-wait failure self-test; returns the error bits it reported."""
    v = C.c_uint32()
    _check("cvd_selftest_wait_timeout", lib().cvd_selftest_wait_timeout(_stream(stream), tries, C.byref(v)))
    return v.value


def last_levels(stream=None) -> int:
    v = C.c_uint32()
    _check("cvd_last_levels", lib().cvd_last_levels(_stream(stream), C.byref(v)))
    return v.value


RUN_DTYPE = np.dtype([("dst", "<u8"), ("src", "<u8"), ("len", "<u8"), ("pad", "<u8")])   # cvd_run


def level_runs(runs: np.ndarray):
    """cvd_level_runs on RUN_DTYPE records: (levels int32 array, highest level, marked runs)."""
    runs = np.ascontiguousarray(runs, dtype=RUN_DTYPE)
    lev = np.zeros(max(len(runs), 1), np.int32)
    marked = C.c_uint64()
    rc = lib().cvd_level_runs(runs.ctypes.data if len(runs) else None, len(runs), lev.ctypes.data, C.byref(marked))
    if rc < 0:
        raise CvdError("cvd_level_runs", rc)
    return lev[:len(runs)], rc, marked.value


def launch_count() -> int:
    return lib().cvd_launch_count()


def translate_shape(guest=None):
    """(resident threads per SM, walks in flight per thread) of cvd_translate
    for ``guest`` (None: a guest whose memslots are searched)."""
    t, w = C.c_uint32(), C.c_uint32()
    _check("cvd_translate_shape", lib().cvd_translate_shape(guest.handle if guest is not None else None,
                                                            C.byref(t), C.byref(w)))
    return t.value, w.value


def probe_latency(buf, steps=200_000, stream=None) -> float:
    """ns per dependent L2-only load along a chain written into the device
    tensor `buf` (overwritten; see cvd_probe_latency)."""
    v = C.c_double()
    _check("cvd_probe_latency", lib().cvd_probe_latency(_ptr(buf), buf.numel() * buf.element_size(), steps,
                                                        _stream(stream), C.byref(v)))
    return v.value


__all__ = ["Guest", "copy_batch", "copy_batch_host", "copy_batches_host", "tune", "get_copy_params", "set_copy_params", "last_levels",
           "level_runs", "RUN_DTYPE",
           "launch_count", "probe_latency", "translate_shape", "records_to_device", "records_from_device", "u64_to_device", "u64_from_device", "W",
           "CvdError", "SIGNATURES", "LIB_PATH"]
