"""Seeded synthetic workloads for the CVD memory operations.

This module only *constructs inputs*: guest-physical memory images whose page
tables follow the public x86-64 4-level paging format (Intel SDM Vol. 3,
ch. 4), KVM-style memslots, and forwarded read/write/ioctl/mmap requests.  It
holds none of the method's arithmetic (no page walk, no copy, no PTE install):
both the CPU oracle and the CUDA library consume what it produces, and neither
imports the other.

Record layouts (little-endian, shared by every consumer as plain bytes):

    SEG_DTYPE     {gva u64, len u64}                          16 B
    REQ_DTYPE     {seg_begin u32, seg_count u32, dir u32,
                   guest u32, host_off u64}                   24 B
    RESULT_DTYPE  {done u64, fault_gva u64, fault_code u32,
                   pad u32}                                   24 B
    MAPREQ_DTYPE  {gva u64, npages u32, flags u32,
                   hf_begin u64}                              24 B
    SLOT_DTYPE    {base_gfn u64, npages u64, host_off u64}    24 B
    PLACE_DTYPE   {npages u32, flags u32, hf_begin u64}      16 B
    CHAIN_REQ_DTYPE {table_gva u64, count u32, guest u32,
                   desc_off u64}                              24 B
    CHAIN_RES_DTYPE {done u64, fault_gva u64, fault_code u32,
                   level u32, payload_off u64, payload_len u64} 40 B

dir: 0 = copy from guest (gather into the staging buffer),
     1 = copy to guest   (scatter from the staging buffer).

Workload shapes stand in for the paper's device classes (GPU command buffers,
camera/framebuffer frames, small input and audio ioctls; Sec. 7.3-7.4); the
paper publishes no traces, so every input here is synthetic and seeded.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

PAGE = 4096
PAGE_SHIFT = 12
HUGE = 2 << 20
ENTRIES = 512
USER_TOP = 1 << 47

# x86-64 page-table entry bits (Intel SDM Vol. 3, Table 4-15..4-20).
PTE_P = 1 << 0
PTE_RW = 1 << 1
PTE_US = 1 << 2
PTE_PWT = 1 << 3
PTE_PCD = 1 << 4
PTE_A = 1 << 5
PTE_D = 1 << 6
PTE_PS = 1 << 7
PTE_G = 1 << 8
PTE_NX = 1 << 63
# mmap request flag word: low bits as in a PTE, NX carried in bit 31.
MAP_NX = 1 << 31

SEG_DTYPE = np.dtype([("gva", "<u8"), ("len", "<u8")])
REQ_DTYPE = np.dtype([("seg_begin", "<u4"), ("seg_count", "<u4"), ("dir", "<u4"),
                      ("guest", "<u4"), ("host_off", "<u8")])
RESULT_DTYPE = np.dtype([("done", "<u8"), ("fault_gva", "<u8"), ("fault_code", "<u4"),
                         ("pad", "<u4")])
MAPREQ_DTYPE = np.dtype([("gva", "<u8"), ("npages", "<u4"), ("flags", "<u4"),
                         ("hf_begin", "<u8")])
SLOT_DTYPE = np.dtype([("base_gfn", "<u8"), ("npages", "<u8"), ("host_off", "<u8")])
PLACE_DTYPE = np.dtype([("npages", "<u4"), ("flags", "<u4"), ("hf_begin", "<u8")])
CHAIN_REQ_DTYPE = np.dtype([("table_gva", "<u8"), ("count", "<u4"), ("guest", "<u4"), ("desc_off", "<u8")])
CHAIN_RES_DTYPE = np.dtype([("done", "<u8"), ("fault_gva", "<u8"), ("fault_code", "<u4"), ("level", "<u4"),
                            ("payload_off", "<u8"), ("payload_len", "<u8")])

DEFAULT_SEED = 0x13043771
PAGING_X86_64, PAGING_PAE = 0, 1


def rng_for(seed: int, *purpose: int) -> np.random.Generator:
    """Independent PCG64 stream keyed by (seed, purpose...)."""
    return np.random.default_rng(np.random.SeedSequence([seed & 0xFFFFFFFF, *purpose]))


# ---------------------------------------------------------------------------
# Guest image
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class GuestImage:
    """A guest's physical memory as laid out in the host pool.

    ``tables`` maps a guest frame number to its 512 x u64 page-table contents;
    everything else in the arena is payload.  ``page_gfn``/``page_flags``
    record, for every 4 KiB page of the data gVA region, the frame and leaf
    flags the generator placed there (``-1`` for pages mapped by a 2 MiB leaf,
    whose frames are in ``huge_gfn``); tests use them as the brute-force
    ground truth of a walk.
    """
    arena_bytes: int
    pool_bytes: int
    slots: np.ndarray                 # SLOT_DTYPE
    cr3_gpa: int
    tables: dict                      # gfn -> np.ndarray[512] uint64
    pt_pool_gfn: int
    pt_pool_n: int
    rsv_gfn: int
    rsv_n: int
    data_gva: int                     # base of the data gVA region
    data_pages: int                   # 4 KiB pages in the data region
    page_gfn: np.ndarray              # int64 per data page (-1: inside a huge leaf)
    page_flags: np.ndarray            # uint64 leaf flags per data page
    huge_gfn: Optional[np.ndarray] = None   # int64 per 2 MiB unit (-1: 4 KiB mapped)
    huge_flags: Optional[np.ndarray] = None
    payload_seed: int = 0
    paging: int = 0                   # 0: x86-64 4-level, 1: 32-bit PAE (3 levels)
    ept_root: Optional[int] = None    # host-pool offset of the EPT PML4 (second dimension), or memslots
    ept_tables: Optional[dict] = None # host offset -> 512 x u64 EPT table
    ept_unmapped: Optional[np.ndarray] = None   # guest frames the EPT leaves unmapped
    ept_readonly: Optional[np.ndarray] = None   # guest frames the EPT maps read-only

    @property
    def va_top(self) -> int:
        """End of the guest's user virtual range (2^47, or 2^32 for PAE)."""
        return (1 << 32) if self.paging == PAGING_PAE else USER_TOP

    def gpa_to_host(self, gpa: int) -> int:
        """Host pool offset of a guest-physical address (memslot image)."""
        gfn = gpa >> PAGE_SHIFT
        for s in self.slots:
            b, n, h = int(s["base_gfn"]), int(s["npages"]), int(s["host_off"])
            if b <= gfn < b + n:
                return h + gpa - b * PAGE
        raise KeyError(hex(gpa))

    def host_ranges(self):
        """(host_off, bytes) of every memslot."""
        return [(int(s["host_off"]), int(s["npages"]) * PAGE) for s in self.slots]


def _alloc_table(tables: dict, free_top: list) -> int:
    gfn = free_top[0]
    free_top[0] -= 1
    tables[gfn] = np.zeros(ENTRIES, dtype=np.uint64)
    return gfn


def build_tables(top_gfn: int, leaves4k, leaves2m=None, inter_flags: int = PTE_P | PTE_RW | PTE_US):
    """Encode x86-64 4-level tables for the given leaves.

    leaves4k: (vpn int64[], entry uint64[])  -- vpn = gva >> 12, entry = full PTE
    leaves2m: (vpn2m int64[], entry uint64[]) -- vpn2m = gva >> 21, entry = full PDE (PS set)
    Table frames are taken downward from ``top_gfn``.  Returns
    (cr3_gpa, tables dict, lowest gfn used).
    """
    tables: dict = {}
    free = [top_gfn]
    pml4 = _alloc_table(tables, free)
    pdpt: dict = {}
    pd: dict = {}
    pt: dict = {}

    def get(level_map, key, parent_gfn, parent_idx):
        g = level_map.get(key)
        if g is None:
            g = _alloc_table(tables, free)
            level_map[key] = g
            tables[parent_gfn][parent_idx] = np.uint64((g << PAGE_SHIFT) | inter_flags)
        return g

    def path_to_pd(vpn2m):
        i4 = (vpn2m >> 18) & 511
        i3 = (vpn2m >> 9) & 511
        g3 = get(pdpt, vpn2m >> 18, pml4, i4)
        g2 = get(pd, vpn2m >> 9, g3, i3)
        return g2

    # Vectorised by unique prefixes, then filled with numpy fancy indexing.
    if leaves2m is not None and len(leaves2m[0]):
        v2, e2 = leaves2m
        v2 = np.asarray(v2, dtype=np.int64)
        for key in np.unique(v2 >> 9):
            g2 = path_to_pd(int(key) << 9)
            sel = (v2 >> 9) == key
            tables[g2][(v2[sel] & 511)] = np.asarray(e2, dtype=np.uint64)[sel]
    v1, e1 = leaves4k
    v1 = np.asarray(v1, dtype=np.int64)
    e1 = np.asarray(e1, dtype=np.uint64)
    if len(v1):
        order = np.argsort(v1, kind="stable")
        v1s, e1s = v1[order], e1[order]
        keys, starts = np.unique(v1s >> 9, return_index=True)
        ends = np.append(starts[1:], len(v1s))
        for key, a, b in zip(keys, starts, ends):
            key = int(key)
            g2 = path_to_pd(key)
            g1 = get(pt, key, g2, key & 511)
            tables[g1][v1s[a:b] & 511] = e1s[a:b]
    return pml4 << PAGE_SHIFT, tables, free[0] + 1


def build_tables_pae(top_gfn: int, leaves4k, leaves2m=None):
    """Encode 32-bit PAE tables (Intel SDM Vol. 3 sec. 4.4) for the given
    leaves: a 4-entry page directory pointer table at the start of a frame
    (its entries carry P and the frame only), page directories, page tables
    (links P|RW|US).  Same arguments and result as ``build_tables``."""
    tables: dict = {}
    free = [top_gfn]
    pdpt = _alloc_table(tables, free)
    pd: dict = {}
    pt: dict = {}

    def get_pd(i3):
        g = pd.get(i3)
        if g is None:
            g = _alloc_table(tables, free)
            pd[i3] = g
            tables[pdpt][i3] = np.uint64((g << PAGE_SHIFT) | PTE_P)
        return g

    def get_pt(vpn2m):
        g = pt.get(vpn2m)
        if g is None:
            g = _alloc_table(tables, free)
            pt[vpn2m] = g
            tables[get_pd(vpn2m >> 9)][vpn2m & 511] = np.uint64((g << PAGE_SHIFT) | PTE_P | PTE_RW | PTE_US)
        return g

    if leaves2m is not None and len(leaves2m[0]):
        v2 = np.asarray(leaves2m[0], dtype=np.int64)
        e2 = np.asarray(leaves2m[1], dtype=np.uint64)
        for v, e in zip(v2, e2):
            tables[get_pd(int(v) >> 9)][int(v) & 511] = e
    v1 = np.asarray(leaves4k[0], dtype=np.int64)
    e1 = np.asarray(leaves4k[1], dtype=np.uint64)
    if len(v1):
        order = np.argsort(v1, kind="stable")
        v1s, e1s = v1[order], e1[order]
        keys, starts = np.unique(v1s >> 9, return_index=True)
        ends = np.append(starts[1:], len(v1s))
        for key, a, b in zip(keys, starts, ends):
            tables[get_pt(int(key))][v1s[a:b] & 511] = e1s[a:b]
    return pdpt << PAGE_SHIFT, tables, free[0] + 1


def _leaf(gfn, flags):
    return (np.asarray(gfn, dtype=np.uint64) << np.uint64(PAGE_SHIFT)) | np.asarray(flags, dtype=np.uint64)


def make_guest(arena_bytes: int, seed: int, *, huge_frac: float = 0.0, np_frac: float = 0.05,
               ro_frac: float = 0.05, nslots: int = 1, pt_pool_n: int = 256, rsv_n: int = 4096,
               slot_gap_pages: int = 0, host_base: Optional[int] = None, purpose: int = 0,
               shuffle: bool = True, paging: str = "x86_64") -> GuestImage:
    """Seeded guest: data gVA region mapped by a random frame permutation.

    The arena's frames are [0, F).  The top frames hold the page tables and,
    below them, the PT pool handed to mmap installs (the frontend's pre-
    allocated pool, Sec. 4.2).  The data region starts at a seeded 1 GiB
    aligned user address; each 2 MiB unit is a 2 MiB leaf with probability
    ``huge_frac`` (placement seeded), otherwise 512 4 KiB leaves.  ``np_frac``
    of 4 KiB leaves have P cleared (frame bits kept), ``ro_frac`` have RW
    cleared.  ``nslots`` memslots split the arena at 2 MiB aligned points and
    are laid out in the host pool in seeded order with gaps.  ``paging="pae"``
    builds a 32-bit PAE guest (the paging mode of the paper's implementation,
    Sec. 6.2): the data region starts at a seeded 1 GiB boundary below 3 GiB.
    """
    pae = paging == "pae"
    assert paging in ("x86_64", "pae")
    rng = rng_for(seed, 1, purpose)
    F = arena_bytes // PAGE
    assert arena_bytes % HUGE == 0
    # Reserve the top: table frames (upper bound) + PT pool, 2 MiB aligned.
    n4k_units_est = int(math.ceil((1 - huge_frac) * (F // 512))) + 2
    table_frames_est = n4k_units_est + (F // 512) // 512 + 8
    top_frames = table_frames_est + pt_pool_n
    top_frames = ((top_frames + 511) // 512) * 512
    data_frames = F - top_frames
    assert data_frames > 0
    units = data_frames // 512
    data_frames = units * 512
    data_gva = int(rng.integers(1, (USER_TOP >> 30) // 4)) << 30
    if pae:
        assert data_frames * PAGE <= (2 << 30), "PAE data region must fit below 3 GiB"
        data_gva = int(rng.integers(1, ((3 << 30) - data_frames * PAGE) // (1 << 30) + 1)) << 30

    is_huge = rng.random(units) < huge_frac
    # 2 MiB units of guest-physical memory, permuted.
    unit_perm = rng.permutation(units) if shuffle else np.arange(units)
    huge_units = np.nonzero(is_huge)[0]
    small_units = np.nonzero(~is_huge)[0]
    # gPA blocks assigned to huge units / small units.
    huge_gblk = unit_perm[: len(huge_units)]
    small_gblk = unit_perm[len(huge_units):]
    # 4 KiB frames of the small blocks, globally permuted across small units.
    small_frames = (small_gblk[:, None] * 512 + np.arange(512)[None, :]).reshape(-1)
    if shuffle:
        small_frames = small_frames[rng.permutation(len(small_frames))]

    page_gfn = np.full(units * 512, -1, dtype=np.int64)
    page_flags = np.zeros(units * 512, dtype=np.uint64)
    small_vpn_local = (small_units[:, None] * 512 + np.arange(512)[None, :]).reshape(-1)
    page_gfn[small_vpn_local] = small_frames
    u = rng.random(len(small_vpn_local))
    fl = np.full(len(small_vpn_local), PTE_P | PTE_RW | PTE_US, dtype=np.uint64)
    fl[u < np_frac] &= ~np.uint64(PTE_P)
    fl[(u >= np_frac) & (u < np_frac + ro_frac)] &= ~np.uint64(PTE_RW)
    page_flags[small_vpn_local] = fl

    huge_gfn = np.full(units, -1, dtype=np.int64)
    huge_flags = np.zeros(units, dtype=np.uint64)
    huge_gfn[huge_units] = huge_gblk * 512
    huge_flags[huge_units] = PTE_P | PTE_RW | PTE_US | PTE_PS

    vpn0 = data_gva >> PAGE_SHIFT
    leaves4k = (vpn0 + small_vpn_local, _leaf(small_frames, fl))
    leaves2m = ((data_gva >> 21) + huge_units, _leaf(huge_gblk * 512, huge_flags[huge_units]))
    cr3, tables, low = (build_tables_pae if pae else build_tables)(F - 1, leaves4k, leaves2m)
    assert low >= F - top_frames + pt_pool_n, "table area overflow"
    pt_pool_gfn = F - top_frames

    # Memslots: split [0, F) at 2 MiB boundaries, place in pool in seeded order.
    if nslots == 1:
        cuts = [0, F]
    else:
        inner = np.sort(rng.choice(np.arange(1, F // 512), size=nslots - 1, replace=False)) * 512
        cuts = [0, *[int(c) for c in inner], F]
    order = rng.permutation(nslots) if nslots > 1 else np.array([0])
    base = host_base if host_base is not None else int(rng.integers(1, 256)) * PAGE
    slots = np.zeros(nslots, dtype=SLOT_DTYPE)
    host_cursor = base
    host_of = {}
    for k in order:
        host_of[int(k)] = host_cursor
        host_cursor += (cuts[k + 1] - cuts[k]) * PAGE + slot_gap_pages * PAGE
    for k in range(nslots):
        slots[k] = (cuts[k], cuts[k + 1] - cuts[k], host_of[k])
    pool_bytes = host_cursor + 16 * PAGE
    # Reserved gPA window above guest RAM (not covered by any memslot).
    rsv_gfn = F + 4096
    return GuestImage(arena_bytes=arena_bytes, pool_bytes=pool_bytes, slots=slots, cr3_gpa=cr3,
                      tables=tables, pt_pool_gfn=pt_pool_gfn, pt_pool_n=pt_pool_n, rsv_gfn=rsv_gfn,
                      rsv_n=rsv_n, data_gva=data_gva, data_pages=units * 512, page_gfn=page_gfn,
                      page_flags=page_flags, huge_gfn=huge_gfn, huge_flags=huge_flags,
                      payload_seed=seed ^ 0x5A5A, paging=PAGING_PAE if pae else PAGING_X86_64)


def payload_bytes(seed: int, n: int) -> np.ndarray:
    return rng_for(seed, 2).integers(0, 256, size=n, dtype=np.uint8)


EPT_R, EPT_W, EPT_X, EPT_LARGE = 1, 2, 4, 1 << 7


def add_ept(img: GuestImage, seed: int, *, huge_frac: float = 0.5, np_frac: float = 0.0, ro_frac: float = 0.0,
            purpose: int = 0) -> GuestImage:
    """The same guest with a software EPT as its second dimension (Intel SDM
    Vol. 3 sec. 28.3.2; the non-KVM case of Sec. 4.2): a 4-level table in an
    extra region of the host pool mapping every memslot frame to the same host
    bytes the memslot gives it.  A 2 MiB-aligned guest unit lying inside one
    slot whose host bytes are 2 MiB aligned becomes a 2 MiB EPT leaf with
    probability ``huge_frac``; ``np_frac`` / ``ro_frac`` of the 4 KiB data
    frames (never table or PT-pool frames) are left unmapped / mapped without
    write permission (their units stay 4 KiB mapped).  Intermediate entries:
    R|W|X; leaves: R|X plus W unless read-only.  Tables are allocated root
    first, then by level and ascending gPA."""
    rng = rng_for(seed, 11, purpose)
    data4k = np.sort(img.page_gfn[img.page_gfn >= 0])
    u = rng.random(len(data4k))
    unmapped = data4k[u < np_frac]
    readonly = data4k[(u >= np_frac) & (u < np_frac + ro_frac)]
    G = np.concatenate([np.arange(int(s["base_gfn"]), int(s["base_gfn"]) + int(s["npages"]), dtype=np.int64)
                        for s in img.slots])
    H = np.concatenate([int(s["host_off"]) + np.arange(int(s["npages"]), dtype=np.int64) * PAGE
                        for s in img.slots])
    order = np.argsort(G, kind="stable")
    G, H = G[order], H[order]
    bad = np.isin(G, unmapped) | np.isin(G, readonly)
    # 2 MiB units entirely inside one slot, host-aligned, with no altered frame
    unit = G >> 9
    uniq, first, cnt = np.unique(unit, return_index=True, return_counts=True)
    nbad = np.bincount(np.searchsorted(uniq, unit[bad]), minlength=len(uniq)) if bad.any() else np.zeros(len(uniq), int)
    contiguous = (H[first + np.minimum(cnt, 512) - 1] - H[first]) == (np.minimum(cnt, 512) - 1) * PAGE
    eligible = (cnt == 512) & (G[first] % 512 == 0) & (H[first] % HUGE == 0) & (nbad == 0) & contiguous
    huge_unit = np.zeros(len(uniq), dtype=bool)
    e_idx = np.nonzero(eligible)[0]
    huge_unit[e_idx] = rng.random(len(e_idx)) < huge_frac
    in_huge = huge_unit[np.searchsorted(uniq, unit)]
    hu_gfn = G[first[huge_unit]]
    hu_host = H[first[huge_unit]]
    small = ~in_huge
    sg, sh = G[small], H[small]
    gpa_all = G << PAGE_SHIFT
    k4 = np.unique(gpa_all >> 39)
    k3 = np.unique(gpa_all >> 30)
    k2 = np.unique(sg << PAGE_SHIFT >> 21)
    base = (img.pool_bytes + PAGE - 1) // PAGE * PAGE
    ntab = 1 + len(k4) + len(k3) + len(k2)
    T = np.zeros((ntab, ENTRIES), dtype=np.uint64)
    off3 = base + PAGE * (1 + np.arange(len(k4)))
    off2 = base + PAGE * (1 + len(k4) + np.arange(len(k3)))
    off1 = base + PAGE * (1 + len(k4) + len(k3) + np.arange(len(k2)))
    inter = np.uint64(EPT_R | EPT_W | EPT_X)
    T[0, k4 & 511] = off3.astype(np.uint64) | inter
    T[1 + np.searchsorted(k4, k3 >> 9), k3 & 511] = off2.astype(np.uint64) | inter
    T[1 + len(k4) + np.searchsorted(k3, k2 >> 9), k2 & 511] = off1.astype(np.uint64) | inter
    hgpa = hu_gfn << PAGE_SHIFT
    T[1 + len(k4) + np.searchsorted(k3, hgpa >> 30), (hgpa >> 21) & 511] = \
        hu_host.astype(np.uint64) | np.uint64(EPT_R | EPT_W | EPT_X | EPT_LARGE)
    keep = ~np.isin(sg, unmapped)
    sg, sh = sg[keep], sh[keep]
    fl = np.where(np.isin(sg, readonly), EPT_R | EPT_X, EPT_R | EPT_W | EPT_X).astype(np.uint64)
    T[1 + len(k4) + len(k3) + np.searchsorted(k2, sg >> 9), sg & 511] = sh.astype(np.uint64) | fl
    tables = {base + PAGE * i: T[i] for i in range(ntab)}
    return dataclasses.replace(img, ept_root=base, ept_tables=tables, ept_unmapped=unmapped,
                               ept_readonly=readonly, pool_bytes=base + ntab * PAGE + 16 * PAGE)


def materialize_pool(img: GuestImage, pool: Optional[np.ndarray] = None, fill: bool = True) -> np.ndarray:
    """Host-side pool image: uniform uint8 payload in every memslot, tables written."""
    if pool is None:
        pool = np.zeros(img.pool_bytes, dtype=np.uint8)
    if fill:
        for h, n in img.host_ranges():
            pool[h:h + n] = payload_bytes(img.payload_seed + h, n)
    write_tables(img, pool)
    return pool


def write_tables(img: GuestImage, pool: np.ndarray):
    for gfn, t in img.tables.items():
        h = img.gpa_to_host(gfn << PAGE_SHIFT)
        pool[h:h + PAGE] = t.view(np.uint8)
    for h, t in (img.ept_tables or {}).items():
        pool[h:h + PAGE] = t.view(np.uint8)


def table_blob(img: GuestImage):
    """(host offsets int64[n], bytes uint8[n, 4096]) of every table frame."""
    gfns = sorted(img.tables)
    offs = [img.gpa_to_host(g << PAGE_SHIFT) for g in gfns]
    blocks = [img.tables[g] for g in gfns]
    for h in sorted(img.ept_tables or {}):
        offs.append(h)
        blocks.append(img.ept_tables[h])
    offs = np.array(offs, dtype=np.int64)
    data = np.stack(blocks).view(np.uint8).reshape(len(offs), PAGE)
    return offs, data


# ---------------------------------------------------------------------------
# Copy requests
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class CopyWorkload:
    reqs: np.ndarray          # REQ_DTYPE
    segs: np.ndarray          # SEG_DTYPE
    staging_bytes: int
    batches: list             # list of (req_lo, req_hi): hazard-free batches (or one batch)
    payload_bytes: int        # sum of segment lengths

    def batch(self, k):
        lo, hi = self.batches[k]
        return self.reqs[lo:hi]


def log_uniform(rng, lo, hi, n):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n)).astype(np.int64).clip(lo, hi)


def tiny_requests(img: GuestImage, seed: int, nreq: int = 1000, max_segs: int = 8,
                  lo: int = 16, hi: int = 65536, purpose: int = 0, guest: int = 0,
                  staging_gap: int = 64, frame_frac: float = 0.0) -> CopyWorkload:
    """The tiny workload's shape: 1..max_segs segments at uniform gVA offsets in the data
    region, log-uniform lengths, 50/50 direction, disjoint staging ranges.
    Requests may overlap each other in guest memory (sequential semantics).
    ``frame_frac`` of requests are instead one 640x480 YUYV frame (614,400 B)."""
    rng = rng_for(seed, 3, purpose)
    nseg = rng.integers(1, max_segs + 1, nreq)
    is_frame = rng.random(nreq) < frame_frac
    nseg[is_frame] = 1
    total = int(nseg.sum())
    lens = log_uniform(rng, lo, hi, total)
    seg_req = np.repeat(np.arange(nreq), nseg)
    frame_len = 640 * 480 * 2
    lens[is_frame[seg_req]] = frame_len
    region = img.data_pages * PAGE
    offs = (rng.random(total) * (region - lens)).astype(np.int64)
    segs = np.zeros(total, dtype=SEG_DTYPE)
    segs["gva"] = img.data_gva + offs
    segs["len"] = lens
    reqs = np.zeros(nreq, dtype=REQ_DTYPE)
    begins = np.concatenate([[0], np.cumsum(nseg)[:-1]])
    reqs["seg_begin"] = begins
    reqs["seg_count"] = nseg
    reqs["dir"] = rng.integers(0, 2, nreq)
    reqs["guest"] = guest
    L = np.add.reduceat(lens, begins)
    host = np.concatenate([[0], np.cumsum(L + staging_gap)[:-1]])
    reqs["host_off"] = host
    return CopyWorkload(reqs=reqs, segs=segs, staging_bytes=int(host[-1] + L[-1] + staging_gap),
                        batches=[(0, nreq)], payload_bytes=int(lens.sum()))


def split_segments(rng, sizes: np.ndarray, max_segs: int):
    """Cut each request of ``sizes[r]`` bytes into k = min(U[1,max_segs], size)
    pieces of >= 1 B at random cut points.  Returns (nseg per request, lens)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    k = np.minimum(rng.integers(1, max_segs + 1, len(sizes)), sizes)
    req = np.repeat(np.arange(len(sizes)), k - 1)
    # k-1 sorted uniform points in [0, size-k] per request -> k parts >= 0, +1 each.
    pts = (rng.random(len(req)) * (sizes[req] - k[req] + 1)).astype(np.int64)
    order = np.lexsort((pts, req))
    pts = pts[order]
    lens = np.empty(int(k.sum()), dtype=np.int64)
    first = np.concatenate([[0], np.cumsum(k)[:-1]])
    # positions of boundaries: [0, p1, ..., p_{k-1}, size-k] per request
    bnd_start = np.concatenate([[0], np.cumsum(k + 1)[:-1]])
    b = np.empty(int((k + 1).sum()), dtype=np.int64)
    b[bnd_start] = 0
    b[bnd_start + k] = sizes - k
    inner = np.ones(len(b), dtype=bool)
    inner[bnd_start] = False
    inner[bnd_start + k] = False
    b[inner] = pts
    d = np.diff(b)
    keep = np.ones(len(d), dtype=bool)
    keep[(bnd_start + k)[:-1]] = False   # drop the diff across request boundaries
    lens[:] = d[keep] + 1
    assert (np.add.reduceat(lens, first) == sizes).all()
    return k, lens


def batched_requests(img: GuestImage, seed: int, sizes: np.ndarray, max_segs: int,
                     purpose: int = 0, seg_gap_max: int = 4096, page_aligned: bool = False,
                     staging_align: int = 16) -> CopyWorkload:
    """Hazard-free batches on a fault-free guest: every segment gets its own gVA
    range, allocated in request order by a cursor that walks the data region
    with seeded gaps; a request that would run past the region end starts a new
    batch at the region start (sequential composition of batches).  Within a
    batch all guest ranges and all staging ranges are pairwise disjoint, so its
    requests may run in any order.  Staging ranges are per batch, aligned to
    ``staging_align`` and reused by every batch."""
    rng = rng_for(seed, 4, purpose)
    sizes = np.asarray(sizes, dtype=np.int64)
    nreq = len(sizes)
    dirs = rng.integers(0, 2, nreq).astype(np.uint32)
    if max_segs == 1:
        nseg, lens = np.ones(nreq, dtype=np.int64), sizes.copy()
    else:
        nseg, lens = split_segments(rng, sizes, max_segs)
    total = len(lens)
    gaps = rng.integers(0, seg_gap_max + 1, total) if seg_gap_max > 0 else np.zeros(total, np.int64)
    if page_aligned:
        foot = ((lens + PAGE - 1) // PAGE) * PAGE
        gaps[:] = 0
    else:
        foot = lens + gaps
    region = img.data_pages * PAGE
    first = np.concatenate([[0], np.cumsum(nseg)[:-1]]).astype(np.int64)
    req_foot = np.add.reduceat(foot, first)
    assert req_foot.max() <= region, "request larger than the data region"
    # Greedy batch assignment (scalar loop over requests only).
    batch_of_req = np.zeros(nreq, dtype=np.int64)
    req_base = np.zeros(nreq, dtype=np.int64)
    cursor, b = 0, 0
    rf = req_foot.tolist()
    for r in range(nreq):
        if cursor + rf[r] > region:
            b += 1
            cursor = 0
        batch_of_req[r] = b
        req_base[r] = cursor
        cursor += rf[r]
    seg_req = np.repeat(np.arange(nreq), nseg)
    incl = np.cumsum(foot)
    excl_in_req = incl - foot - (incl[first] - foot[first])[seg_req]
    gva = req_base[seg_req] + excl_in_req + (0 if page_aligned else gaps)
    segs = np.zeros(total, dtype=SEG_DTYPE)
    segs["gva"] = img.data_gva + gva
    segs["len"] = lens
    reqs = np.zeros(nreq, dtype=REQ_DTYPE)
    reqs["seg_begin"] = first
    reqs["seg_count"] = nseg
    reqs["dir"] = dirs
    host = np.zeros(nreq, dtype=np.int64)
    batches = []
    staging = 0
    bounds = np.concatenate([[0], np.nonzero(np.diff(batch_of_req))[0] + 1, [nreq]])
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        al = ((sizes[lo:hi] + staging_align - 1) // staging_align) * staging_align
        host[lo:hi] = np.concatenate([[0], np.cumsum(al)[:-1]])
        staging = max(staging, int(al.sum()))
        batches.append((int(lo), int(hi)))
    reqs["host_off"] = host
    return CopyWorkload(reqs=reqs, segs=segs, staging_bytes=staging, batches=batches,
                        payload_bytes=int(lens.sum()))


def batching_sizes(seed: int, nreq: int, purpose: int = 0) -> np.ndarray:
    """80% 16-256 B ioctl structs, 19% 4 KiB-1 MiB command buffers, 1% 1-4 MiB
    (each log-uniform)."""
    rng = rng_for(seed, 5, purpose)
    u = rng.random(nreq)
    s = log_uniform(rng, 16, 256, nreq)
    m = log_uniform(rng, 4096, 1 << 20, nreq)
    l = log_uniform(rng, 1 << 20, 4 << 20, nreq)
    return np.where(u < 0.80, s, np.where(u < 0.99, m, l)).astype(np.int64)


def frame_sizes(seed: int, nreq: int, purpose: int = 0) -> np.ndarray:
    """50/50 1920x1080 and 3840x2160 RGBA8 frames."""
    rng = rng_for(seed, 6, purpose)
    return np.where(rng.random(nreq) < 0.5, 1920 * 1080 * 4, 3840 * 2160 * 4).astype(np.int64)


# ---------------------------------------------------------------------------
# Translation and mmap requests
# ---------------------------------------------------------------------------

def translate_gvas(img: GuestImage, seed: int, n: int, purpose: int = 0) -> np.ndarray:
    """50% uniform mapped page + uniform offset, 45% uniform in the user range
    (the canonical lower half; [0, 2^32) for a PAE guest), 5% uniform u64
    (mostly non-canonical, or beyond 2^32)."""
    rng = rng_for(seed, 7, purpose)
    u = rng.random(n)
    mapped = img.data_gva + rng.integers(0, img.data_pages * PAGE, n, dtype=np.int64).astype(np.uint64)
    user = rng.integers(0, img.va_top, n, dtype=np.int64).astype(np.uint64)
    anyv = rng.integers(0, np.iinfo(np.uint64).max, n, dtype=np.uint64, endpoint=True)
    return np.where(u < 0.5, mapped, np.where(u < 0.95, user, anyv)).astype(np.uint64)


FLAG_CHOICES = np.array([PTE_RW | PTE_US, PTE_US, PTE_RW | PTE_US | MAP_NX, PTE_RW | PTE_US | PTE_PCD,
                         PTE_RW | PTE_US | PTE_G, PTE_RW | PTE_US | PTE_PWT], dtype=np.uint32)


def mmap_requests(img: GuestImage, seed: int, nreq: int, max_pages: int = 512,
                  window_bytes: int = 64 << 30, busy_frac: float = 0.02,
                  bad_flag_frac: float = 0.0, purpose: int = 0):
    """mmap install requests: page-aligned gVA ranges of U[1, max_pages] pages
    uniform in an unmapped 64 GiB user window (overlaps between requests give
    EBUSY on later duplicates); ``busy_frac`` target the mapped data region.
    Host frames are seeded frame numbers inside the host pool.
    Returns (MAPREQ_DTYPE array, hf uint64 array, window base gva)."""
    rng = rng_for(seed, 8, purpose)
    gap = 0 if img.paging == PAGING_PAE else 1    # a PAE space is only 4 GiB
    win = img.data_gva + ((img.data_pages * PAGE + (1 << 30) - 1) // (1 << 30) + gap) * (1 << 30)
    assert win + window_bytes <= img.va_top
    npg = rng.integers(1, max_pages + 1, nreq)
    start = rng.integers(0, window_bytes // PAGE - max_pages, nreq) * PAGE + win
    busy = rng.random(nreq) < busy_frac
    bstart = img.data_gva + rng.integers(0, img.data_pages - max_pages, nreq) * PAGE
    start = np.where(busy, bstart, start)
    flags = FLAG_CHOICES[rng.integers(0, len(FLAG_CHOICES), nreq)]
    bad = rng.random(nreq) < bad_flag_frac
    flags = np.where(bad, flags | np.uint32(PTE_PS), flags).astype(np.uint32)
    reqs = np.zeros(nreq, dtype=MAPREQ_DTYPE)
    reqs["gva"] = start
    reqs["npages"] = npg
    reqs["flags"] = flags
    reqs["hf_begin"] = np.concatenate([[0], np.cumsum(npg)[:-1]])
    pool_frames = img.pool_bytes // PAGE
    hf = rng.integers(0, pool_frames, int(npg.sum()), dtype=np.int64).astype(np.uint64)
    return reqs, hf, win


def place_requests(img: GuestImage, seed: int, nreq: int, max_pages: int = 512, bad_flag_frac: float = 0.0,
                   purpose: int = 0):
    """Driver-initiated map requests (Sec. 6.6): U[1, max_pages] pages each,
    no address, flags from the mmap mix (``bad_flag_frac`` with PS added,
    which is malformed), seeded host frames inside the pool.  Returns
    (PLACE_DTYPE array, hf uint64 array)."""
    rng = rng_for(seed, 12, purpose)
    npg = rng.integers(1, max_pages + 1, nreq)
    flags = FLAG_CHOICES[rng.integers(0, len(FLAG_CHOICES), nreq)]
    bad = rng.random(nreq) < bad_flag_frac
    flags = np.where(bad, flags | np.uint32(PTE_PS), flags).astype(np.uint32)
    reqs = np.zeros(nreq, dtype=PLACE_DTYPE)
    reqs["npages"] = npg
    reqs["flags"] = flags
    reqs["hf_begin"] = np.concatenate([[0], np.cumsum(npg)[:-1]])
    hf = rng.integers(0, img.pool_bytes // PAGE, int(npg.sum()), dtype=np.int64).astype(np.uint64)
    return reqs, hf


def host_of_gva(img: GuestImage, gva: int) -> int:
    """Host-pool offset of a byte of the data region, from the generator's
    own record of where it placed every page (memslot image; the page may be
    one whose leaf is not present)."""
    p = (gva - img.data_gva) // PAGE
    g = int(img.page_gfn[p])
    if g < 0:
        g = int(img.huge_gfn[p // 512]) + p % 512
    return img.gpa_to_host((g << PAGE_SHIFT) + gva % PAGE)


def write_gva(img: GuestImage, pool: np.ndarray, gva: int, data: np.ndarray):
    """Write bytes at a data-region gVA into the pool, page by page."""
    data = np.ascontiguousarray(data).view(np.uint8).reshape(-1)
    done = 0
    while done < len(data):
        va = gva + done
        n = min(len(data) - done, PAGE - va % PAGE)
        h = host_of_gva(img, va)
        pool[h:h + n] = data[done:done + n]
        done += n


def host_of_gva_array(img: GuestImage, gva: np.ndarray) -> np.ndarray:
    """host_of_gva for an array of data-region addresses."""
    gva = np.asarray(gva, dtype=np.int64)
    p = (gva - img.data_gva) // PAGE
    g = img.page_gfn[p].copy()
    hp = g < 0
    g[hp] = img.huge_gfn[p[hp] // 512] + p[hp] % 512
    gpa = (g << PAGE_SHIFT) + gva % PAGE
    base = img.slots["base_gfn"].astype(np.int64)
    order = np.argsort(base)
    k = order[np.searchsorted(base[order], g, side="right") - 1]
    return img.slots["host_off"].astype(np.int64)[k] + gpa - (base[k] << PAGE_SHIFT)


@dataclasses.dataclass
class ChainWorkload:
    reqs: np.ndarray          # CHAIN_REQ_DTYPE
    entries: np.ndarray       # uint64 [entries, 2]: {gva, len} of every table, tables in request order
    first: np.ndarray         # int64 [nreq + 1]: first entry of each request's table
    desc_bytes: int
    payload_bytes: int        # sum of the entries' lengths

    @property
    def tables(self):
        """(gva, uint8 bytes) of every descriptor table."""
        return [(int(self.reqs["table_gva"][r]),
                 self.entries[self.first[r]:self.first[r + 1]].reshape(-1).view(np.uint8))
                for r in range(len(self.reqs))]

    def entry_gvas(self) -> np.ndarray:
        """gVA of every entry (16-byte aligned, so none crosses a page)."""
        cnt = np.diff(self.first)
        return (np.repeat(self.reqs["table_gva"].astype(np.int64), cnt) +
                16 * (np.arange(len(self.entries)) - np.repeat(self.first[:-1], cnt)))


def chained_requests(img: GuestImage, seed: int, nreq: int, max_count: int = 32, lo: int = 64,
                     hi: int = 65536, table_area: float = 0.05, purpose: int = 0) -> ChainWorkload:
    """DRM-style command submissions (generic class drivers, Sec. 6.1): each
    request names a descriptor table of U[1, max_count] entries {gva, len},
    lengths log-uniform in [lo, hi], buffers uniform in the data region past
    its first ``table_area`` fraction; tables packed at 16-byte aligned
    places (U[0, 256] B gaps) in that first fraction, so they never overlap
    one another; desc_off packs the tables back to back."""
    rng = rng_for(seed, 13, purpose)
    region = img.data_pages * PAGE
    t_end = int(region * table_area) // 16 * 16
    count = rng.integers(1, max_count + 1, nreq).astype(np.int64)
    gaps = rng.integers(0, 17, nreq).astype(np.int64) * 16
    ends = np.cumsum(gaps + 16 * count)
    starts = ends - 16 * count
    assert nreq == 0 or ends[-1] <= t_end, "table area too small"
    total = int(count.sum())
    lens = log_uniform(rng, lo, hi, total)
    offs = t_end + (rng.random(total) * (region - t_end - lens)).astype(np.int64)
    entries = np.zeros((total, 2), dtype=np.uint64)
    entries[:, 0] = img.data_gva + offs
    entries[:, 1] = lens
    first = np.concatenate([[0], np.cumsum(count)]).astype(np.int64)
    reqs = np.zeros(nreq, dtype=CHAIN_REQ_DTYPE)
    reqs["table_gva"] = img.data_gva + starts
    reqs["count"] = count
    reqs["desc_off"] = 16 * first[:-1]
    return ChainWorkload(reqs=reqs, entries=entries, first=first, desc_bytes=16 * total,
                         payload_bytes=int(lens.sum()))
