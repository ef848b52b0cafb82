// cvd_device.cuh -- device-side guest model, software page walk and warp copy
// primitives for the CVD memory operations on sm_103a.
//
// Paper: Sec. 4.2 (software hybrid address space: walk the guest page tables
// in software, then KVM memslot gPA -> host, once per page), Sec. 6.2-6.3
// (redirected memory routines; page-table root captured per guest process).
// Format: x86-64 4-level paging (Intel SDM Vol. 3 ch. 4).  Second dimension:
// memslots (KVM), or a software walk of an EPT (Sec. 4.2 on other
// hypervisors; Intel SDM Vol. 3 sec. 28.3.2).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cvd {

constexpr int kMaxSlots = 64;
// Unit tables (translate kernel): for guests whose memslots all start and end
// on 2 MiB guest-frame boundaries below 32 GiB, every 2 MiB unit of guest
// memory up to the last slot's end has its host-frame delta (host frame -
// guest frame, kNoUnitDelta: no slot) and its slot (kNoUnit: none), so a
// gPA -> host lookup is one load and one add instead of a binary search.
constexpr uint32_t kUnitSlots = 16384;   // units covered at most (32 GiB)
constexpr uint8_t kNoUnit = 0xFF;
constexpr int32_t kNoUnitDelta = INT32_MIN;
constexpr uint64_t kPage = 4096;
constexpr uint64_t kUserTop = 1ull << 47;
constexpr uint64_t kAllOnes = ~0ull;

constexpr uint64_t kP = 1ull << 0, kRW = 1ull << 1, kUS = 1ull << 2, kPS = 1ull << 7;
constexpr uint64_t kFrame4K = 0x000FFFFFFFFFF000ull;  // bits 51:12
constexpr uint64_t kFrame2M = 0x000FFFFFFFE00000ull;  // bits 51:21
constexpr uint64_t kFrame1G = 0x000FFFFFC0000000ull;  // bits 51:30

enum Fault : uint32_t {
  kOk = 0, kNotPresent = 1, kWriteProtect = 2, kNonCanonical = 3, kRange = 4,
  kNoSlot = 5, kRsvd = 6, kUser = 7, kHostBuf = 8, kBadReq = 9, kEptViolation = 10
};

struct DevSlot { uint64_t base_gfn, npages, host_off; };

// Guest paging formats: x86-64 4-level, and 32-bit PAE (3 levels from a
// 4-entry page directory pointer table; the paging of the paper's own
// implementation, Sec. 6.2).
constexpr uint32_t kPagingX86_64 = 0, kPagingPae = 1;
constexpr uint64_t kPaeTop = 1ull << 32;
// PDPTE bits reserved in PAE paging (RW, US, and bits 5..8 including PS).
constexpr uint64_t kPaePdpteRsvd = (1ull << 1) | (1ull << 2) | (0xFull << 5);

// Library-owned device descriptor of one guest (one per cvd_guest handle).
struct DevGuest {
  uint8_t* pool;
  uint64_t pool_bytes;
  uint64_t cr3_gpa;
  uint64_t rsv_gfn, rsv_n;
  uint64_t* p2m;
  uint64_t pt_pool_gfn, pt_pool_n;
  uint64_t* alloc;          // [0] = PT-pool frames used, [1] = reserved frames used
  uint32_t nslots;
  uint32_t paging;          // kPagingX86_64 or kPagingPae
  uint32_t ept;             // 1: second dimension = software EPT walk (nslots = 0)
  uint32_t pad0;
  uint64_t ept_root;        // host-pool byte offset of the EPT PML4 (4 KiB aligned)
  DevSlot slots[kMaxSlots]; // sorted by base_gfn, non-overlapping
  uint32_t nunits;           // units covered by the unit tables (0: no tables)
  const int32_t* unit_delta; // device i32[nunits rounded up to 4] (library owned, 16-byte aligned)
  const uint8_t* unit_slot;  // device u8[nunits]
};

// Request / result records (same layout as include/cvd.h).
struct Seg { uint64_t gva, len; };
struct Req { uint32_t seg_begin, seg_count, dir, guest; uint64_t host_off; };
struct Result { uint64_t done, fault_gva; uint32_t fault_code, pad; };

// Per-segment work record written by the planner (32 B).
struct SegWork {
  uint64_t gva;
  uint64_t soff;    // stream offset of the segment's first byte in its request
  uint64_t len;     // segment length
  uint64_t ncopy;   // bytes of this segment before the request's first fault
};
// Per-request work record written by the planner.
struct ReqWork {
  uint64_t host_off;
  uint64_t sb;      // first SegWork index
  uint32_t nsw;     // SegWork entries (0: request copies nothing)
  uint32_t guest_dir;  // guest index << 1 | dir
};

// Warp-wide reductions and scans (all 32 lanes participate).
__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t t = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += t;
  }
  return v;
}
__device__ __forceinline__ uint64_t warp_sat_sum(uint64_t v) {
#pragma unroll
  for (int d = 16; d; d >>= 1) {
    uint64_t t = __shfl_xor_sync(0xffffffffu, v, d);
    v = (v + t < v) ? ~0ull : v + t;
  }
  return v;
}
__device__ __forceinline__ uint64_t warp_max(uint64_t v) {
#pragma unroll
  for (int d = 16; d; d >>= 1) { uint64_t t = __shfl_xor_sync(0xffffffffu, v, d); v = t > v ? t : v; }
  return v;
}
__device__ __forceinline__ uint64_t warp_min(uint64_t v) {
#pragma unroll
  for (int d = 16; d; d >>= 1) { uint64_t t = __shfl_xor_sync(0xffffffffu, v, d); v = t < v ? t : v; }
  return v;
}

// Work distribution over the request-cost stream (planner and copy engines).
// Next window [cs, ce) of the cost stream [0, total), taken from a shared byte
// cursor (guided self-scheduling): windows are `chunk` long while plenty of
// work is left, then shrink to 1/(2 x warps) of what remains, down to
// chunk/16, so that the warps run out of work at about the same time instead
// of idling behind the last full-size windows.  A stale read of the cursor
// only makes a window a little longer.  All lanes call it; false when no
// work is left.
__device__ __forceinline__ bool next_chunk(unsigned long long* cursor, uint64_t total, uint64_t chunk,
                                           uint64_t nwarps, int lane, uint64_t* cs, uint64_t* ce) {
  uint64_t start = 0, len = 0;
  if (lane == 0) {
    uint64_t cur = *reinterpret_cast<volatile unsigned long long*>(cursor);
    uint64_t rem = cur < total ? total - cur : 0;
    uint64_t lo = chunk >> 4;
    len = rem / (2 * nwarps);
    len = len < lo ? lo : (len > chunk ? chunk : len);
    start = atomicAdd(cursor, (unsigned long long)len);
  }
  start = __shfl_sync(0xffffffffu, start, 0);
  len = __shfl_sync(0xffffffffu, len, 0);
  if (start >= total) return false;
  *cs = start;
  *ce = start + len < total ? start + len : total;
  return true;
}

// Last request index r in [0, n) with R[r] <= b (R = exclusive stream starts,
// the odd words of pairs_out).  32-ary warp search: ~4 rounds for 1M requests.
__device__ __forceinline__ uint64_t find_req(const uint64_t* pairs_out, uint64_t n, uint64_t b, int lane) {
  uint64_t lo = 0, hi = n;  // answer in [lo, hi)
  while (hi - lo > 1) {
    uint64_t step = (hi - lo + 31) / 32;
    uint64_t p = lo + (uint64_t)lane * step;
    bool ok = p < hi && pairs_out[2 * p + 1] <= b;
    unsigned m = __ballot_sync(0xffffffffu, ok);
    int t = 31 - __clz(m);   // lane 0 always ok: R[lo] <= b
    lo = lo + (uint64_t)t * step;
    uint64_t nhi = lo + step;
    hi = nhi < hi ? nhi : hi;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Shared-memory staging of the top two levels (one guest per launch).
// ---------------------------------------------------------------------------
constexpr int kTopPdpt = 2;   // PDPT tables staged per CTA

struct TopCache {
  uint64_t pml4[512];
  uint64_t pdpt[kTopPdpt][512];
  uint32_t pdpt_idx4[kTopPdpt];   // PML4 index each staged PDPT hangs from (~0: none)
  DevSlot slots[kMaxSlots];
  uint32_t nslots;
  uint32_t valid;                  // PML4 staged
  uint32_t paging;                 // the guest's paging format (kPaging*)
  uint32_t cand[16];               // staging scratch: PML4 entries that can hang a staged PDPT
  uint32_t ept;                    // the guest's second dimension is an EPT
  uint64_t ept_root;
  const struct EptTop* et;         // staged EPT top levels (EPT launches), or null
};

// The EPT's root table and the first usable table below it, staged in shared
// memory by launches over a guest behind an EPT (the EPT does not change
// during a call, so staged entries equal the entries a walk would load).
struct EptTop {
  uint64_t l4[512];
  uint64_t l3[512];    // the table hanging from l4[l3_i4]
  uint32_t l3_i4;      // ~0: none staged
  uint32_t pad;
};
constexpr size_t kTopCacheBytes = ((sizeof(TopCache) + 127) / 128) * 128;
constexpr size_t kEptTopBytes = ((sizeof(EptTop) + 127) / 128) * 128;

// EPT unit entries (translate kernel): for every 2 MiB unit of gPA [0, 4 GiB),
// staged right after the EptTop, the level-2 entry the walk reaches with the
// write bit ANDed over levels 4..2, 0 when the walk ends unusable above or at
// level 2, or kEptUnitWalk when a 1 GiB leaf at level 3 maps the unit (the
// walk then starts from the root).  A usable entry has bit 0 set, so the
// marker (bit 0 clear, bit 1 set) is never one.
constexpr uint32_t kEptUnits = 2048;
constexpr uint64_t kEptUnitWalk = 2;
constexpr size_t kEptUnitBytes = (size_t)kEptUnits * 8;

struct WalkOut {
  uint64_t gpa, hpa;
  uint64_t span;    // bytes from va on which hpa stays contiguous and valid
  uint32_t code;
};

__device__ __forceinline__ bool canonical(uint64_t va) {
  uint64_t top = va >> 47;
  return top == 0 || top == 0x1FFFFull;
}

// gPA -> hPA: reserved window through the p2m, else the memslot containing
// the frame (binary search over slots sorted by base_gfn).  *lim = gPA bytes
// from gpa to the end of the backing region (slot end or 4 KiB page end).
__device__ __forceinline__ bool gpa_to_hpa(const DevGuest& g, const DevSlot* slots, uint32_t nslots,
                                           uint64_t gpa, uint64_t* hpa, uint64_t* lim) {
  uint64_t gfn = gpa >> 12;
  if (gfn >= g.rsv_gfn && gfn - g.rsv_gfn < g.rsv_n) {
    uint64_t hf = g.p2m[gfn - g.rsv_gfn];
    if (hf == kAllOnes || hf >= (g.pool_bytes >> 12)) return false;
    *hpa = (hf << 12) | (gpa & 4095);
    *lim = kPage - (gpa & 4095);
    return true;
  }
  int lo = 0, hi = (int)nslots - 1, found = -1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    if (slots[mid].base_gfn <= gfn) { found = mid; lo = mid + 1; } else hi = mid - 1;
  }
  if (found < 0) return false;
  DevSlot s = slots[found];
  if (gfn - s.base_gfn >= s.npages) return false;
  uint64_t rel = gpa - (s.base_gfn << 12);
  *hpa = s.host_off + rel;
  *lim = (s.npages << 12) - rel;
  return true;
}

// gPA -> hPA through a software EPT (Intel SDM Vol. 3 sec. 28.3.2): 4 levels
// indexed by gPA bits 47:39 / 38:30 / 29:21 / 20:12 from the root at host
// pool offset `root`; an entry is usable when its read bit (0) is set; the
// write bit (1) is ANDed over the levels; bit 7 makes a 1 GiB / 2 MiB leaf at
// levels 3 / 2 and is reserved (entry unusable) at level 4; addresses are
// host-pool byte offsets.  A page is backed only when its whole 4 KiB host
// frame lies in the pool.  Reserved frames still go through the p2m first.
// Returns kOk (*hpa, *lim = bytes to the end of the leaf or of the pool's
// last whole frame), kNoSlot (not backed) or kEptViolation (write through a
// mapping without write permission).  The EPT does not change during a call.
__device__ __forceinline__ uint32_t ept_walk(const DevGuest& g, uint64_t root, uint64_t gpa, bool write,
                                             uint64_t* hpa, uint64_t* lim, const EptTop* et) {
  const uint64_t gfn = gpa >> 12;
  if (gfn >= g.rsv_gfn && gfn - g.rsv_gfn < g.rsv_n) {
    uint64_t hf = g.p2m[gfn - g.rsv_gfn];
    if (hf == kAllOnes || hf >= (g.pool_bytes >> 12)) return kNoSlot;
    *hpa = (hf << 12) | (gpa & 4095);
    *lim = kPage - (gpa & 4095);
    return kOk;
  }
  if (gpa >> 48) return kNoSlot;
  const uint64_t pool_end = g.pool_bytes & ~4095ull;   // end of the last whole frame
  uint64_t table = root, w = 2;
#pragma unroll
  for (int level = 4; level >= 1; level--) {
    const uint32_t idx = (uint32_t)(gpa >> (3 + 9 * level)) & 511;
    const uint64_t at = table + 8ull * idx;
    uint64_t e;
    if (et && level == 4) {
      e = et->l4[idx];
    } else if (et && level == 3 && et->l3_i4 == ((uint32_t)(gpa >> 39) & 511)) {
      e = et->l3[idx];
    } else {
      if (at + 8 > g.pool_bytes) return kNoSlot;
      e = __ldg(reinterpret_cast<const unsigned long long*>(g.pool + at));
    }
    if (!(e & 1)) return kNoSlot;
    w &= e;
    const bool big = (e >> 7) & 1;
    if (level == 4 && big) return kNoSlot;
    if (level == 1 || big) {
      const uint64_t size = 1ull << (3 + 9 * level);
      const uint64_t h = (e & kFrame4K & ~(size - 1)) | (gpa & (size - 1));
      if ((h & ~4095ull) + kPage > pool_end) return kNoSlot;
      if (write && !(w & 2)) return kEptViolation;
      const uint64_t left = size - (gpa & (size - 1)), room = pool_end - h;
      *hpa = h;
      *lim = left < room ? left : room;
      return kOk;
    }
    table = e & kFrame4K;
  }
  return kNoSlot;
}

// ept_walk for the translate kernel, whose launch staged the EPT unit entries
// (stage_ept_units) after the EptTop: the same result.  A separate function
// keeps the planner's and copy engine's EPT walk as it was (the shared
// version cost the planner registers).
__device__ __forceinline__ uint32_t ept_walk_units(const DevGuest& g, uint64_t root, uint64_t gpa, bool write,
                                             uint64_t* hpa, uint64_t* lim, const EptTop* et) {
  const uint64_t gfn = gpa >> 12;
  if (gfn >= g.rsv_gfn && gfn - g.rsv_gfn < g.rsv_n) {
    uint64_t hf = g.p2m[gfn - g.rsv_gfn];
    if (hf == kAllOnes || hf >= (g.pool_bytes >> 12)) return kNoSlot;
    *hpa = (hf << 12) | (gpa & 4095);
    *lim = kPage - (gpa & 4095);
    return kOk;
  }
  if (gpa >> 48) return kNoSlot;
  const uint64_t pool_end = g.pool_bytes & ~4095ull;   // end of the last whole frame
  uint64_t table = root, w = 2;
  // the staged unit entry stands for levels 4..2 (see kEptUnits)
  int top = 4;
  uint64_t e_unit = 0;
  if (et && (gpa >> 21) < kEptUnits) {
    const uint64_t v = reinterpret_cast<const uint64_t*>(reinterpret_cast<const uint8_t*>(et) + kEptTopBytes)[gpa >> 21];
    if (v != kEptUnitWalk) {
      if (!(v & 1)) return kNoSlot;
      top = 2;
      e_unit = v;
    }
  }
#pragma unroll
  for (int level = 4; level >= 1; level--) {
    if (level > top) continue;
    const uint32_t idx = (uint32_t)(gpa >> (3 + 9 * level)) & 511;
    const uint64_t at = table + 8ull * idx;
    uint64_t e;
    if (level == 2 && top == 2) {
      e = e_unit;
    } else if (et && level == 4) {
      e = et->l4[idx];
    } else if (et && level == 3 && et->l3_i4 == ((uint32_t)(gpa >> 39) & 511)) {
      e = et->l3[idx];
    } else {
      if (at + 8 > g.pool_bytes) return kNoSlot;
      e = __ldg(reinterpret_cast<const unsigned long long*>(g.pool + at));
    }
    if (!(e & 1)) return kNoSlot;
    w &= e;
    const bool big = (e >> 7) & 1;
    if (level == 4 && big) return kNoSlot;
    if (level == 1 || big) {
      const uint64_t size = 1ull << (3 + 9 * level);
      const uint64_t h = (e & kFrame4K & ~(size - 1)) | (gpa & (size - 1));
      if ((h & ~4095ull) + kPage > pool_end) return kNoSlot;
      if (write && !(w & 2)) return kEptViolation;
      const uint64_t left = size - (gpa & (size - 1)), room = pool_end - h;
      *hpa = h;
      *lim = left < room ? left : room;
      return kOk;
    }
    table = e & kFrame4K;
  }
  return kNoSlot;
}

// The same walk out of line: the copy engine and the planner keep their hot
// loops smaller with the EPT walk as a call (inlined, translate ran 1.5x
// faster and the copy engine 5% slower).
static __device__ __noinline__ uint32_t ept_to_hpa(const DevGuest& g, uint64_t root, uint64_t gpa, bool write,
                                                   uint64_t* hpa, uint64_t* lim, const EptTop* et) {
  return ept_walk(g, root, gpa, write, hpa, lim, et);
}

// gPA -> hPA through the staged unit deltas (ut: {u32 nunits, pad to 16 B,
// i32 delta[nunits]}; the guest has unit tables): the same result as
// gpa_to_hpa.  A unit lies wholly inside one slot or outside all of them, and
// the reserved window overlaps no slot, so the window is looked at only for
// units without a slot.  The span (*lim) reads the unit's slot from the
// device table; callers that use only *hpa leave that load out.
__device__ __forceinline__ bool gpa_to_hpa_units(const DevGuest& g, const DevSlot* slots, const uint8_t* ut,
                                                 uint64_t gpa, uint64_t* hpa, uint64_t* lim) {
  const uint64_t u = gpa >> 21;
  if (u < *reinterpret_cast<const uint32_t*>(ut)) {
    const int32_t d = reinterpret_cast<const int32_t*>(ut + 16)[u];
    if (d != kNoUnitDelta) {
      *hpa = gpa + ((uint64_t)(int64_t)d << 12);
      const DevSlot& sl = slots[g.unit_slot[u]];
      *lim = ((sl.base_gfn + sl.npages) << 12) - gpa;
      return true;
    }
  }
  const uint64_t gfn = gpa >> 12;
  if (gfn - g.rsv_gfn < g.rsv_n) {   // the window does not wrap (checked at create)
    const uint64_t hf = g.p2m[gfn - g.rsv_gfn];
    if (hf == kAllOnes || hf >= (g.pool_bytes >> 12)) return false;
    *hpa = (hf << 12) | (gpa & 4095);
    *lim = kPage - (gpa & 4095);
    return true;
  }
  return false;
}

// Second dimension chosen when a walk is compiled: kSdSlots = memslots (and
// the p2m) only; kSdAny = the guest's own choice, read per call (EPT walk
// out of line); kSdAnyInl = the same with the EPT walk inlined; kSdUnits =
// memslots through the staged unit table.
constexpr int kSdSlots = 0, kSdAny = 1, kSdAnyInl = 2, kSdUnits = 3;

template <int SD>
__device__ __forceinline__ uint32_t to_host(const DevGuest& g, const TopCache* tc, const DevSlot* slots,
                                            uint32_t nslots, uint64_t gpa, bool write, uint64_t* hpa, uint64_t* lim) {
  if ((SD == kSdAny || SD == kSdAnyInl) && (tc ? tc->ept : g.ept)) {
    if (SD == kSdAnyInl)   // the translate kernel: EPT unit entries staged (stage_ept_units)
      return ept_walk_units(g, tc ? tc->ept_root : g.ept_root, gpa, write, hpa, lim, tc ? tc->et : nullptr);
    return ept_to_hpa(g, tc ? tc->ept_root : g.ept_root, gpa, write, hpa, lim, tc ? tc->et : nullptr);
  }
  // the unit table sits right after the top cache (stage_units)
  if (SD == kSdUnits)
    return gpa_to_hpa_units(g, slots, reinterpret_cast<const uint8_t*>(tc) + kTopCacheBytes, gpa, hpa, lim) ? kOk
                                                                                                          : kNoSlot;
  return gpa_to_hpa(g, slots, nslots, gpa, hpa, lim) ? kOk : kNoSlot;
}

// Page tables are read-only for the duration of a launch (they change only
// in the mmap-install kernels), so entries go through the read-only path.
// A table read needs read access only (behind an EPT too).
template <int SD>
__device__ __forceinline__ bool read_entry(const DevGuest& g, const TopCache* tc, const DevSlot* slots,
                                           uint32_t nslots, uint64_t table_gpa, uint32_t idx, uint64_t* e) {
  uint64_t h, lim;
  if (to_host<SD>(g, tc, slots, nslots, table_gpa + 8ull * idx, false, &h, &lim) != kOk) return false;
  *e = __ldg(reinterpret_cast<const unsigned long long*>(g.pool + h));
  return true;
}

// Address checks of a guest's virtual space: a 4-level guest's user buffers
// lie in the canonical lower half [0, 2^47); a PAE guest's whole space is
// [0, 2^32) and has no non-canonical addresses.
__device__ __forceinline__ bool va_canonical(const DevGuest& g, uint64_t va) {
  return g.paging == kPagingPae || canonical(va);
}
__device__ __forceinline__ uint64_t va_top(const DevGuest& g) { return g.paging == kPagingPae ? kPaeTop : kUserTop; }

// Software walk of a 32-bit PAE guest (Intel SDM Vol. 3 sec. 4.4).  The
// staged copy, when present, holds the 4 PDPTEs (in pml4[0..3]) and the first
// kTopPdpt present page directories (pdpt[k] for PDPT index pdpt_idx4[k]).
// Levels: PDPTE 3, PDE 2, PTE 1; a present PDPTE with reserved bits -> RSVD;
// RW and US come from the PDE and the PTE only.
template <int SD>
static __device__ __noinline__ WalkOut walk_pae(const DevGuest& g, const TopCache* tc, uint64_t va, bool write) {
  WalkOut o;
  o.gpa = kAllOnes; o.hpa = kAllOnes; o.span = 0;
  if (va >= kPaeTop) { o.code = kRange; return o; }
  const DevSlot* slots = tc ? tc->slots : g.slots;
  const uint32_t nslots = tc ? tc->nslots : g.nslots;
  const uint32_t i3 = (va >> 30) & 3, i2 = (va >> 21) & 511, i1 = (va >> 12) & 511;
  uint64_t e;
  if (tc && tc->valid) e = tc->pml4[i3];
  else if (!read_entry<SD>(g, tc, slots, nslots, g.cr3_gpa & ~31ull, i3, &e)) { o.code = kNoSlot; return o; }
  if (!(e & kP)) { o.code = kNotPresent | (3u << 8); return o; }
  if (e & kPaePdpteRsvd) { o.code = kRsvd; return o; }
  int st = -1;
  if (tc && tc->valid) {
#pragma unroll
    for (int k = 0; k < kTopPdpt; k++) if (tc->pdpt_idx4[k] == i3) st = k;
  }
  if (st >= 0) e = tc->pdpt[st][i2];
  else if (!read_entry<SD>(g, tc, slots, nslots, e & kFrame4K, i2, &e)) { o.code = kNoSlot; return o; }
  if (!(e & kP)) { o.code = kNotPresent | (2u << 8); return o; }
  bool rw = (e >> 1) & 1, us = (e >> 2) & 1;
  uint64_t gpa, leaf_left;
  if (e & kPS) {
    gpa = (e & kFrame2M) | (va & ((1ull << 21) - 1));
    leaf_left = (1ull << 21) - (va & ((1ull << 21) - 1));
  } else {
    if (!read_entry<SD>(g, tc, slots, nslots, e & kFrame4K, i1, &e)) { o.code = kNoSlot; return o; }
    if (!(e & kP)) { o.code = kNotPresent | (1u << 8); return o; }
    rw &= (e >> 1) & 1; us &= (e >> 2) & 1;
    gpa = (e & kFrame4K) | (va & 4095);
    leaf_left = kPage - (va & 4095);
  }
  if (!us) { o.code = kUser; return o; }
  if (write && !rw) { o.code = kWriteProtect; return o; }
  uint64_t h, lim;
  const uint32_t c = to_host<SD>(g, tc, slots, nslots, gpa, write, &h, &lim);
  if (c != kOk) { o.code = c; return o; }
  o.gpa = gpa; o.hpa = h;
  o.span = leaf_left < lim ? leaf_left : lim;
  o.code = kOk;
  return o;
}

// Software walk of a 4-level guest (Sec. 4.2).  tc may be null (no staging).
// Levels 4 and 3 come from shared memory when staged; the result is identical
// either way since staging copies exactly the entries a walk would read
// through the memslots.
template <int SD>
__device__ __forceinline__ WalkOut walk4(const DevGuest& g, const TopCache* tc, uint64_t va, bool write) {
  WalkOut o;
  o.gpa = kAllOnes; o.hpa = kAllOnes; o.span = 0;
  if (!canonical(va)) { o.code = kNonCanonical; return o; }
  if (va >= kUserTop) { o.code = kRange; return o; }
  const DevSlot* slots = tc ? tc->slots : g.slots;
  uint32_t nslots = tc ? tc->nslots : g.nslots;
  uint32_t i4 = (va >> 39) & 511, i3 = (va >> 30) & 511, i2 = (va >> 21) & 511, i1 = (va >> 12) & 511;
  uint64_t e;
  bool rw = true, us = true;
  // level 4
  if (tc && tc->valid) e = tc->pml4[i4];
  else if (!read_entry<SD>(g, tc, slots, nslots, g.cr3_gpa & kFrame4K, i4, &e)) { o.code = kNoSlot; return o; }
  if (!(e & kP)) { o.code = kNotPresent | (4u << 8); return o; }
  if (e & kPS) { o.code = kRsvd; return o; }
  rw &= (e >> 1) & 1; us &= (e >> 2) & 1;
  // level 3
  int st = -1;
  if (tc && tc->valid) {
#pragma unroll
    for (int k = 0; k < kTopPdpt; k++) if (tc->pdpt_idx4[k] == i4) st = k;
  }
  uint64_t t3 = e & kFrame4K;
  if (st >= 0) e = tc->pdpt[st][i3];
  else if (!read_entry<SD>(g, tc, slots, nslots, t3, i3, &e)) { o.code = kNoSlot; return o; }
  if (!(e & kP)) { o.code = kNotPresent | (3u << 8); return o; }
  rw &= (e >> 1) & 1; us &= (e >> 2) & 1;
  uint64_t gpa, leaf_left;
  if (e & kPS) {
    gpa = (e & kFrame1G) | (va & ((1ull << 30) - 1));
    leaf_left = (1ull << 30) - (va & ((1ull << 30) - 1));
  } else {
    if (!read_entry<SD>(g, tc, slots, nslots, e & kFrame4K, i2, &e)) { o.code = kNoSlot; return o; }
    if (!(e & kP)) { o.code = kNotPresent | (2u << 8); return o; }
    rw &= (e >> 1) & 1; us &= (e >> 2) & 1;
    if (e & kPS) {
      gpa = (e & kFrame2M) | (va & ((1ull << 21) - 1));
      leaf_left = (1ull << 21) - (va & ((1ull << 21) - 1));
    } else {
      if (!read_entry<SD>(g, tc, slots, nslots, e & kFrame4K, i1, &e)) { o.code = kNoSlot; return o; }
      if (!(e & kP)) { o.code = kNotPresent | (1u << 8); return o; }
      rw &= (e >> 1) & 1; us &= (e >> 2) & 1;
      gpa = (e & kFrame4K) | (va & 4095);
      leaf_left = kPage - (va & 4095);
    }
  }
  if (!us) { o.code = kUser; return o; }
  if (write && !rw) { o.code = kWriteProtect; return o; }
  uint64_t h, lim;
  const uint32_t c = to_host<SD>(g, tc, slots, nslots, gpa, write, &h, &lim);
  if (c != kOk) { o.code = c; return o; }
  o.gpa = gpa; o.hpa = h;
  o.span = leaf_left < lim ? leaf_left : lim;
  o.code = kOk;
  return o;
}

// Paging dispatch fixed when a kernel is compiled: a launch over memslot
// guests of one format knows it on the host (kPmX86 / kPmPae); a launch over
// memslot guests of several formats decides the format per walk (kPmAny); a
// launch with a guest behind an EPT decides format and second dimension per
// walk (kPmEpt).  A per-walk test on the hot single-guest paths cost 1% of
// the copy engine and 10% of the planner.
// kPmEptT: kPmEpt with the EPT walk inlined (the translate kernel); kPmX86U
// and kPmPaeU: kPmX86 and kPmPae with memslot lookups through the unit
// tables (the translate kernel).
constexpr int kPmX86 = 0, kPmPae = 1, kPmAny = 2, kPmEpt = 3, kPmEptT = 4, kPmX86U = 5, kPmPaeU = 6;

// Whether a paging mode looks memslots up through the staged unit tables.
__host__ __device__ constexpr bool pm_units(int PM) { return PM == kPmX86U || PM == kPmPaeU; }

// The second dimension a paging mode compiles in.
template <int PM> struct SdOf {
  static constexpr int v = PM == kPmEptT ? kSdAnyInl : (PM == kPmEpt ? kSdAny : (pm_units(PM) ? kSdUnits : kSdSlots));
};
// Whether a paging mode reads the guest's format per walk.
__host__ __device__ constexpr bool pm_runtime(int PM) { return PM == kPmAny || PM == kPmEpt || PM == kPmEptT; }

template <int PM>
__device__ __forceinline__ WalkOut walk_t(const DevGuest& g, const TopCache* tc, uint64_t va, bool write) {
  constexpr int SD = SdOf<PM>::v;
  if (PM == kPmX86) return walk4<kSdSlots>(g, tc, va, write);
  if (PM == kPmX86U) return walk4<kSdUnits>(g, tc, va, write);
  if (PM == kPmPae) return walk_pae<kSdSlots>(g, tc, va, write);
  if (PM == kPmPaeU) return walk_pae<kSdUnits>(g, tc, va, write);
  return ((tc ? tc->paging : g.paging) == kPagingPae) ? walk_pae<SD>(g, tc, va, write)
                                                       : walk4<SD>(g, tc, va, write);
}

// Walk with the format and the second dimension read from the guest (cold paths).
__device__ __forceinline__ WalkOut walk(const DevGuest& g, const TopCache* tc, uint64_t va, bool write) {
  return walk_t<kPmEpt>(g, tc, va, write);
}

// N independent walks advanced level by level in lockstep: at each level the
// entries of every walk still at that level are read before any is examined,
// so a thread keeps N table reads in flight instead of one (a walk is a chain
// of dependent loads; its throughput per thread is bound by their latency).
// Each walk takes exactly the steps and the fault order of walk().
template <int N, int PM>
__device__ __forceinline__ void walk_multi(const DevGuest& g, const TopCache* tc, const uint64_t (&va)[N], bool write,
                                           WalkOut (&o)[N]) {
  constexpr int SD = SdOf<PM>::v;
  if (PM == kPmPae || PM == kPmPaeU || (pm_runtime(PM) && (tc ? tc->paging : g.paging) == kPagingPae)) {
#pragma unroll
    for (int k = 0; k < N; k++) o[k] = walk_pae<SD>(g, tc, va[k], write);
    return;
  }
  const DevSlot* slots = tc ? tc->slots : g.slots;
  const uint32_t nslots = tc ? tc->nslots : g.nslots;
  const bool staged = tc && tc->valid;
  uint64_t tbl[N], gpa[N], left[N];
  uint32_t lvl[N], rwus[N];   // lvl: level to read next (4..1), 0 = done; rwus: bit 0 RW, bit 1 US
#pragma unroll
  for (int k = 0; k < N; k++) {
    o[k].gpa = kAllOnes; o[k].hpa = kAllOnes; o[k].span = 0; o[k].code = kOk;
    tbl[k] = g.cr3_gpa & kFrame4K; gpa[k] = 0; left[k] = 0; rwus[k] = 3; lvl[k] = 0;
    if (!canonical(va[k])) o[k].code = kNonCanonical;
    else if (va[k] >= kUserTop) o[k].code = kRange;
    else lvl[k] = 4;
  }
#pragma unroll
  for (uint32_t level = 4; level >= 1; level--) {
    uint64_t e[N];
#pragma unroll
    for (int k = 0; k < N; k++) {   // read
      e[k] = 0;
      if (lvl[k] != level) continue;
      const uint32_t idx = (uint32_t)(va[k] >> (3 + 9 * level)) & 511;
      if (level == 4 && staged) { e[k] = tc->pml4[idx]; continue; }
      if (level == 3 && staged) {
        const uint32_t i4 = (uint32_t)(va[k] >> 39) & 511;
        int st = -1;
#pragma unroll
        for (int j = 0; j < kTopPdpt; j++) if (tc->pdpt_idx4[j] == i4) st = j;
        if (st >= 0) { e[k] = tc->pdpt[st][idx]; continue; }
      }
      uint64_t h, lim;
      if (to_host<SD>(g, tc, slots, nslots, tbl[k] + 8ull * idx, false, &h, &lim) != kOk) {
        o[k].code = kNoSlot; lvl[k] = 0; continue;
      }
      e[k] = __ldg(reinterpret_cast<const unsigned long long*>(g.pool + h));
    }
#pragma unroll
    for (int k = 0; k < N; k++) {   // examine
      if (lvl[k] != level) continue;
      const uint64_t x = e[k];
      lvl[k] = 0;
      if (!(x & kP)) { o[k].code = kNotPresent | (level << 8); continue; }
      if (level == 4 && (x & kPS)) { o[k].code = kRsvd; continue; }
      rwus[k] &= (uint32_t)((x >> 1) & 1) | ((uint32_t)((x >> 2) & 1) << 1);
      if (level == 3 && (x & kPS)) {
        gpa[k] = (x & kFrame1G) | (va[k] & ((1ull << 30) - 1));
        left[k] = (1ull << 30) - (va[k] & ((1ull << 30) - 1));
      } else if (level == 2 && (x & kPS)) {
        gpa[k] = (x & kFrame2M) | (va[k] & ((1ull << 21) - 1));
        left[k] = (1ull << 21) - (va[k] & ((1ull << 21) - 1));
      } else if (level == 1) {
        gpa[k] = (x & kFrame4K) | (va[k] & 4095);
        left[k] = kPage - (va[k] & 4095);
      } else {
        tbl[k] = x & kFrame4K;
        lvl[k] = level - 1;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < N; k++) {     // leaf checks, in walk()'s order
    if (o[k].code != kOk) continue;
    if (!(rwus[k] & 2)) { o[k].code = kUser; continue; }
    if (write && !(rwus[k] & 1)) { o[k].code = kWriteProtect; continue; }
    uint64_t h, lim;
    const uint32_t c = to_host<SD>(g, tc, slots, nslots, gpa[k], write, &h, &lim);
    if (c != kOk) { o[k].code = c; continue; }
    o[k].gpa = gpa[k]; o[k].hpa = h;
    o[k].span = left[k] < lim ? left[k] : lim;
  }
}

// Stage the PML4 table, the first kTopPdpt present PDPT tables below it and
// the memslots of guest g into shared memory.  All threads of the CTA call it.
// SD: the second dimension compiled in (kSdSlots for memslot-only launches).
template <int SD = kSdAny>
__device__ inline void stage_top(TopCache* tc, const DevGuest& g) {
  for (uint32_t i = threadIdx.x; i < g.nslots; i += blockDim.x) tc->slots[i] = g.slots[i];
  if (threadIdx.x == 0) {
    tc->nslots = g.nslots;
    tc->paging = g.paging;
    tc->ept = g.ept;
    tc->ept_root = g.ept_root;
    tc->et = nullptr;
  }
  __syncthreads();
  // top table: a 512-entry PML4, or (PAE) the 4-entry PDPT at cr3 & ~31
  const bool pae = g.paging == kPagingPae;
  const int ntop = pae ? 4 : 512;
  uint64_t h, lim;
  bool ok = to_host<SD>(g, tc, tc->slots, tc->nslots, pae ? (g.cr3_gpa & ~31ull) : (g.cr3_gpa & kFrame4K),
                            false, &h, &lim) == kOk;
  if (ok) {
    const uint64_t* t = reinterpret_cast<const uint64_t*>(g.pool + h);
    for (int i = threadIdx.x; i < ntop; i += blockDim.x) tc->pml4[i] = t[i];
  }
  if (threadIdx.x < 16) tc->cand[threadIdx.x] = 0u;
  if (threadIdx.x == 0) {
    tc->valid = ok ? 1u : 0u;
    for (int k = 0; k < kTopPdpt; k++) tc->pdpt_idx4[k] = ~0u;
  }
  __syncthreads();
  if (!ok) return;
  // choose second-level tables: the first kTopPdpt present top entries that
  // link a table (4-level: PS clear; PAE: no reserved bit set) backed by a
  // slot.  Every thread tests its entries into a 512-bit mask; one thread
  // then takes the lowest set bits.
  for (int i = threadIdx.x; i < ntop; i += blockDim.x) {
    uint64_t e = tc->pml4[i];
    uint64_t hh, ll;
    const bool link = pae ? !(e & kPaePdpteRsvd) : !(e & kPS);
    if ((e & kP) && link && to_host<SD>(g, tc, tc->slots, tc->nslots, e & kFrame4K, false, &hh, &ll) == kOk)
      atomicOr(&tc->cand[i >> 5], 1u << (i & 31));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = 0;
    for (int w = 0; w < 16 && k < kTopPdpt; w++) {
      uint32_t m = tc->cand[w];
      while (m && k < kTopPdpt) {
        tc->pdpt_idx4[k++] = (uint32_t)(w * 32 + __ffs(m) - 1);
        m &= m - 1;
      }
    }
  }
  __syncthreads();
  for (int k = 0; k < kTopPdpt; k++) {
    uint32_t i4 = tc->pdpt_idx4[k];
    if (i4 == ~0u) break;
    uint64_t hh, ll;
    to_host<SD>(g, tc, tc->slots, tc->nslots, tc->pml4[i4] & kFrame4K, false, &hh, &ll);
    const uint64_t* t = reinterpret_cast<const uint64_t*>(g.pool + hh);
    for (int i = threadIdx.x; i < 512; i += blockDim.x) tc->pdpt[k][i] = t[i];
  }
  __syncthreads();
}

// Stage the EPT's root table and the first usable table below it (read bit
// set, bit 7 clear, the table inside the pool) into `et`, after stage_top.
// All threads of the CTA call it; the root lies inside the pool (checked
// when the guest is created).
__device__ inline void stage_ept(TopCache* tc, const DevGuest& g, EptTop* et) {
  if (!g.ept) return;
  const uint64_t* root = reinterpret_cast<const uint64_t*>(g.pool + g.ept_root);
  for (int i = threadIdx.x; i < 512; i += blockDim.x) et->l4[i] = root[i];
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t pick = ~0u;
    for (int c = 0; c < 16 && pick == ~0u; c++) {
      const uint64_t e = et->l4[c * 32 + threadIdx.x];
      const bool ok = (e & 1) && !(e & 0x80) && (e & kFrame4K) + 4096 <= g.pool_bytes;
      const unsigned b = __ballot_sync(0xffffffffu, ok);
      if (b) pick = (uint32_t)(c * 32 + __ffs(b) - 1);
    }
    if (threadIdx.x == 0) et->l3_i4 = pick;
  }
  __syncthreads();
  const uint32_t i4 = et->l3_i4;
  if (i4 != ~0u) {
    const uint64_t* t = reinterpret_cast<const uint64_t*>(g.pool + (et->l4[i4] & kFrame4K));
    for (int i = threadIdx.x; i < 512; i += blockDim.x) et->l3[i] = t[i];
  }
  if (threadIdx.x == 0) tc->et = et;
  __syncthreads();
}

// Stage the EPT unit entries (kEptUnits) right after the EptTop, after
// stage_ept; all threads of the CTA call it.  Each entry is what the walk of
// ept_walk finds at levels 4..2 for the unit's gPAs: the same staged or
// global entries, bounds checks and permission rules.
__device__ inline void stage_ept_units(TopCache* tc, const DevGuest& g, EptTop* et) {
  if (tc->et == nullptr) return;   // not an EPT guest (the same for every thread)
  uint64_t* eu = reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(et) + kEptTopBytes);
  const uint64_t e4 = et->l4[0];   // gPA < 4 GiB: PML4 index 0
  const bool ok4 = (e4 & 1) && !(e4 & 0x80);
  for (uint32_t u = threadIdx.x; u < kEptUnits; u += blockDim.x) {
    const uint32_t i3 = u >> 9, i2 = u & 511;
    uint64_t v = 0;
    if (ok4) {
      uint64_t e3 = 0;
      if (et->l3_i4 == 0) {
        e3 = et->l3[i3];
      } else {
        const uint64_t at = (e4 & kFrame4K) + 8ull * i3;
        if (at + 8 <= g.pool_bytes) e3 = __ldg(reinterpret_cast<const unsigned long long*>(g.pool + at));
      }
      if (e3 & 1) {
        if (e3 & 0x80) {
          v = kEptUnitWalk;
        } else {
          const uint64_t at = (e3 & kFrame4K) + 8ull * i2;
          if (at + 8 <= g.pool_bytes) {
            const uint64_t e2 = __ldg(reinterpret_cast<const unsigned long long*>(g.pool + at));
            if (e2 & 1) v = (e2 & ~2ull) | (e4 & e3 & e2 & 2);
          }
        }
      }
    }
    eu[u] = v;
  }
  __syncthreads();
}

// Bytes of shared memory the staged unit deltas of a guest take.
__host__ __device__ constexpr size_t unit_stage_bytes(uint32_t nunits) { return 16 + 4 * (((size_t)nunits + 3) & ~3ull); }

// Stage the guest's unit deltas right after the top cache (where kSdUnits
// lookups find them), after stage_top; all threads of the CTA call it.  The
// launch gives unit_stage_bytes(g.nunits) bytes beyond kTopCacheBytes.
__device__ inline void stage_units(TopCache* tc, const DevGuest& g) {
  uint8_t* base = reinterpret_cast<uint8_t*>(tc) + kTopCacheBytes;
  const uint32_t nu = g.nunits;
  if (threadIdx.x == 0) *reinterpret_cast<uint32_t*>(base) = nu;
  const uint4* src = reinterpret_cast<const uint4*>(g.unit_delta);
  uint4* dst = reinterpret_cast<uint4*>(base + 16);
  for (uint32_t i = threadIdx.x; i < (nu + 3) / 4; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Warp copy primitives.  All 32 lanes call them with identical arguments.
// Destination writes are exact (head/tail bytes stored individually, body in
// aligned VEC-byte stores); the source is read in whole aligned VEC-byte
// words, each containing at least one source byte, so no read crosses a
// 4 KiB page that holds no source byte.
// ---------------------------------------------------------------------------
template <int VEC> struct VecT;
template <> struct VecT<16> { using T = uint4; };
template <> struct VecT<8> { using T = uint2; };
template <> struct VecT<4> { using T = uint32_t; };

__device__ __forceinline__ uint32_t fsh(uint32_t lo, uint32_t hi, uint32_t bytes) {
  // bytes in [0,3]: low word of (hi:lo) >> 8*bytes
  return __funnelshift_r(lo, hi, 8 * bytes);
}

template <int VEC>
__device__ __forceinline__ void load_words(const uint8_t* p, uint32_t* w) {
  using T = typename VecT<VEC>::T;
  T v = __ldcs(reinterpret_cast<const T*>(p));
  const uint32_t* s = reinterpret_cast<const uint32_t*>(&v);
#pragma unroll
  for (int i = 0; i < VEC / 4; i++) w[i] = s[i];
}

template <int VEC>
__device__ __forceinline__ void store_words(uint8_t* p, const uint32_t* w) {
  using T = typename VecT<VEC>::T;
  T v;
  uint32_t* d = reinterpret_cast<uint32_t*>(&v);
#pragma unroll
  for (int i = 0; i < VEC / 4; i++) d[i] = w[i];
  __stcs(reinterpret_cast<T*>(p), v);
}

// Realigned body: dst vector v (aligned) takes bytes [Q*4 + r, Q*4 + r + VEC)
// of the source words v and v+1 (aligned, sal = src rounded down).  Lane l
// loads word v; word v+1 comes from lane l+1 by shuffle (lane 31 loads it).
template <int VEC, int U, int Q>
__device__ __forceinline__ void realign_body(uint8_t* dst, const uint8_t* sal, uint64_t nvec,
                                             uint32_t r, int lane) {
  constexpr int W = VEC / 4;
  for (uint64_t base = 0; base < nvec; base += 32ull * U) {
    uint32_t a[U][W], b[U][W];
#pragma unroll
    for (int u = 0; u < U; u++) {
      uint64_t v = base + (uint64_t)u * 32 + lane;
      // word nvec still holds source bytes of the last vector
      if (v <= nvec) load_words<VEC>(sal + v * VEC, a[u]);
      else {
#pragma unroll
        for (int i = 0; i < W; i++) a[u][i] = 0;
      }
      uint32_t x[W];
#pragma unroll
      for (int i = 0; i < W; i++) x[i] = 0;
      if (lane == 31 && v < nvec) load_words<VEC>(sal + (v + 1) * VEC, x);
#pragma unroll
      for (int i = 0; i < W; i++) {
        uint32_t nb = __shfl_down_sync(0xffffffffu, a[u][i], 1);
        b[u][i] = (lane == 31) ? x[i] : nb;
      }
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      uint64_t v = base + (uint64_t)u * 32 + lane;
      if (v < nvec) {
        uint32_t o[W];
#pragma unroll
        for (int i = 0; i < W; i++) {
          const int k = Q + i;
          uint32_t lo = k < W ? a[u][k] : b[u][k - W];
          uint32_t hi = (k + 1) < W ? a[u][k + 1] : b[u][k + 1 - W];
          o[i] = fsh(lo, hi, r);
        }
        store_words<VEC>(dst + v * VEC, o);
      }
    }
  }
}

// Copy n bytes src -> dst (arbitrary alignments), warp cooperative.
template <int VEC, int U>
__device__ __forceinline__ void warp_copy(uint8_t* dst, const uint8_t* src, uint64_t n, int lane) {
  uint64_t head = (VEC - ((uintptr_t)dst & (VEC - 1))) & (VEC - 1);
  if (head > n) head = n;
  if ((uint64_t)lane < head) dst[lane] = src[lane];
  dst += head; src += head; n -= head;
  uint64_t nvec = n / VEC;
  uint32_t sh = (uint32_t)((uintptr_t)src & (VEC - 1));
  if (sh == 0) {
    for (uint64_t base = 0; base < nvec; base += 32ull * U) {
      uint32_t w[U][VEC / 4];
#pragma unroll
      for (int u = 0; u < U; u++) {
        uint64_t v = base + (uint64_t)u * 32 + lane;
        if (v < nvec) load_words<VEC>(src + v * VEC, w[u]);
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        uint64_t v = base + (uint64_t)u * 32 + lane;
        if (v < nvec) store_words<VEC>(dst + v * VEC, w[u]);
      }
    }
  } else {
    const uint8_t* sal = src - sh;
    const uint32_t q = sh >> 2, r = sh & 3;
    switch (q) {
      case 0: realign_body<VEC, U, 0>(dst, sal, nvec, r, lane); break;
      case 1: if constexpr (VEC >= 8) realign_body<VEC, U, 1>(dst, sal, nvec, r, lane); break;
      case 2: if constexpr (VEC >= 16) realign_body<VEC, U, 2>(dst, sal, nvec, r, lane); break;
      default: if constexpr (VEC >= 16) realign_body<VEC, U, 3>(dst, sal, nvec, r, lane); break;
    }
  }
  uint64_t done = nvec * VEC;
  uint64_t tail = n - done;
  if ((uint64_t)lane < tail) dst[done + lane] = src[done + lane];
}

template <int VEC>
__device__ __forceinline__ void warp_zero(uint8_t* dst, uint64_t n, int lane) {
  uint64_t head = (VEC - ((uintptr_t)dst & (VEC - 1))) & (VEC - 1);
  if (head > n) head = n;
  if ((uint64_t)lane < head) dst[lane] = 0;
  dst += head; n -= head;
  uint64_t nvec = n / VEC;
  uint32_t z[VEC / 4];
#pragma unroll
  for (int i = 0; i < VEC / 4; i++) z[i] = 0;
  for (uint64_t v = lane; v < nvec; v += 32) store_words<VEC>(dst + v * VEC, z);
  uint64_t done = nvec * VEC;
  if ((uint64_t)lane < n - done) dst[done + lane] = 0;
}

}  // namespace cvd
