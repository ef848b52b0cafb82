// cvd_translate.cu -- cvd_translate for memslot guests with unit tables and
// for guests behind a software EPT (sm_103a): the software page walk of
// Sec. 4.2 (gVA -> gPA through the guest's tables, gPA -> host through KVM's
// memslots, or through the EPT in software for other hypervisors) over a
// batch of addresses, with every level above the leaf tables staged in
// shared memory.
//
// A walk is a chain of dependent 8-byte loads; the paper keeps a 10-entry
// translation cache against that cost (Sec. 4.2).  Here each block copies the
// guest's top table, the first second-level tables, and as many third-level
// tables (page directories) as the guest's memory can need into shared
// memory, plus the second dimension per 2 MiB unit of guest-physical memory
// -- the memslot deltas, or for an EPT guest the level-2 EPT entry of every
// unit below 4 GiB (a unit under a 2 MiB EPT leaf then resolves from shared
// memory, one under a 4 KiB EPT table with one load).  For 4-level guests the
// staged copies are then rewritten for the walk: a top or second-level entry
// carries the slot of the staged table it links, a page-directory entry
// linking a page table carries that table's host frame.  A mapped 4 KiB walk
// of a memslot guest thus reads one entry from L2/HBM (the page-table entry
// itself) and everything else from shared memory, with one second-dimension
// lookup (the page's own).  Every thread keeps tf_walks(PAE) walks in flight,
// advanced in phases: staged levels for all of them, then all their
// leaf-table loads back to back, then the leaf checks.  A walk that meets
// anything unstaged above the leaf table (a second-level table not staged, a
// table or page not in a 2 MiB unit of a memslot: the reserved window, a
// missing slot) is finished by the generic walk out of line, so the common
// path stays short; a page directory that was not staged is read from the
// pool inline.
//
// Staging copies exactly the entries a walk would read (the tables do not
// change during a call); the rewritten bits are ones the walk ignores in a
// table link, so results are those of the generic walk.
#include "cvd_internal.h"

namespace cvd {

namespace {

constexpr int kTfThreads = 512;
// Walks in flight per thread: three for 4-level guests, two for PAE guests
// (each the faster on the translation workloads).
__host__ __device__ constexpr int tf_walks(bool pae) { return pae ? 2 : 3; }
constexpr uint32_t kTfMaxL3 = 2;       // staged second-level tables (4-level guests)
constexpr uint8_t kTfNone = 0xFF;
// 4-level guests: the staged copies of the top and second-level tables carry
// the slot of the staged table each entry links in bits 52..58 (ignored by
// the walk in a table link), kTfSlotNone for none; a staged page-directory
// entry linking a page table carries the table's host frame instead of its
// gPA, or kTfGeneric (an ignored bit) when the second dimension does not
// settle it.
constexpr int kTfSlotShift = 52;
constexpr uint64_t kTfSlotMask = 0x7Full << kTfSlotShift;
constexpr uint32_t kTfSlotNone = 0x7F;
constexpr uint64_t kTfGeneric = 1ull << 9;

// Most page directories a launch stages.
constexpr uint32_t kTfMaxL2 = 64;

// Shared-memory header; the tables follow it (see tf_layout).
struct TfHdr {
  uint32_t valid;                      // top table staged
  uint32_t n3, n2;                     // staged second- / third-level tables
  uint32_t nunits;                     // unit deltas staged
  uint64_t src3[kTfMaxL3];             // host offsets of the staged second-level tables
  uint64_t src2[kTfMaxL2];             // host offsets of the staged page directories
  uint8_t map4[512];                   // top index -> staged table slot (4-level: L3 slot; PAE: PD slot)
  uint8_t map3[kTfMaxL3][512];         // (L3 slot, index) -> staged PD slot (4-level)
};

struct TfLayout {
  size_t l4, l3, l2, units, bytes;
};

__host__ __device__ inline size_t tf_round(size_t x) { return (x + 127) & ~(size_t)127; }

// Offsets of the staged tables for a launch staging up to n2max page
// directories and, for a memslot guest, nunits unit deltas (EPT guests:
// kEptUnits level-2 EPT entries).
__host__ __device__ inline TfLayout tf_layout(uint32_t n2max, uint32_t nunits, bool ept) {
  TfLayout L;
  L.l4 = tf_round(sizeof(TfHdr));
  L.l3 = L.l4 + 4096;
  L.l2 = L.l3 + 4096 * (size_t)kTfMaxL3;
  L.units = L.l2 + 4096 * (size_t)n2max;
  L.bytes = L.units + (ept ? kEptUnitBytes : tf_round(4 * (((size_t)nunits + 3) & ~(size_t)3)));
  return L;
}

// gPA -> host offset through the staged unit deltas; false when the gPA lies
// in no 2 MiB unit of a memslot (the generic walk then decides).
__device__ __forceinline__ bool tf_unit(const int32_t* ud, uint32_t nunits, uint64_t gpa, uint64_t* h) {
  const uint64_t u = gpa >> 21;
  if (u >= nunits) return false;
  const int32_t d = ud[u];
  if (d == kNoUnitDelta) return false;
  *h = gpa + ((uint64_t)(int64_t)d << 12);
  return true;
}

// The second dimension from shared memory: gPA -> host offset, or false when
// the staged entries do not settle it (the generic walk then decides).
template <bool EPT> struct TfBack;
template <> struct TfBack<false> {   // memslots: the unit deltas
  const int32_t* ud;
  uint32_t nunits;
  __device__ __forceinline__ bool host(uint64_t gpa, bool, uint64_t* h) const { return tf_unit(ud, nunits, gpa, h); }
};
template <> struct TfBack<true> {    // software EPT: the staged level-2 entries of gPA [0, 4 GiB)
  const uint64_t* eu;
  const uint8_t* pool;
  uint64_t pool_bytes, rsv_gfn, rsv_n;
  // The rules of ept_walk for the mappings it settles: the level-2 entry is a
  // usable 2 MiB leaf, or links a level-1 table whose entry is usable; the
  // whole host frame lies in the pool; a write needs the write bit ANDed over
  // the levels.  Reserved frames (the p2m), gPAs from 4 GiB and units under
  // 1 GiB EPT leaves or unusable entries go to the generic walk.
  __device__ __forceinline__ bool host(uint64_t gpa, bool write, uint64_t* h) const {
    if ((gpa >> 12) - rsv_gfn < rsv_n || (gpa >> 32)) return false;
    const uint64_t v = eu[gpa >> 21];
    if (!(v & 1)) return false;
    uint64_t w = v, hh;
    if (v & 0x80) {
      hh = (v & kFrame2M) | (gpa & ((1ull << 21) - 1));
    } else {
      const uint64_t at = (v & kFrame4K) + 8ull * ((gpa >> 12) & 511);
      if (at + 8 > pool_bytes) return false;
      const uint64_t e = __ldg(reinterpret_cast<const unsigned long long*>(pool + at));
      if (!(e & 1)) return false;
      w &= e;
      hh = (e & kFrame4K) | (gpa & 4095);
    }
    if ((hh & ~4095ull) + kPage > (pool_bytes & ~4095ull)) return false;
    if (write && !(w & 2)) return false;
    *h = hh;
    return true;
  }
};

// Pick, in index order, entries of a table that link a stageable table
// (present, a table link, the table settled by `back`) until `want`
// slots are taken; slot numbers go to map[index], the linked tables' host
// offsets to src[slot].  One warp (all lanes) calls it.
template <class B>
__device__ inline void tf_pick(const uint64_t* t, uint32_t nent, const B& back, uint8_t* map, uint64_t* src, uint32_t* n,
                               uint32_t want, bool pae_pdpt) {
  const int lane = threadIdx.x & 31;
  uint32_t base = *n;
  for (uint32_t c = 0; c < nent && base < want; c += 32) {
    const uint32_t i = c + lane;
    bool ok = false;
    uint64_t h = 0;
    if (i < nent) {
      const uint64_t e = t[i];
      const bool link = pae_pdpt ? !(e & kPaePdpteRsvd) : !(e & kPS);
      ok = (e & kP) && link && back.host(e & kFrame4K, false, &h);
    }
    const uint32_t m = __ballot_sync(0xffffffffu, ok);
    const uint32_t rank = __popc(m & ((1u << lane) - 1));
    if (ok && base + rank < want) {
      map[i] = (uint8_t)(base + rank);
      src[base + rank] = h;
    }
    base += __popc(m);
    if (base > want) base = want;
  }
  __syncwarp();
  if (lane == 0) *n = base;
  __syncwarp();
}

// Copy `n` 4 KiB tables whose host offsets are src[0..n) to dst (all threads).
__device__ inline void tf_copy_tables(uint64_t* dst, const uint64_t* src, uint32_t n, const uint8_t* pool) {
  for (uint32_t w = threadIdx.x; w < n * 256; w += blockDim.x) {   // 16-byte words
    const uint32_t t = w >> 8, k = w & 255;
    reinterpret_cast<uint4*>(dst + 512ull * t)[k] = __ldg(reinterpret_cast<const uint4*>(pool + src[t]) + k);
  }
}

// The level-2 EPT entry of unit u (gPA u << 21, below 4 GiB) as ept_walk
// meets it from the root: the write bit ANDed over levels 4..2; 0 when the
// walk ends unusable above level 1; kEptUnitWalk under a 1 GiB EPT leaf.
__device__ inline uint64_t tf_ept_unit(const DevGuest& g, uint32_t u) {
  const uint8_t* pool = g.pool;
  const uint64_t e4 = __ldg(reinterpret_cast<const unsigned long long*>(pool + g.ept_root));   // PML4 index 0
  if (!(e4 & 1) || (e4 & 0x80)) return 0;
  const uint64_t a3 = (e4 & kFrame4K) + 8ull * (u >> 9);
  if (a3 + 8 > g.pool_bytes) return 0;
  const uint64_t e3 = __ldg(reinterpret_cast<const unsigned long long*>(pool + a3));
  if (!(e3 & 1)) return 0;
  if (e3 & 0x80) return kEptUnitWalk;
  const uint64_t a2 = (e3 & kFrame4K) + 8ull * (u & 511);
  if (a2 + 8 > g.pool_bytes) return 0;
  const uint64_t e2 = __ldg(reinterpret_cast<const unsigned long long*>(pool + a2));
  if (!(e2 & 1)) return 0;
  return (e2 & ~2ull) | (e4 & e3 & e2 & 2);
}

// Stage the tables (all threads of the block call it).
template <bool PAE, bool EPT>
__device__ inline void tf_stage(unsigned char* smem, const DevGuest& g, uint32_t n2max, const TfBack<EPT>& back) {
  TfHdr* H = reinterpret_cast<TfHdr*>(smem);
  const TfLayout L = tf_layout(n2max, g.nunits, EPT);
  uint64_t* L4 = reinterpret_cast<uint64_t*>(smem + L.l4);
  uint64_t* L3 = reinterpret_cast<uint64_t*>(smem + L.l3);
  uint64_t* L2 = reinterpret_cast<uint64_t*>(smem + L.l2);
  // the second dimension first: every backing check below goes through it
  if (EPT) {
    uint64_t* eu = reinterpret_cast<uint64_t*>(smem + L.units);
    for (uint32_t u = threadIdx.x; u < kEptUnits; u += blockDim.x) eu[u] = tf_ept_unit(g, u);
  } else {
    const uint4* usrc = reinterpret_cast<const uint4*>(g.unit_delta);
    uint4* dst = reinterpret_cast<uint4*>(smem + L.units);
    for (uint32_t i = threadIdx.x; i < (g.nunits + 3) / 4; i += blockDim.x) dst[i] = usrc[i];
  }
  for (uint32_t i = threadIdx.x; i < 512; i += blockDim.x) H->map4[i] = kTfNone;
  for (uint32_t i = threadIdx.x; i < kTfMaxL3 * 512; i += blockDim.x) (&H->map3[0][0])[i] = kTfNone;
  if (threadIdx.x == 0) {
    H->n3 = 0;
    H->n2 = 0;
    H->nunits = g.nunits;
  }
  __syncthreads();
  const uint32_t ntop = PAE ? 4 : 512;
  uint64_t h = 0;
  const bool ok = back.host(PAE ? (g.cr3_gpa & ~31ull) : (g.cr3_gpa & kFrame4K), false, &h);
  if (threadIdx.x == 0) H->valid = ok ? 1u : 0u;
  if (ok)
    for (uint32_t i = threadIdx.x; i < ntop; i += blockDim.x)
      L4[i] = __ldg(reinterpret_cast<const unsigned long long*>(g.pool + h) + i);
  __syncthreads();
  if (!ok) return;
  if (PAE) {   // page directories hang from the 4 PDPTEs
    if (threadIdx.x < 32) tf_pick(L4, 4, back, H->map4, H->src2, &H->n2, n2max < 4 ? n2max : 4, true);
    __syncthreads();
  } else {
    if (threadIdx.x < 32) tf_pick(L4, 512, back, H->map4, H->src3, &H->n3, kTfMaxL3, false);
    __syncthreads();
    tf_copy_tables(L3, H->src3, H->n3, g.pool);
    __syncthreads();
    if (threadIdx.x < 32)
      for (uint32_t s = 0; s < H->n3; s++) tf_pick(L3 + 512 * s, 512, back, H->map3[s], H->src2, &H->n2, n2max, false);
    __syncthreads();
  }
  tf_copy_tables(L2, H->src2, H->n2, g.pool);
  __syncthreads();
  if (!PAE) {   // fold the slots and the page tables' host frames into the staged entries
    for (uint32_t i = threadIdx.x; i < 512; i += blockDim.x) {
      const uint32_t s3 = H->map4[i];
      L4[i] = (L4[i] & ~kTfSlotMask) | ((uint64_t)(s3 == kTfNone ? kTfSlotNone : s3) << kTfSlotShift);
    }
    for (uint32_t i = threadIdx.x; i < H->n3 * 512; i += blockDim.x) {
      const uint32_t s2 = H->map3[i >> 9][i & 511];
      L3[i] = (L3[i] & ~kTfSlotMask) | ((uint64_t)(s2 == kTfNone ? kTfSlotNone : s2) << kTfSlotShift);
    }
    for (uint32_t i = threadIdx.x; i < H->n2 * 512; i += blockDim.x) {
      uint64_t e = L2[i], h;
      if ((e & kP) && !(e & kPS))
        e = back.host(e & kFrame4K, false, &h) ? (e & ~(kFrame4K | kTfGeneric)) | h : e | kTfGeneric;
      L2[i] = e;
    }
    __syncthreads();
  }
}

// The generic walk (memslots searched or the EPT walked, nothing staged) for
// the rare walks the staged path does not finish.
template <bool PAE, bool EPT>
__device__ __noinline__ WalkOut tf_generic(const DevGuest& g, uint64_t va, bool write) {
  if (EPT) return walk(g, nullptr, va, write);   // format and second dimension read from the guest
  return PAE ? walk_pae<kSdSlots>(g, nullptr, va, write) : walk4<kSdSlots>(g, nullptr, va, write);
}

// Walk states between the phases.
constexpr uint32_t kStDone = 0, kStLeafLoad = 1, kStLeaf = 2, kStGeneric = 3;

// I: the index type (32-bit for launches under 2^31 addresses: fewer
// instructions per walk in the loop and the address arithmetic).
template <bool PAE, bool EPT, typename I>
__global__ void __launch_bounds__(kTfThreads) k_translate_staged(const DevGuest* __restrict__ gp,
                                                                  const uint64_t* __restrict__ gva, uint64_t n,
                                                                  int write, uint32_t n2max,
                                                                  uint64_t* __restrict__ gpa_out,
                                                                  uint64_t* __restrict__ hpa_out,
                                                                  uint32_t* __restrict__ code_out) {
  extern __shared__ __align__(128) unsigned char smem[];
  const DevGuest& G = *gp;
  const TfLayout L = tf_layout(n2max, G.nunits, EPT);
  TfBack<EPT> back;
  if constexpr (EPT) {
    back.eu = reinterpret_cast<const uint64_t*>(smem + L.units);
    back.pool = G.pool;
    back.pool_bytes = G.pool_bytes;
    back.rsv_gfn = G.rsv_gfn;
    back.rsv_n = G.rsv_n;
  } else {
    back.ud = reinterpret_cast<const int32_t*>(smem + L.units);
    back.nunits = G.nunits;
  }
  tf_stage<PAE, EPT>(smem, G, n2max, back);
  const TfHdr* H = reinterpret_cast<const TfHdr*>(smem);
  const uint64_t* L4 = reinterpret_cast<const uint64_t*>(smem + L.l4);
  const uint64_t* L3 = reinterpret_cast<const uint64_t*>(smem + L.l3);
  const uint64_t* L2 = reinterpret_cast<const uint64_t*>(smem + L.l2);
  const bool valid = H->valid != 0;
  const uint8_t* pool = G.pool;
  const bool wr = write != 0;
  const I stride = (I)gridDim.x * blockDim.x, nn = (I)n;
  constexpr int kTfWalks = tf_walks(PAE);
  for (I i = (I)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += kTfWalks * stride) {
    uint64_t va[kTfWalks], gpa[kTfWalks], hpa[kTfWalks], at[kTfWalks];
    uint32_t code[kTfWalks], st[kTfWalks], f[kTfWalks];
#pragma unroll
    for (int k = 0; k < kTfWalks; k++) {
      const I j = i + k * stride;
      va[k] = j < nn ? __ldcs(gva + j) : (1ull << 63) | 1ull;   // past the end: non-canonical, no table read
    }
    // phase 1: the staged levels
#pragma unroll
    for (int k = 0; k < kTfWalks; k++) {
      const uint64_t v = va[k];
      const uint32_t hi = (uint32_t)(v >> 32), lo = (uint32_t)v;
      code[k] = kOk; st[k] = kStDone; f[k] = 0; gpa[k] = kAllOnes; at[k] = 0;
      uint64_t e2 = 0;
      bool have2 = false;
      if (PAE) {
        if (hi != 0) { code[k] = kRange; continue; }
        if (!valid) { st[k] = kStGeneric; continue; }
        const uint32_t i3 = lo >> 30;
        const uint64_t e3 = L4[i3];
        if (!(e3 & kP)) { code[k] = kNotPresent | (3u << 8); continue; }
        if (e3 & kPaePdpteRsvd) { code[k] = kRsvd; continue; }
        const uint32_t s2 = H->map4[i3];
        if (s2 == kTfNone) { st[k] = kStGeneric; continue; }
        e2 = L2[s2 * 512 + ((lo >> 21) & 511)];
        f[k] = 6;   // RW and US come from the PDE and the PTE only
        have2 = true;
      } else {
        const uint32_t top = hi >> 15;
        if (top != 0) { code[k] = top == 0x1FFFFu ? kRange : kNonCanonical; continue; }
        if (!valid) { st[k] = kStGeneric; continue; }
        const uint32_t i4 = (hi >> 7) & 511, i3 = ((hi << 2) | (lo >> 30)) & 511;
        const uint64_t e4 = L4[i4];
        if (!(e4 & kP)) { code[k] = kNotPresent | (4u << 8); continue; }
        if (e4 & kPS) { code[k] = kRsvd; continue; }
        const uint32_t s3 = (uint32_t)(e4 >> kTfSlotShift) & kTfSlotNone;
        if (s3 == kTfSlotNone) { st[k] = kStGeneric; continue; }
        const uint64_t e3 = L3[s3 * 512 + i3];
        f[k] = (uint32_t)e4 & (uint32_t)e3;
        if (!(e3 & kP)) { code[k] = kNotPresent | (3u << 8); continue; }
        if (e3 & kPS) {
          gpa[k] = (e3 & kFrame1G) | (v & ((1ull << 30) - 1));
          st[k] = kStLeaf;
          continue;
        }
        const uint32_t s2 = (uint32_t)(e3 >> kTfSlotShift) & kTfSlotNone;
        if (s2 != kTfSlotNone) {   // staged: the link already holds the page table's host frame
          e2 = L2[s2 * 512 + ((lo >> 21) & 511)];
          f[k] &= (uint32_t)e2;
          if (!(e2 & kP)) { code[k] = kNotPresent | (2u << 8); continue; }
          if (e2 & kPS) {
            gpa[k] = (e2 & kFrame2M) | (v & ((1ull << 21) - 1));
            st[k] = kStLeaf;
            continue;
          }
          if (e2 & kTfGeneric) { st[k] = kStGeneric; continue; }
          at[k] = (e2 & kFrame4K) + 8ull * ((lo >> 12) & 511);
          st[k] = kStLeafLoad;
          continue;
        }
        {   // a page directory beyond the staged ones: read it from the pool
          uint64_t h;
          if (!back.host((e3 & kFrame4K) + 8ull * ((lo >> 21) & 511), false, &h)) { st[k] = kStGeneric; continue; }
          e2 = __ldg(reinterpret_cast<const unsigned long long*>(pool + h));
        }
        have2 = true;
      }
      if (have2) {
        f[k] &= (uint32_t)e2;
        if (!(e2 & kP)) { code[k] = kNotPresent | (2u << 8); continue; }
        if (e2 & kPS) {
          gpa[k] = (e2 & kFrame2M) | (v & ((1ull << 21) - 1));
          st[k] = kStLeaf;
          continue;
        }
        uint64_t h;
        if (!back.host((e2 & kFrame4K) + 8ull * ((lo >> 12) & 511), false, &h)) { st[k] = kStGeneric; continue; }
        at[k] = h;
        st[k] = kStLeafLoad;
      }
    }
    // phase 2: the leaf-table entries, all loads in flight together
    uint64_t e1[kTfWalks];
#pragma unroll
    for (int k = 0; k < kTfWalks; k++)
      e1[k] = st[k] == kStLeafLoad ? __ldg(reinterpret_cast<const unsigned long long*>(pool + at[k])) : 0;
    // phase 3: leaf checks, in the generic walk's order
#pragma unroll
    for (int k = 0; k < kTfWalks; k++) {
      if (st[k] == kStLeafLoad) {
        f[k] &= (uint32_t)e1[k];
        if (!(e1[k] & kP)) {
          code[k] = kNotPresent | (1u << 8);
          st[k] = kStDone;
        } else {
          gpa[k] = (e1[k] & kFrame4K) | (va[k] & 4095);
          st[k] = kStLeaf;
        }
      }
      hpa[k] = kAllOnes;
      if (st[k] == kStLeaf) {
        if (!(f[k] & 4)) code[k] = kUser;
        else if (wr && !(f[k] & 2)) code[k] = kWriteProtect;
        else if (!back.host(gpa[k], wr, &hpa[k])) st[k] = kStGeneric;
      }
      if (st[k] == kStGeneric) {
        const WalkOut w = tf_generic<PAE, EPT>(G, va[k], wr);
        gpa[k] = w.gpa;
        hpa[k] = w.hpa;
        code[k] = w.code;
      } else if (code[k] != kOk) {
        gpa[k] = kAllOnes;
        hpa[k] = kAllOnes;
      }
      const I j = i + k * stride;
      if (j < nn) {
        __stcs(gpa_out + j, gpa[k]);
        __stcs(hpa_out + j, hpa[k]);
        __stcs(code_out + j, code[k]);
      }
    }
  }
}

using TfFn = void (*)(const DevGuest*, const uint64_t*, uint64_t, int, uint32_t, uint64_t*, uint64_t*, uint32_t*);

// Page directories staged: for a memslot guest whose memslots end at unit
// nunits, enough for its memory's virtual span (a 1 GiB directory per 512
// units, plus two for unaligned ends); for a guest behind an EPT (whose span
// the host does not know) eight; both within a shared-memory budget of a
// third of an SM's so that three blocks (1,536 threads) stay resident.
uint32_t tf_n2max(bool pae, bool ept, uint32_t nunits) {
  if (pae) return 4;
  uint32_t want = ept ? 8 : (nunits + 511) / 512 + 2;
  if (want > kTfMaxL2) want = kTfMaxL2;
  const size_t budget = 74 * 1024;
  while (want > 1 && tf_layout(want, nunits, ept).bytes > budget) want--;
  return want;
}

template <typename I>
TfFn tf_kernel_i(bool pae, bool ept) {
  if (ept) return pae ? k_translate_staged<true, true, I> : k_translate_staged<false, true, I>;
  return pae ? k_translate_staged<true, false, I> : k_translate_staged<false, false, I>;
}

// Launches under 2^31 addresses index in 32 bits (with one resident wave of
// at most 148 x 4 x 512 threads, i + 3 x stride stays below 2^32).
constexpr uint64_t kTfIdx32 = 1ull << 31;

TfFn tf_kernel(bool pae, bool ept, uint64_t n) {
  return n < kTfIdx32 ? tf_kernel_i<uint32_t>(pae, ept) : tf_kernel_i<uint64_t>(pae, ept);
}

unsigned tf_blocks(TfFn fn, size_t smem) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kTfThreads, smem) != cudaSuccess || b < 1) {
    cudaGetLastError();
    b = 1;
  }
  return (unsigned)b;
}

}  // namespace

bool translate_staged_ok(uint32_t sel, uint32_t paging, uint32_t nunits) {
  const bool ept = sel == kWalkEpt;
  if (!ept && nunits == 0) return false;
  const bool pae = paging == kPagingPae;
  return tf_layout(tf_n2max(pae, ept, nunits), nunits, ept).bytes <= 227 * 1024;
}

void prepare_translate_staged() {
  for (bool pae : {false, true})
    for (bool ept : {false, true})
      for (uint64_t n : {(uint64_t)0, kTfIdx32})
        cudaFuncSetAttribute(tf_kernel(pae, ept, n), cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

void translate_staged_shape(uint32_t sel, uint32_t paging, uint32_t nunits, uint32_t* threads_per_sm,
                            uint32_t* walks_per_thread) {
  const bool pae = paging == kPagingPae, ept = sel == kWalkEpt;
  const size_t sm = tf_layout(tf_n2max(pae, ept, nunits), nunits, ept).bytes;
  *threads_per_sm = tf_blocks(tf_kernel(pae, ept, 0), sm) * kTfThreads;
  *walks_per_thread = tf_walks(pae);
}

cudaError_t launch_translate_staged(const DevGuest* g, uint32_t sel, uint32_t paging, uint32_t nunits,
                                    const uint64_t* gva, uint64_t n, bool write, uint64_t* gpa, uint64_t* hpa,
                                    uint32_t* code, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const bool pae = paging == kPagingPae, ept = sel == kWalkEpt;
  const uint32_t n2max = tf_n2max(pae, ept, nunits);
  const size_t sm = tf_layout(n2max, nunits, ept).bytes;
  const TfFn fn = tf_kernel(pae, ept, n);
  // one resident wave (a second, partial wave would run under-occupied)
  const uint64_t want = (n + kTfThreads - 1) / kTfThreads;
  const uint64_t cap = (uint64_t)num_sms() * tf_blocks(fn, sm);
  fn<<<(unsigned)(want < cap ? want : cap), kTfThreads, sm, st>>>(g, gva, n, write ? 1 : 0, n2max, gpa, hpa, code);
  g_launches++;
  return cudaGetLastError();
}

}  // namespace cvd
