// cvd_mmap.cu -- mmap PTE install (insert_pfn) on the GPU, sm_103a.
//
// Paper: Sec. 4.2, second category of redirected routines -- map a page at a
// guest virtual address: the backend writes the guest PTE, pointing at a
// guest-physical frame the guest OS does not use (reserved through the
// hypervisor), and the second-dimension mapping of that frame to the host
// frame; page-table pages it must add come from a pool the frontend handed
// over at initialisation.  Sec. 6.2 names insert_pfn as one of the routines.
//
// Semantics are the sequential ones (requests in order, pages in order, bump
// allocation of PT-pool frames and reserved frames, ENOMEM latching).  The
// parallel form reproduces them exactly:
//   regions -- every well-formed request is counted in each 64 KiB region
//             it touches (a page in a region of one request has no rival
//             for its leaf);
//   probe  -- every page walks the tables as they were at call start
//             (read-only) and classifies itself: EINVAL / EBUSY / EFAULT, or
//             a candidate with the first missing level m (tables m-1..1 are
//             needed);
//   own    -- a hash table keyed by (level, VA prefix) takes the atomicMin of
//             the candidate page indexes: the minimum owns (creates) that
//             table, or installs that leaf (later duplicates are EBUSY); a
//             page alone in its region owns its leaf without a key;
//   scan   -- exclusive scan of (tables owned, leaf owned) per page gives each
//             owner its bump-allocator positions; the first installing page
//             whose needs pass the pools is the ENOMEM latch point;
//   zero   -- every new table frame is zeroed;
//   write  -- links, leaves, p2m entries and per-page status.
// PAE guests walk 3 levels from their 4-entry PDPT (whose entries are linked
// with P only); x86-64 guests 4 levels from the PML4.
#include <cstring>

#include <map>

#include "cvd_internal.h"

namespace cvd {

namespace {

constexpr uint32_t kMapNx = 1u << 31;
constexpr uint32_t kMapAllowed = 0x1u | 0x2u | 0x4u | 0x8u | 0x10u | 0x100u | kMapNx;
constexpr uint64_t kEmpty = ~0ull;
constexpr int32_t kSOk = 0, kSBusy = -16, kSNoMem = -12, kSInval = -22, kSFault = -14, kSNoSpace = -28;

// page kinds after the probe
constexpr uint32_t kKindCand = 0, kKindInval = 1, kKindBusy = 2, kKindFault = 3, kKindNoSpace = 4;

struct __align__(16) HSlot {
  unsigned long long key;   // kEmpty: free
  unsigned long long min;   // lowest page index with this key (~0: none yet)
};

struct MapScratch {
  const MapReq* req;
  uint32_t nreq;
  const uint64_t* hf;
  uint64_t nhf;
  int32_t* status;
  const DevGuest* g;
  uint32_t place;           // records come from the placer (kMapNoSpace marks unplaced requests)
  uint64_t npages;          // P
  uint64_t* req_pairs;      // [2*(nreq+1)] (npages, 0) per request
  uint64_t* req_offs;       // exclusive scan
  uint64_t* scan_tmp;
  uint32_t* page_req;       // [P]
  uint32_t* page_info;      // [P]  kind | m << 8 | tables_owned << 16 | leaf_owner << 24 | sole << 28
  uint64_t* page_tab;       // [P]  gPA of the deepest existing table on the path (level m)
  uint64_t* page_pairs;     // [2*(P+1)] (tables owned, leaf owned)
  uint64_t* page_offs;      // exclusive scan
  HSlot* hslot;             // [S] key and owner (lowest page) side by side: one sector per insert
  uint64_t* hframe;         // [S] frame of a created table
  uint64_t hmask;
  unsigned long long* rkey; // [R] 64 KiB regions the well-formed requests touch (kEmpty: free)
  unsigned int* rcnt;       // [R] requests touching each region
  uint64_t rmask;
  unsigned long long* cut;  // [0] = first ENOMEM page (P if none); [1] tables used; [2] frames used
};

// MurmurHash3 64-bit finaliser (Appleby, public domain) as the slot mixer.
__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ uint64_t tkey(int level, uint64_t va) {
  // level 0 = leaf (4 KiB page), 1 = PT, 2 = PD, 3 = PDPT; prefix < 2^36
  return ((uint64_t)level << 60) | (va >> (12 + 9 * level));
}

__device__ uint64_t h_insert(const MapScratch& s, uint64_t key, uint64_t page) {
  uint64_t slot = fmix64(key) & s.hmask;
  for (uint64_t i = 0; i <= s.hmask; i++) {
    unsigned long long prev = atomicCAS(&s.hslot[slot].key, kEmpty, key);
    if (prev == kEmpty || prev == key) {
      atomicMin(&s.hslot[slot].min, (unsigned long long)page);
      return slot;
    }
    slot = (slot + 1) & s.hmask;
  }
  return kEmpty;   // unreachable: the table is sized for twice the keys
}

// 64 KiB regions: a page whose region only one request touches is the only
// candidate for its virtual address (a request's pages are distinct), so it
// owns its leaf without an ownership slot.
constexpr uint32_t kRegionShift = 16;
constexpr uint32_t kInfoSole = 1u << 28;

__device__ void r_count(const MapScratch& s, uint64_t region) {
  uint64_t slot = fmix64(region) & s.rmask;
  for (uint64_t i = 0; i <= s.rmask; i++) {
    const unsigned long long prev = atomicCAS(&s.rkey[slot], kEmpty, region);
    if (prev == kEmpty || prev == region) {
      atomicAdd(&s.rcnt[slot], 1u);
      return;
    }
    slot = (slot + 1) & s.rmask;
  }
}

__device__ unsigned int r_requests(const MapScratch& s, uint64_t region) {
  uint64_t slot = fmix64(region) & s.rmask;
  for (uint64_t i = 0; i <= s.rmask; i++) {
    const unsigned long long k = s.rkey[slot];
    if (k == region) return s.rcnt[slot];
    if (k == kEmpty) return ~0u;   // not counted: cannot happen for a candidate; stay safe
    slot = (slot + 1) & s.rmask;
  }
  return ~0u;
}

__device__ uint64_t h_find(const MapScratch& s, uint64_t key) {
  uint64_t slot = fmix64(key) & s.hmask;
  for (uint64_t i = 0; i <= s.hmask; i++) {
    uint64_t k = s.hslot[slot].key;
    if (k == key) return slot;
    if (k == kEmpty) return kEmpty;
    slot = (slot + 1) & s.hmask;
  }
  return kEmpty;
}

__device__ __forceinline__ uint32_t find_req_of_page(const MapScratch& s, uint64_t p) {
  // last r with offs[r] <= p (offs = even words of the (npages, 0) pair scan)
  uint32_t lo = 0, hi = s.nreq;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (s.req_offs[2 * (uint64_t)mid] <= p) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ bool req_bad(const MapScratch& s, const MapReq& q) {
  const uint64_t top = va_top(*s.g);
  return (q.gva & 4095) != 0 || q.gva >= top || (uint64_t)q.npages * kPage > top - q.gva ||
         q.hf_begin > s.nhf || q.npages > s.nhf - q.hf_begin || (q.flags & ~kMapAllowed) != 0;
}

// One warp per well-formed request: count it once in every 64 KiB region
// its range touches.
__global__ void k_map_regions(MapScratch s) {
  const int lane = threadIdx.x & 31;
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = w0; r < s.nreq; r += nw) {
    const MapReq q = s.req[r];
    if (q.npages == 0 || (s.place && q.flags == kMapNoSpace) || s.g->ept || req_bad(s, q)) continue;
    const uint64_t r0 = q.gva >> kRegionShift, r1 = (q.gva + (uint64_t)q.npages * kPage - 1) >> kRegionShift;
    for (uint64_t g = r0 + lane; g <= r1; g += 32) r_count(s, g);
  }
}

__global__ void k_map_count(MapScratch s) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < s.nreq; r += (uint64_t)gridDim.x * blockDim.x) {
    s.req_pairs[2 * r] = s.req[r].npages;
    s.req_pairs[2 * r + 1] = 0;
  }
}

__device__ bool read_table_entry(const DevGuest& G, uint64_t table_gpa, uint32_t idx, uint64_t* e) {
  uint64_t h, lim;
  if (!gpa_to_hpa(G, G.slots, G.nslots, table_gpa + 8ull * idx, &h, &lim)) return false;
  *e = *reinterpret_cast<const volatile uint64_t*>(G.pool + h);
  return true;
}

// probe: classify every page against the tables as they were at call start
__global__ void k_map_probe(MapScratch s) {
  const DevGuest& G = *s.g;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < s.npages; p += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t r = find_req_of_page(s, p);
    MapReq q = s.req[r];
    uint64_t k = p - s.req_offs[2 * (uint64_t)r];
    uint64_t va = q.gva + k * kPage;
    s.page_req[p] = r;
    uint32_t kind = kKindCand, m = 0;
    uint64_t tab = 0;
    // installs into a guest behind an EPT are not supported: every page EINVAL
    if (s.place && q.flags == kMapNoSpace) {
      kind = kKindNoSpace;
    } else if (G.ept || req_bad(s, q) || s.hf[q.hf_begin + k] >= (G.pool_bytes >> 12)) {
      kind = kKindInval;
    } else {
      // 4-level: from the PML4; PAE: from the 4-entry PDPT (a present PDPTE
      // with reserved bits set is in the way, like a present PS entry)
      const bool pae = G.paging == kPagingPae;
      uint64_t t = pae ? (G.cr3_gpa & ~31ull) : (G.cr3_gpa & kFrame4K);
      for (int level = pae ? 3 : 4; level >= 1; level--) {
        uint32_t idx = (va >> (12 + 9 * (level - 1))) & 511;
        uint64_t e;
        if (!read_table_entry(G, t, idx, &e)) { kind = kKindFault; break; }
        if (!(e & kP)) { m = level; tab = t; break; }
        if (level == 1 || (e & kPS) || (pae && level == 3 && (e & kPaePdpteRsvd))) { kind = kKindBusy; break; }
        t = e & kFrame4K;
      }
    }
    const bool sole = kind == kKindCand && r_requests(s, va >> kRegionShift) == 1;
    s.page_info[p] = kind | (m << 8) | (sole ? kInfoSole : 0u);
    s.page_tab[p] = tab;
    if (kind == kKindCand) {
      if (!sole) h_insert(s, tkey(0, va), p);
      // A table's key needs only the lowest candidate page under it.  The
      // previous page of the same request, inside the same table's range,
      // walks the same entries down to level m, so it is a candidate needing
      // that table unless its own host frame is out of range: then this page
      // cannot be the lowest and skips the insert (no atomics on a key that
      // hundreds of thousands of pages share).
      const bool prev_cand = k > 0 && s.hf[q.hf_begin + k - 1] < (G.pool_bytes >> 12);
      for (int L = (int)m - 1; L >= 1; L--)
        if (!prev_cand || ((va - kPage) >> (12 + 9 * L)) != (va >> (12 + 9 * L))) h_insert(s, tkey(L, va), p);
    }
  }
}

// own: tables and leaf owned by each candidate page
__global__ void k_map_own(MapScratch s) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < s.npages; p += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t info = s.page_info[p];
    uint64_t t = 0, f = 0;
    if ((info & 0xff) == kKindCand) {
      uint32_t m = (info >> 8) & 0xff;
      uint32_t r = s.page_req[p];
      MapReq q = s.req[r];
      uint64_t va = q.gva + (p - s.req_offs[2 * (uint64_t)r]) * kPage;
      if ((info & kInfoSole) || s.hslot[h_find(s, tkey(0, va))].min == p) {
        f = 1;
        for (int L = (int)m - 1; L >= 1; L--) {
          uint64_t sl = h_find(s, tkey(L, va));
          if (s.hslot[sl].min == p) t++;
        }
      }
      s.page_info[p] = info | ((uint32_t)t << 16) | ((uint32_t)f << 24);
    }
    s.page_pairs[2 * p] = t;
    s.page_pairs[2 * p + 1] = f;
  }
}

// cut: the first installing page whose needs pass the pools latches ENOMEM
__global__ void k_map_cut(MapScratch s) {
  const DevGuest& G = *s.g;
  uint64_t pt_free = G.pt_pool_n - G.alloc[0];
  uint64_t rsv_free = G.rsv_n - G.alloc[1];
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < s.npages; p += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t f = s.page_pairs[2 * p + 1];
    if (!f) continue;
    uint64_t t = s.page_pairs[2 * p];
    uint64_t T = s.page_offs[2 * p], F = s.page_offs[2 * p + 1];
    if (T + t > pt_free || F + 1 > rsv_free) atomicMin(s.cut, (unsigned long long)p);
  }
}

__global__ void k_map_summary(MapScratch s) {
  uint64_t c = s.cut[0];
  if (c > s.npages) c = s.npages;
  s.cut[0] = c;
  s.cut[1] = s.page_offs[2 * c];
  s.cut[2] = s.page_offs[2 * c + 1];
}

// assign: owners record the frames of the tables they create
__global__ void k_map_assign(MapScratch s) {
  const DevGuest& G = *s.g;
  uint64_t cut = s.cut[0];
  uint64_t base = G.pt_pool_gfn + G.alloc[0];
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < cut; p += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t info = s.page_info[p];
    if ((info & 0xff) != kKindCand || !((info >> 24) & 1)) continue;
    uint32_t m = (info >> 8) & 0xff;
    uint32_t r = s.page_req[p];
    MapReq q = s.req[r];
    uint64_t va = q.gva + (p - s.req_offs[2 * (uint64_t)r]) * kPage;
    uint64_t T = s.page_offs[2 * p];
    uint64_t j = 0;
    for (int L = (int)m - 1; L >= 1; L--) {   // top-down, as the sequential walk creates them
      uint64_t sl = h_find(s, tkey(L, va));
      if (s.hslot[sl].min == p) s.hframe[sl] = base + T + j++;
    }
  }
}

// zero: one warp per new table frame
__global__ void k_map_zero(MapScratch s) {
  const DevGuest& G = *s.g;
  uint64_t ntab = s.cut[1];
  uint64_t base = G.pt_pool_gfn + G.alloc[0];
  int lane = threadIdx.x & 31;
  uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t k = w; k < ntab; k += nw) {
    uint64_t h, lim;
    if (!gpa_to_hpa(G, G.slots, G.nslots, (base + k) << 12, &h, &lim)) continue;  // validated at create
    uint4* t = reinterpret_cast<uint4*>(G.pool + h);
    for (int i = lane; i < 256; i += 32) t[i] = make_uint4(0, 0, 0, 0);
  }
}

__device__ void write_table_entry(const DevGuest& G, uint64_t table_gpa, uint32_t idx, uint64_t e) {
  uint64_t h, lim;
  if (!gpa_to_hpa(G, G.slots, G.nslots, table_gpa + 8ull * idx, &h, &lim)) return;
  *reinterpret_cast<volatile uint64_t*>(G.pool + h) = e;
}

// write: links of created tables, leaves, p2m, status
__global__ void k_map_write(MapScratch s) {
  const DevGuest& G = *s.g;
  uint64_t cut = s.cut[0];
  uint64_t rsv_base = G.rsv_gfn + G.alloc[1];
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < s.npages; p += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t info = s.page_info[p];
    uint32_t kind = info & 0xff;
    int32_t st;
    if (kind == kKindInval) st = kSInval;
    else if (kind == kKindNoSpace) st = kSNoSpace;
    else if (p >= cut) st = kSNoMem;
    else if (kind == kKindBusy) st = kSBusy;
    else if (kind == kKindFault) st = kSFault;
    else if (!((info >> 24) & 1)) st = kSBusy;            // an earlier page installed this VA
    else {
      st = kSOk;
      uint32_t m = (info >> 8) & 0xff;
      uint32_t r = s.page_req[p];
      MapReq q = s.req[r];
      uint64_t k = p - s.req_offs[2 * (uint64_t)r];
      uint64_t va = q.gva + k * kPage;
      // tables on the path: level m is the deepest existing one; below it, created ones
      uint64_t tab = s.page_tab[p];
      for (int L = (int)m; L >= 2; L--) {
        uint64_t sl = h_find(s, tkey(L - 1, va));
        uint64_t child = s.hframe[sl];
        // link P|RW|US; a PAE PDPTE has no RW/US bits: P only
        const uint64_t link = (G.paging == kPagingPae && L == 3) ? kP : 0x7;
        if (s.hslot[sl].min == p) write_table_entry(G, tab, (va >> (12 + 9 * (L - 1))) & 511, (child << 12) | link);
        tab = child << 12;
      }
      uint64_t rg = rsv_base + s.page_offs[2 * p + 1];
      uint64_t leaf = (rg << 12) | kP | (q.flags & 0x11Eu);
      if (q.flags & kMapNx) leaf |= 1ull << 63;
      write_table_entry(G, tab, (va >> 12) & 511, leaf);
      G.p2m[rg - G.rsv_gfn] = s.hf[q.hf_begin + k];
    }
    s.status[p] = st;
  }
}

__global__ void k_map_commit(MapScratch s) {
  uint64_t* a = s.g->alloc;
  a[0] += s.cut[1];
  a[1] += s.cut[2];
}

// Grow-only scratch of the installer, one per device (callers hold the map
// mutex; every call synchronises its stream before returning, so a buffer is
// never in use when the next call grows it).
struct MapWs {
  void* p = nullptr;
  size_t cap = 0;
  bool need(size_t bytes) {
    if (bytes <= cap) return true;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return false; }
    cap = bytes;
    return true;
  }
};
struct MapScratchDev { MapWs small, big; };
std::map<int, MapScratchDev> g_map_ws;

MapScratchDev& map_ws() {
  int dev = 0;
  cudaGetDevice(&dev);
  return g_map_ws[dev];
}

unsigned grid_for(uint64_t n, unsigned threads) {
  uint64_t want = (n + threads - 1) / threads;
  uint64_t cap = (uint64_t)num_sms() * 16;
  if (want > cap) want = cap;
  return (unsigned)(want ? want : 1);
}

}  // namespace

int mmap_install(const DevGuest* dg, const DevGuest& hg, const MapReq* req, uint32_t nreq, const uint64_t* hf,
                 uint64_t nhf, int32_t* status, cudaStream_t st, bool place) {
  (void)hg;
  if (nreq == 0) return 0;
  MapScratch s;
  memset(&s, 0, sizeof(s));
  s.req = req; s.nreq = nreq; s.hf = hf; s.nhf = nhf; s.status = status; s.g = dg; s.place = place ? 1u : 0u;
  // phase 0: pages per request (scan) -> total P (one synchronisation)
  size_t rp = 2 * ((size_t)nreq + 1) * 8;
  size_t tmp0 = 2 * scan_tmp_elems(nreq) * 8;
  MapScratchDev& ws = map_ws();
  if (!ws.small.need(2 * rp + tmp0 + 64)) return -12;
  void* small = ws.small.p;
  s.req_pairs = reinterpret_cast<uint64_t*>(small);
  s.req_offs = reinterpret_cast<uint64_t*>((char*)small + rp);
  uint64_t* tmp_req = reinterpret_cast<uint64_t*>((char*)small + 2 * rp);
  k_map_count<<<grid_for(nreq, 256), 256, 0, st>>>(s);
  g_launches++;
  cudaError_t e = launch_scan_pairs(s.req_pairs, s.req_offs, nreq, tmp_req, st);
  uint64_t tot[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(tot, s.req_offs + 2 * (uint64_t)nreq, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return -5;
  uint64_t P = tot[0];
  s.npages = P;
  if (P == 0) return 0;
  // per-page scratch and the ownership hash, at least twice its keys: a key
  // per page, and per request of n pages at most n / 512 + 2 page tables, n /
  // 512^2 + 2 directories and n / 512^3 + 2 pointer tables -- under
  // P / 256 + 8 nreq in all
  const uint64_t keys = P + P / 256 + 8 * (uint64_t)nreq;
  uint64_t S = 1;
  while (S < 2 * keys) S <<= 1;
  s.hmask = S - 1;
  // the region counts, at least twice their keys: per request of n pages at
  // most n / 16 + 2 regions of 64 KiB
  uint64_t R = 1;
  while (R < 2 * (P / 16 + 2 * (uint64_t)nreq + 16)) R <<= 1;
  s.rmask = R - 1;
  size_t pp = 2 * ((size_t)P + 1) * 8;
  const size_t pad = 256;
  size_t need = 64 + S * sizeof(HSlot) + S * 8 + R * 12 + P * 4 + P * 4 + P * 8 + 2 * pp + 2 * scan_tmp_elems(P) * 8 + 10 * pad;
  if (!ws.big.need(need)) return -12;
  char* b = reinterpret_cast<char*>(ws.big.p);
  auto take = [&](size_t n) { char* r = b; b += (n + pad - 1) & ~(pad - 1); return r; };
  s.cut = reinterpret_cast<unsigned long long*>(take(64));
  s.hslot = reinterpret_cast<HSlot*>(take(S * sizeof(HSlot)));
  s.hframe = reinterpret_cast<uint64_t*>(take(S * 8));
  s.rkey = reinterpret_cast<unsigned long long*>(take(R * 8));
  s.rcnt = reinterpret_cast<unsigned int*>(take(R * 4));
  s.page_req = reinterpret_cast<uint32_t*>(take(P * 4));
  s.page_info = reinterpret_cast<uint32_t*>(take(P * 4));
  s.page_tab = reinterpret_cast<uint64_t*>(take(P * 8));
  s.page_pairs = reinterpret_cast<uint64_t*>(take(pp));
  s.page_offs = reinterpret_cast<uint64_t*>(take(pp));
  s.scan_tmp = reinterpret_cast<uint64_t*>(take(2 * scan_tmp_elems(P) * 8));
  e = cudaMemsetAsync(s.hslot, 0xFF, S * sizeof(HSlot), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.rkey, 0xFF, R * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.rcnt, 0, R * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.cut, 0xFF, 8, st);
  if (e != cudaSuccess) return -5;
  k_map_regions<<<grid_for((uint64_t)nreq * 32, 256), 256, 0, st>>>(s);
  g_launches++;
  unsigned gp = grid_for(P, 256);
  ProfSpan ps;
  prof_begin(&ps, st);
  k_map_probe<<<gp, 256, 0, st>>>(s);
  prof_end(&ps, kProfMapProbe, st);
  k_map_own<<<gp, 256, 0, st>>>(s);
  g_launches += 2;
  e = launch_scan_pairs(s.page_pairs, s.page_offs, P, s.scan_tmp, st);
  if (e != cudaSuccess) return -5;
  k_map_cut<<<gp, 256, 0, st>>>(s);
  k_map_summary<<<1, 1, 0, st>>>(s);
  k_map_assign<<<gp, 256, 0, st>>>(s);
  k_map_zero<<<(unsigned)num_sms() * 4, 256, 0, st>>>(s);
  k_map_write<<<gp, 256, 0, st>>>(s);
  k_map_commit<<<1, 1, 0, st>>>(s);
  g_launches += 6;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // scratch is reused by the next call
  return e == cudaSuccess ? 0 : -5;
}

}  // namespace cvd
