// cvd_place.cu -- driver-initiated maps on the GPU, sm_103a.
//
// Paper: Sec. 6.6 -- a driver (i915) creates a memory map from inside an
// operation, so no guest virtual range was chosen; the backend records the
// request, allocates the range in the guest and re-executes.  Here a call
// takes map requests without an address and a window [va_lo, va_hi): it
// finds the pages of the window that are free in the guest's tables (the
// walk stops at a non-present entry), gives each request, in index order,
// the lowest range of free pages not given to an earlier request (first
// fit), and installs the placed requests with the mmap installer.
//
// Data-parallel form:
//   expand -- the window as a list of blocks in address order; a block
//             covered by a present table entry that links a table is
//             replaced by the entries of that table inside it (one pass per
//             level, count / scan / emit), a non-present entry is a free
//             block, a leaf or an unusable entry a taken one;
//   extents -- maximal runs of free blocks (flags / scan / emit);
//   fit    -- one warp answers the requests in order from a 32-ary max tree
//             over the extents' remaining lengths (shared memory when it
//             fits): descend to the leftmost extent with room, take its
//             first pages, update the maxima on the way back up;
//   finish -- ranges to install records (the unplaced marked), then the
//             installer, which writes the per-page statuses.
#include <cstring>

#include <map>

#include "cvd_internal.h"

namespace cvd {

namespace {

constexpr uint32_t kMapAllowedPl = 0x1u | 0x2u | 0x4u | 0x8u | 0x10u | 0x100u | (1u << 31);

// Block kinds.  A mixed block carries the gPA of the table whose entries
// cover it and the level of those entries.
constexpr uint64_t kBlkFree = 0, kBlkTaken = 1, kBlkMixed = 2;

struct Blk {
  uint64_t lo, hi;   // byte range inside the window
  uint64_t tag;      // kind | level << 2 | table gPA (32-byte aligned)
};

__device__ __forceinline__ uint64_t blk_kind(uint64_t t) { return t & 3; }
__device__ __forceinline__ uint32_t blk_level(uint64_t t) { return (uint32_t)(t >> 2) & 7; }
__device__ __forceinline__ uint64_t blk_table(uint64_t t) { return t & ~31ull; }

__device__ __forceinline__ uint64_t span_shift(uint32_t level) { return 12 + 9 * (uint64_t)(level - 1); }

__device__ __forceinline__ bool table_backed(const DevGuest& G, uint64_t table_gpa) {
  uint64_t h, lim;
  return gpa_to_hpa(G, G.slots, G.nslots, table_gpa, &h, &lim);
}

// children of block b: the entries of its table inside [lo, hi), or 1 (itself)
__device__ __forceinline__ uint64_t blk_children(const DevGuest& G, const Blk& b) {
  if (blk_kind(b.tag) != kBlkMixed || !table_backed(G, blk_table(b.tag))) return 1;
  const uint64_t s = span_shift(blk_level(b.tag));
  return ((b.hi - 1) >> s) - (b.lo >> s) + 1;
}

__global__ void k_pl_count(const DevGuest* __restrict__ gp, const Blk* __restrict__ in, uint64_t n,
                           uint64_t* __restrict__ pairs) {
  const DevGuest& G = *gp;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    pairs[2 * i] = blk_children(G, in[i]);
    pairs[2 * i + 1] = 0;
  }
}

// last i with offs[2 i] <= j
__device__ __forceinline__ uint64_t find_blk(const uint64_t* offs, uint64_t n, uint64_t j) {
  uint64_t lo = 0, hi = n;
  while (hi - lo > 1) {
    uint64_t mid = (lo + hi) >> 1;
    if (offs[2 * mid] <= j) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_pl_emit(const DevGuest* __restrict__ gp, const Blk* __restrict__ in, uint64_t n,
                          const uint64_t* __restrict__ offs, Blk* __restrict__ out, uint64_t total) {
  const DevGuest& G = *gp;
  const bool pae = G.paging == kPagingPae;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = find_blk(offs, n, j);
    const Blk b = in[i];
    const uint64_t k = j - offs[2 * i];
    if (blk_kind(b.tag) != kBlkMixed) { out[j] = b; continue; }
    const uint64_t tab = blk_table(b.tag);
    const uint32_t level = blk_level(b.tag);
    uint64_t h, lim;
    if (!gpa_to_hpa(G, G.slots, G.nslots, tab, &h, &lim)) {   // a table no memslot backs: taken
      out[j] = Blk{b.lo, b.hi, kBlkTaken};
      continue;
    }
    const uint64_t s = span_shift(level);
    const uint64_t idx = (b.lo >> s) + k;                     // entry number in the whole space
    const uint64_t elo = idx << s, ehi = (idx + 1) << s;
    Blk c;
    c.lo = elo > b.lo ? elo : b.lo;
    c.hi = ehi < b.hi ? ehi : b.hi;
    const uint64_t e = __ldg(reinterpret_cast<const unsigned long long*>(G.pool + h) + (idx & 511));
    if (!(e & kP)) c.tag = kBlkFree;
    else if (level == 1 || (e & kPS) || (pae && level == 3 && (e & kPaePdpteRsvd))) c.tag = kBlkTaken;
    else c.tag = kBlkMixed | ((uint64_t)(level - 1) << 2) | (e & kFrame4K);
    out[j] = c;
  }
}

// extent starts / ends among the final (terminal) blocks
__global__ void k_pl_flags(const Blk* __restrict__ b, uint64_t n, uint64_t* __restrict__ pairs) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
    const bool f = blk_kind(b[j].tag) == kBlkFree;
    const bool pf = j > 0 && blk_kind(b[j - 1].tag) == kBlkFree;
    const bool nf = j + 1 < n && blk_kind(b[j + 1].tag) == kBlkFree;
    pairs[2 * j] = (f && !pf) ? 1 : 0;
    pairs[2 * j + 1] = (f && !nf) ? 1 : 0;
  }
}

__global__ void k_pl_extents(const Blk* __restrict__ b, uint64_t n, const uint64_t* __restrict__ offs,
                             uint64_t* __restrict__ ext_hi, uint64_t* __restrict__ leaves) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x) {
    if (blk_kind(b[j].tag) != kBlkFree) continue;
    const bool pf = j > 0 && blk_kind(b[j - 1].tag) == kBlkFree;
    const bool nf = j + 1 < n && blk_kind(b[j + 1].tag) == kBlkFree;
    // an extent's start block adds its lo, its end block its hi: length = hi - lo
    if (!pf) atomicAdd(reinterpret_cast<unsigned long long*>(leaves + offs[2 * j]),
                       (unsigned long long)(0 - (b[j].lo >> 12)));
    if (!nf) {
      const uint64_t e = offs[2 * j + 1];
      ext_hi[e] = b[j].hi >> 12;
      atomicAdd(reinterpret_cast<unsigned long long*>(leaves + e), (unsigned long long)(b[j].hi >> 12));
    }
  }
}

// 32-ary max tree: level 0 = the extents' remaining pages (leaves), level d+1
// node i = max of level d nodes 32 i .. 32 i + 31.
constexpr int kTreeMaxDepth = 7;
struct Tree {
  uint64_t* lev[kTreeMaxDepth];
  uint64_t n[kTreeMaxDepth];
  int depth;
};

__global__ void k_pl_tree_level(const uint64_t* __restrict__ child, uint64_t nc, uint64_t* __restrict__ parent,
                                uint64_t np) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t m = 0;
    for (uint64_t c = 32 * i; c < 32 * i + 32 && c < nc; c++) m = child[c] > m ? child[c] : m;
    parent[i] = m;
  }
}

struct FitOut { uint64_t leaf, rem_before; };   // leaf ~0: no range (or malformed)

// Shared-memory or global-memory node access (the global form reads and
// writes through L2: one warp is the only reader and writer).
template <bool SMEM>
__device__ __forceinline__ uint64_t node_ld(const uint64_t* p) {
  if (SMEM) return *reinterpret_cast<const volatile uint64_t*>(p);
  return __ldcg(reinterpret_cast<const unsigned long long*>(p));
}
template <bool SMEM>
__device__ __forceinline__ void node_st(uint64_t* p, uint64_t v) {
  if (SMEM) *reinterpret_cast<volatile uint64_t*>(p) = v;
  else __stcg(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

// Warp maximum of a 64-bit value with two 32-bit reductions (high words,
// then the low words of the lanes holding the highest high word).
__device__ __forceinline__ uint64_t warp_max64(uint64_t v) {
  const uint32_t hi = __reduce_max_sync(0xffffffffu, (uint32_t)(v >> 32));
  const uint32_t lo = __reduce_max_sync(0xffffffffu, (uint32_t)(v >> 32) == hi ? (uint32_t)v : 0u);
  return ((uint64_t)hi << 32) | lo;
}

// One warp answers the requests in index order (first fit).  Requests are
// read 32 at a time (one per lane) and results written 32 at a time, so the
// sequential loop touches only the tree.  With SMEM the whole tree is first
// copied into shared memory (the finish step needs only `out`, so nothing is
// copied back).  An ancestor is rewritten only while the maximum below it
// changes.
template <bool SMEM>
__global__ void __launch_bounds__(32) k_pl_fit(Tree t, const MapPlaceReq* __restrict__ req, uint32_t nreq,
                                               uint64_t nhf, FitOut* __restrict__ out) {
  extern __shared__ __align__(16) uint64_t sm_tree[];
  const int lane = threadIdx.x;
  uint64_t* lev[kTreeMaxDepth];
  if (SMEM) {
    uint64_t off = 0;
    for (int d = 0; d < t.depth; d++) {
      lev[d] = sm_tree + off;
      for (uint64_t i = lane; i < t.n[d]; i += 32) lev[d][i] = t.lev[d][i];
      off += t.n[d];
    }
  } else {
    for (int d = 0; d < t.depth; d++) lev[d] = t.lev[d];
  }
  __syncwarp();
  const int D = t.depth;
  for (uint32_t c0 = 0; c0 < nreq; c0 += 32) {
    // this lane's request of the chunk
    uint64_t my_need = 0;
    if (c0 + lane < nreq) {
      const MapPlaceReq q = req[c0 + lane];
      const bool bad = q.npages == 0 || (q.flags & ~kMapAllowedPl) || q.hf_begin > nhf ||
                       q.npages > nhf - q.hf_begin;
      my_need = bad ? 0 : q.npages;   // 0: malformed (no range)
    }
    FitOut mine{~0ull, 0};
    const uint32_t m = nreq - c0 < 32 ? nreq - c0 : 32;
    for (uint32_t j = 0; j < m; j++) {
      const uint64_t need = __shfl_sync(0xffffffffu, my_need, j);
      if (need == 0 || D == 0) continue;
      uint64_t vals[kTreeMaxDepth];
      uint32_t pick[kTreeMaxDepth];
      uint64_t base = 0;
      bool found = true;
#pragma unroll
      for (int d = kTreeMaxDepth - 1; d >= 0; d--) {
        if (d >= D) continue;
        const uint64_t i = base + lane;
        vals[d] = i < t.n[d] ? node_ld<SMEM>(lev[d] + i) : 0;
        const unsigned b = __ballot_sync(0xffffffffu, vals[d] >= need);
        if (!b) { found = false; break; }
        pick[d] = (uint32_t)(__ffs(b) - 1);
        base = (base + pick[d]) * 32;
      }
      if (!found) continue;
      const uint64_t leaf = base / 32;
      const uint64_t before = __shfl_sync(0xffffffffu, vals[0], pick[0]);
      if (lane == (int)j) { mine.leaf = leaf; mine.rem_before = before; }
      // the leaf, then ancestors while their maximum changes
      uint64_t nv = before - need, node = leaf;
#pragma unroll
      for (int d = 0; d < kTreeMaxDepth; d++) {
        if (d >= D) break;
        const uint64_t old = __shfl_sync(0xffffffffu, vals[d], pick[d]);
        if (lane == (int)pick[d]) {
          vals[d] = nv;
          node_st<SMEM>(lev[d] + node, nv);
        }
        if (d + 1 >= D) break;
        const uint64_t parent_old = __shfl_sync(0xffffffffu, vals[d + 1], pick[d + 1]);
        if (old < parent_old) break;               // another child holds the maximum
        const uint64_t mx = warp_max64(vals[d]);
        if (mx == parent_old) break;               // unchanged
        node /= 32;
        nv = mx;
      }
      __syncwarp();
    }
    if (c0 + lane < nreq) out[c0 + lane] = mine;
  }
}

// Parallel first fit (extents up to kParLeaves, windows under 2^32 pages): a
// binary max tree of the extents' remaining pages (u32, P leaves, a power of
// two) in shared memory, built by the whole block; then one warp takes the
// requests 32 at a time.  Every lane finds, alone, the leftmost extent with
// room for its request at the round's start.  Allocations in other extents
// cannot change a lane's answer (extents to its left had too little room and
// only shrink), so a lane keeps its answer when its extent still has room
// after the earlier lanes that chose the same extent; the round commits the
// lanes before the first one that does not (at least one), each taking the
// extent's front after those earlier lanes, and the tree is updated from the
// committed allocations.  The result is first fit in request order.
constexpr uint32_t kParLeaves = 16384;
constexpr uint32_t kParChunk = 8192;   // requests whose page counts are staged in shared memory at a time

__global__ void __launch_bounds__(1024) k_pl_fit_par(const uint64_t* __restrict__ leaves, uint32_t E, uint32_t P,
                                                     const MapPlaceReq* __restrict__ req, uint32_t nreq,
                                                     uint64_t nhf, FitOut* __restrict__ out) {
  extern __shared__ __align__(16) uint32_t tr[];   // nodes 1 .. 2P - 1; leaves at P + e
  __shared__ uint32_t needs[kParChunk];           // page counts of the chunk's requests (0: malformed)
  __shared__ uint32_t sneed[32];
  for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) tr[P + i] = i < E ? (uint32_t)leaves[i] : 0u;
  __syncthreads();
  for (uint32_t w = P >> 1; w >= 1; w >>= 1) {
    for (uint32_t i = threadIdx.x; i < w; i += blockDim.x) {
      const uint32_t a = tr[2 * (w + i)], b = tr[2 * (w + i) + 1];
      tr[w + i] = a > b ? a : b;
    }
    __syncthreads();
  }
  const uint32_t lane = threadIdx.x & 31;
  for (uint32_t k0 = 0; k0 < nreq; k0 += kParChunk) {
    const uint32_t kn = nreq - k0 < kParChunk ? nreq - k0 : kParChunk;
    for (uint32_t i = threadIdx.x; i < kn; i += blockDim.x) {
      const MapPlaceReq q = req[k0 + i];
      const bool bad = q.npages == 0 || (q.flags & ~kMapAllowedPl) || q.hf_begin > nhf ||
                       q.npages > nhf - q.hf_begin;
      needs[i] = bad ? 0u : q.npages;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      for (uint32_t c0 = 0; c0 < kn;) {
        const uint32_t r = c0 + lane;
        const uint32_t need = r < kn ? needs[r] : 0u;
        uint32_t cand = ~0u;
        if (need && tr[1] >= need) {
          uint32_t i = 1;
          while (i < P) { i <<= 1; if (tr[i] < need) i++; }
          cand = i - P;
        }
        sneed[lane] = need;
        __syncwarp();
        const unsigned same = __match_any_sync(0xffffffffu, cand);
        uint64_t S = 0;   // pages the earlier lanes of this extent take first
        for (unsigned m = same & ((1u << lane) - 1); m; m &= m - 1) S += sneed[__ffs(m) - 1];
        const uint32_t remc = cand != ~0u ? tr[P + cand] : 0u;
        const bool ok = cand == ~0u || S + need <= remc;
        const unsigned fail = __ballot_sync(0xffffffffu, !ok);
        const uint32_t f = fail ? (uint32_t)(__ffs(fail) - 1) : 32u;
        const bool commit = lane < f && r < kn;
        if (commit) out[k0 + r] = cand != ~0u ? FitOut{cand, remc - S} : FitOut{~0ull, 0};
        const unsigned cm = __ballot_sync(0xffffffffu, commit && cand != ~0u) & same;
        bool up = commit && cand != ~0u && (int)lane == 31 - __clz(cm);
        __syncwarp();                                 // every lane has read its extent's room
        uint32_t node = P + cand;
        if (up) tr[node] = (uint32_t)(remc - S - need);
        __syncwarp();
        // ancestors, one level at a time, while some maximum still changes
        while (__ballot_sync(0xffffffffu, up && node > 1)) {
          uint32_t v = 0;
          if (up && node > 1) {
            node >>= 1;
            const uint32_t a = tr[2 * node], b = tr[2 * node + 1];
            v = a > b ? a : b;
            up = tr[node] != v;
          } else {
            up = false;
          }
          __syncwarp();
          if (up) tr[node] = v;
          __syncwarp();
        }
        c0 += f;
      }
    }
    __syncthreads();
  }
}

// Placed ranges -> install records; unplaced requests marked for the installer.
__global__ void k_pl_finish(const MapPlaceReq* __restrict__ req, uint32_t nreq, uint64_t nhf,
                            const FitOut* __restrict__ fit, const uint64_t* __restrict__ ext_hi,
                            MapReq* __restrict__ mreq, uint64_t* __restrict__ gva_out) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nreq; r += (uint64_t)gridDim.x * blockDim.x) {
    const MapPlaceReq q = req[r];
    const FitOut f = fit[r];
    MapReq m;
    m.npages = q.npages;
    m.hf_begin = q.hf_begin;
    if (f.leaf != ~0ull) {
      m.gva = (ext_hi[f.leaf] - f.rem_before) << 12;
      m.flags = q.flags;
    } else {
      const bool bad = q.npages == 0 || (q.flags & ~kMapAllowedPl) || q.hf_begin > nhf || q.npages > nhf - q.hf_begin;
      m.gva = ~0ull;
      m.flags = bad ? ~0u : kMapNoSpace;
    }
    mreq[r] = m;
    gva_out[r] = m.gva;
  }
}

__global__ void k_pl_none(const MapPlaceReq* __restrict__ req, uint32_t nreq, MapReq* __restrict__ mreq,
                          uint64_t* __restrict__ gva_out) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nreq; r += (uint64_t)gridDim.x * blockDim.x) {
    const MapPlaceReq q = req[r];
    mreq[r] = MapReq{~0ull, q.npages, ~0u, q.hf_begin};   // EINVAL for every page
    gva_out[r] = ~0ull;
  }
}

unsigned grid_n(uint64_t n) {
  uint64_t want = (n + 255) / 256;
  uint64_t cap = (uint64_t)num_sms() * 8;
  if (want > cap) want = cap;
  return (unsigned)(want ? want : 1);
}

// Grow-only device workspace of the placer (callers hold the map mutex).
// Growing waits for the device first: kernels still queued may use the old
// buffer.
struct PlaceWs {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t need(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (cudaDeviceSynchronize() != cudaSuccess) return cudaErrorUnknown;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); return e; }
    cap = bytes;
    return cudaSuccess;
  }
};
// One set per device (callers hold the map mutex).
struct PlaceScratch { PlaceWs blk[2], misc, fit; };
std::map<int, PlaceScratch> g_place_ws;
PlaceScratch& place_ws() {
  int dev = 0;
  cudaGetDevice(&dev);
  return g_place_ws[dev];
}

size_t al256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace

// Largest tree kept in shared memory by the fit kernel (nodes of 8 bytes).
constexpr uint64_t kFitSmemNodes = 27 * 1024;

int mmap_place(const DevGuest* dg, const DevGuest& hg, uint64_t va_lo, uint64_t va_hi, const MapPlaceReq* req,
               uint32_t nreq, const uint64_t* hf, uint64_t nhf, uint64_t* gva_out, int32_t* status,
               cudaStream_t st) {
  if (nreq == 0) return 0;
  PlaceScratch& W = place_ws();
  PlaceWs(&g_pl_blk)[2] = W.blk;
  PlaceWs& g_pl_misc = W.misc;
  PlaceWs& g_pl_fit = W.fit;
  // records for the installer + fit results
  if (g_pl_fit.need(al256((size_t)nreq * sizeof(MapReq)) + al256((size_t)nreq * sizeof(FitOut))) != cudaSuccess)
    return -12;
  MapReq* mreq = reinterpret_cast<MapReq*>(g_pl_fit.p);
  FitOut* fit = reinterpret_cast<FitOut*>((char*)g_pl_fit.p + al256((size_t)nreq * sizeof(MapReq)));
  if (hg.ept) {   // no installs into a guest behind an EPT
    k_pl_none<<<grid_n(nreq), 256, 0, st>>>(req, nreq, mreq, gva_out);
    g_launches++;
    return mmap_install(dg, hg, mreq, nreq, hf, nhf, status, st, true);
  }
  // expand the window level by level
  const bool pae = hg.paging == kPagingPae;
  const uint32_t top = pae ? 3 : 4;
  const uint64_t top_tab = pae ? (hg.cr3_gpa & ~31ull) : (hg.cr3_gpa & kFrame4K);
  Blk first{va_lo, va_hi, kBlkMixed | ((uint64_t)top << 2) | top_tab};
  uint64_t n = 1;
  if (g_pl_blk[0].need(sizeof(Blk)) != cudaSuccess) return -12;
  if (cudaMemcpyAsync(g_pl_blk[0].p, &first, sizeof(Blk), cudaMemcpyHostToDevice, st) != cudaSuccess) return -5;
  int cur = 0;
  uint64_t tot[2];
  for (uint32_t level = top; level >= 1; level--) {
    const size_t pb = 2 * (n + 1) * 8;
    if (g_pl_misc.need(2 * al256(pb) + al256(2 * scan_tmp_elems(n) * 8)) != cudaSuccess) return -12;
    uint64_t* pairs = reinterpret_cast<uint64_t*>(g_pl_misc.p);
    uint64_t* offs = reinterpret_cast<uint64_t*>((char*)g_pl_misc.p + al256(pb));
    uint64_t* tmp = reinterpret_cast<uint64_t*>((char*)g_pl_misc.p + 2 * al256(pb));
    const Blk* in = reinterpret_cast<const Blk*>(g_pl_blk[cur].p);
    k_pl_count<<<grid_n(n), 256, 0, st>>>(dg, in, n, pairs);
    g_launches++;
    if (launch_scan_pairs(pairs, offs, n, tmp, st) != cudaSuccess) return -5;
    if (cudaMemcpyAsync(tot, offs + 2 * n, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess) return -5;
    if (cudaStreamSynchronize(st) != cudaSuccess) return -5;
    const uint64_t total = tot[0];
    if (g_pl_blk[cur ^ 1].need(total * sizeof(Blk)) != cudaSuccess) return -12;
    k_pl_emit<<<grid_n(total), 256, 0, st>>>(dg, reinterpret_cast<const Blk*>(g_pl_blk[cur].p), n, offs,
                                            reinterpret_cast<Blk*>(g_pl_blk[cur ^ 1].p), total);
    g_launches++;
    cur ^= 1;
    n = total;
  }
  // extents
  const Blk* blks = reinterpret_cast<const Blk*>(g_pl_blk[cur].p);
  const size_t pb = 2 * (n + 1) * 8;
  if (g_pl_misc.need(2 * al256(pb) + al256(2 * scan_tmp_elems(n) * 8)) != cudaSuccess) return -12;
  uint64_t* pairs = reinterpret_cast<uint64_t*>(g_pl_misc.p);
  uint64_t* offs = reinterpret_cast<uint64_t*>((char*)g_pl_misc.p + al256(pb));
  uint64_t* tmp = reinterpret_cast<uint64_t*>((char*)g_pl_misc.p + 2 * al256(pb));
  k_pl_flags<<<grid_n(n), 256, 0, st>>>(blks, n, pairs);
  g_launches++;
  if (launch_scan_pairs(pairs, offs, n, tmp, st) != cudaSuccess) return -5;
  if (cudaMemcpyAsync(tot, offs + 2 * n, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess) return -5;
  if (cudaStreamSynchronize(st) != cudaSuccess) return -5;
  const uint64_t E = tot[0];
  // tree levels (in the same buffer as the extent ends, after them)
  Tree t;
  memset(&t, 0, sizeof(t));
  uint64_t nodes = 0;
  for (uint64_t m = E; m > 0 && t.depth < kTreeMaxDepth;) {
    t.n[t.depth++] = m;
    nodes += m;
    if (m <= 32) break;
    m = (m + 31) / 32;
  }
  if (E > 0 && t.n[t.depth - 1] > 32) return -12;   // beyond 32^7 extents
  size_t ext_bytes = al256((E ? E : 1) * 8);
  void* ebuf = g_pl_blk[cur ^ 1].p;   // the other block list is free now
  if (g_pl_blk[cur ^ 1].need(ext_bytes + al256((nodes ? nodes : 1) * 8)) != cudaSuccess) return -12;
  ebuf = g_pl_blk[cur ^ 1].p;
  uint64_t* ext_hi = reinterpret_cast<uint64_t*>(ebuf);
  uint64_t* tree = reinterpret_cast<uint64_t*>((char*)ebuf + ext_bytes);
  for (int d = 0, off = 0; d < t.depth; off += (int)t.n[d], d++) t.lev[d] = tree + off;
  if (E > 0) {
    if (cudaMemsetAsync(t.lev[0], 0, E * 8, st) != cudaSuccess) return -5;
    k_pl_extents<<<grid_n(n), 256, 0, st>>>(blks, n, offs, ext_hi, t.lev[0]);
    g_launches++;
    for (int d = 1; d < t.depth; d++) {
      k_pl_tree_level<<<grid_n(t.n[d]), 256, 0, st>>>(t.lev[d - 1], t.n[d - 1], t.lev[d], t.n[d]);
      g_launches++;
    }
  }
  const uint64_t window_pages = (va_hi - va_lo) >> 12;
  if (E <= kParLeaves && window_pages < (1ull << 32)) {
    uint32_t P = 1;
    while (P < E) P <<= 1;
    static bool pattr = false;
    if (!pattr) { allow_smem(k_pl_fit_par, 2 * kParLeaves * 4); pattr = true; }
    k_pl_fit_par<<<1, 1024, 2 * (size_t)P * 4, st>>>(t.lev[0], (uint32_t)E, P, req, nreq, nhf, fit);
  } else if (nodes <= kFitSmemNodes) {
    static bool attr = false;
    if (!attr) { allow_smem(k_pl_fit<true>, kFitSmemNodes * 8); attr = true; }
    k_pl_fit<true><<<1, 32, nodes * 8, st>>>(t, req, nreq, nhf, fit);
  } else {
    k_pl_fit<false><<<1, 32, 0, st>>>(t, req, nreq, nhf, fit);
  }
  k_pl_finish<<<grid_n(nreq), 256, 0, st>>>(req, nreq, nhf, fit, ext_hi, mreq, gva_out);
  g_launches += 2;
  if (cudaGetLastError() != cudaSuccess) return -5;
  return mmap_install(dg, hg, mreq, nreq, hf, nhf, status, st, true);
}

}  // namespace cvd
