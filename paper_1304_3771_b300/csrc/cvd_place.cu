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
//   fit    -- one warp answers the requests in order from a max tree over
//             the extents' remaining lengths (64-ary, top level in
//             registers, the rest in shared memory, up to 32,768 extents;
//             32-ary in shared or global memory beyond): descend to the
//             leftmost extent with room, take its first pages, update the
//             maxima on the way back up;
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

// Node access through L2 (one warp is the only reader and writer).
__device__ __forceinline__ uint64_t node_ld(const uint64_t* p) {
  return __ldcg(reinterpret_cast<const unsigned long long*>(p));
}
__device__ __forceinline__ void node_st(uint64_t* p, uint64_t v) {
  __stcg(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

// Warp maximum of a 64-bit value with two 32-bit reductions (high words,
// then the low words of the lanes holding the highest high word).
__device__ __forceinline__ uint64_t warp_max64(uint64_t v) {
  const uint32_t hi = __reduce_max_sync(0xffffffffu, (uint32_t)(v >> 32));
  const uint32_t lo = __reduce_max_sync(0xffffffffu, (uint32_t)(v >> 32) == hi ? (uint32_t)v : 0u);
  return ((uint64_t)hi << 32) | lo;
}

// One warp answers the requests in index order (first fit) on a 32-ary tree
// in global memory (windows with more extents than the shared-memory tree
// holds, or of 2^32 pages and more).  Requests are read 32 at a time (one per
// lane) and results written 32 at a time, so the sequential loop touches only
// the tree.  An ancestor is rewritten only while the maximum below it
// changes.
__global__ void __launch_bounds__(32) k_pl_fit(Tree t, const MapPlaceReq* __restrict__ req, uint32_t nreq,
                                               uint64_t nhf, FitOut* __restrict__ out) {
  const int lane = threadIdx.x;
  uint64_t* lev[kTreeMaxDepth];
  for (int d = 0; d < t.depth; d++) lev[d] = t.lev[d];
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
        vals[d] = i < t.n[d] ? node_ld(lev[d] + i) : 0;
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
          node_st(lev[d] + node, nv);
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

// First fit on a 64-ary max tree of the extents' remaining pages (u32;
// windows under 2^32 pages) in shared memory: leaves, for more than 4,096
// extents one middle level (LV = 2), and a top level of 64 nodes; one 8-byte
// load per lane reads all 64 children of a node, and a pair of ballots picks
// the leftmost child with room.
//
// The requests go in rounds of up to kFitWarps, one per warp.  Every warp
// finds its request's leftmost extent with room on the tree as the round
// starts, in parallel.  Rooms only shrink, so the extents left of that answer
// still lack room later in the round, and the answer is the request's first
// fit exactly when the extent still holds it after the round's earlier
// requests that chose it.  Warp 0 checks the round's answers in request
// order and commits the requests before the first one that fails (at least
// one: the first request searched the exact tree), each at the front of its
// extent's remaining pages; it rewrites the changed leaves, one warp per
// changed leaf rewrites its ancestors, and the next round starts at the
// failed request.  The result is first fit in request order.
constexpr uint32_t kParLeaves = 32768;
constexpr uint32_t kParChunk = 8192;   // requests whose page counts are staged in shared memory at a time
constexpr uint32_t kFitWarps = 16;
static_assert(kFitWarps % 4 == 0, "answers are read 16 bytes at a time");
static_assert(kFitWarps < 32, "a round's requests are lanes of one warp");

// Leftmost of the 64 nodes (two per lane, lane-major) holding at least n;
// false when none does.  Every lane of the warp gets the same answer.
__device__ __forceinline__ bool pick64(uint2 v, uint32_t n, uint32_t* node) {
  const unsigned ba = __ballot_sync(0xffffffffu, v.x >= n), bb = __ballot_sync(0xffffffffu, v.y >= n);
  const unsigned any = ba | bb;
  if (!any) return false;
  const uint32_t l = (uint32_t)(__ffs(any) - 1);
  *node = 2 * l + ((ba >> l) & 1u ? 0u : 1u);
  return true;
}

// Maximum of the 64 nodes below a node (children at c), for every lane.
__device__ __forceinline__ uint32_t max64(const uint32_t* c, uint32_t lane) {
  const uint2 v = *reinterpret_cast<const uint2*>(c + 2 * lane);
  return __reduce_max_sync(0xffffffffu, max(v.x, v.y));
}

template <int LV>
__global__ void __launch_bounds__(kFitWarps * 32) k_pl_fit_par(const uint64_t* __restrict__ leaves, uint32_t E,
                                                               uint32_t L0, uint32_t L1,
                                                               const MapPlaceReq* __restrict__ req, uint32_t nreq,
                                                               uint64_t nhf, FitOut* __restrict__ out) {
  extern __shared__ __align__(16) uint32_t tr[];   // leaves [0, L0); LV == 2: middle level [L0, L0 + L1)
  __shared__ uint32_t needs[kParChunk];           // page counts of the chunk's requests (0: malformed)
  __shared__ __align__(8) uint32_t top[64];
  __shared__ __align__(16) uint32_t cx[kFitWarps], croom[kFitWarps], cn[kFitWarps];   // the round's answers
                                                                          // (leaf, its room, pages)
  __shared__ uint32_t s_commit;
  uint32_t* lf = tr;
  uint32_t* mid = tr + L0;
  const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (uint32_t i = threadIdx.x; i < L0; i += blockDim.x) lf[i] = i < E ? (uint32_t)leaves[i] : 0u;
  __syncthreads();
  const uint32_t* below = lf;
  uint32_t nb = L0;
  if (LV == 2) {
    for (uint32_t i = w; i < L1; i += kFitWarps) {
      const uint32_t m = 64 * i < L0 ? max64(lf + 64 * i, lane) : 0u;
      if (lane == 0) mid[i] = m;
    }
    __syncthreads();
    below = mid;
    nb = L1;
  }
  for (uint32_t i = w; i < 64; i += kFitWarps) {
    const uint32_t m = 64 * i < nb ? max64(below + 64 * i, lane) : 0u;
    if (lane == 0) top[i] = m;
  }
  __syncthreads();
  for (uint32_t k0 = 0; k0 < nreq; k0 += kParChunk) {
    const uint32_t kn = nreq - k0 < kParChunk ? nreq - k0 : kParChunk;
    for (uint32_t i = threadIdx.x; i < kn; i += blockDim.x) {
      const MapPlaceReq q = req[k0 + i];
      const bool bad = q.npages == 0 || (q.flags & ~kMapAllowedPl) || q.hf_begin > nhf ||
                       q.npages > nhf - q.hf_begin;
      needs[i] = bad ? 0u : q.npages;
    }
    __syncthreads();
    for (uint32_t i0 = 0; i0 < kn;) {
      const uint32_t nk = kn - i0 < kFitWarps ? kn - i0 : kFitWarps;
      // this warp's request: leftmost extent with room on the round-start tree
      if (w < nk) {
        const uint32_t n = needs[i0 + w];
        uint32_t x = ~0u, room = 0, k;
        if (n != 0 && pick64(*reinterpret_cast<const uint2*>(top + 2 * lane), n, &k)) {
          uint32_t j = k;
          if (LV == 2) {
            pick64(*reinterpret_cast<const uint2*>(mid + 64 * k + 2 * lane), n, &j);
            j += 64 * k;
          }
          const uint2 v = *reinterpret_cast<const uint2*>(lf + 64 * j + 2 * lane);
          pick64(v, n, &x);
          room = __shfl_sync(0xffffffffu, (x & 1) ? v.y : v.x, x >> 1);
          x += 64 * j;
        }
        if (lane == 0) { cx[w] = x; croom[w] = room; cn[w] = n; }
      }
      __syncthreads();
      // warp 0 checks the answers in request order (lane j: request i0 + j),
      // writes the committed results and leaves, and names the leaves whose
      // ancestors change
      if (w == 0) {
        const bool in = lane < nk;
        const uint32_t xj = in ? cx[lane] : ~0u - 1 - lane;   // lanes past the round: distinct non-leaves
        const uint32_t rj = in ? croom[lane] : 0u;
        const uint32_t nj = in ? cn[lane] : 0u;
        uint32_t X[kFitWarps], N[kFitWarps];   // every answer, in every lane (broadcast loads)
#pragma unroll
        for (uint32_t q = 0; q < kFitWarps / 4; q++) {
          *reinterpret_cast<uint4*>(X + 4 * q) = reinterpret_cast<const uint4*>(cx)[q];
          *reinterpret_cast<uint4*>(N + 4 * q) = reinterpret_cast<const uint4*>(cn)[q];
        }
        unsigned same = 0;     // the round's requests that chose this lane's extent
        uint64_t before = 0;   // pages the earlier ones take from it first
#pragma unroll
        for (uint32_t t = 0; t < kFitWarps; t++) {
          const uint32_t xt = t < nk ? X[t] : ~0u - 1 - t;
          same |= xt == xj ? 1u << t : 0u;
          before += xt == xj && t < lane ? N[t] : 0u;
        }
        const bool ok = !in || xj == ~0u || before + nj <= rj;
        const unsigned fail = __ballot_sync(0xffffffffu, !ok);
        const uint32_t c = fail ? (uint32_t)(__ffs(fail) - 1) : nk;   // committed: requests i0 .. i0 + c - 1
        const unsigned later = same & ~((2u << lane) - 1) & ((1u << c) - 1);
        const bool last = lane < c && xj != ~0u && later == 0;   // the extent's last commit of the round
        if (lane < c) out[k0 + i0 + lane] = xj != ~0u ? FitOut{xj, rj - (uint32_t)before} : FitOut{~0ull, 0};
        if (last) lf[xj] = rj - (uint32_t)before - nj;
        if (lane < kFitWarps) cx[lane] = last ? xj : ~0u;
        if (lane == 0) s_commit = c;
      }
      __syncthreads();
      const uint32_t xw = cx[w], c = s_commit;   // this warp rewrites the ancestors of leaf xw
      if (LV == 2) {
        if (xw != ~0u) {
          const uint32_t m = max64(lf + 64 * (xw / 64), lane);
          if (lane == 0) mid[xw / 64] = m;
        }
        __syncthreads();
        if (xw != ~0u) {
          const uint32_t m = max64(mid + 64 * (xw / 4096), lane);
          if (lane == 0) top[xw / 4096] = m;
        }
      } else if (xw != ~0u) {
        const uint32_t m = max64(lf + 64 * (xw / 64), lane);
        if (lane == 0) top[xw / 64] = m;
      }
      __syncthreads();
      i0 += c;
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
  const uint64_t window_pages = (va_hi - va_lo) >> 12;
  const bool par = E <= kParLeaves && window_pages < (1ull << 32);   // the shared-memory fit (leaves only)
  if (E > 0) {
    if (cudaMemsetAsync(t.lev[0], 0, E * 8, st) != cudaSuccess) return -5;
    k_pl_extents<<<grid_n(n), 256, 0, st>>>(blks, n, offs, ext_hi, t.lev[0]);
    g_launches++;
    for (int d = 1; d < t.depth && !par; d++) {
      k_pl_tree_level<<<grid_n(t.n[d]), 256, 0, st>>>(t.lev[d - 1], t.n[d - 1], t.lev[d], t.n[d]);
      g_launches++;
    }
  }
  if (par) {
    const uint32_t L0 = 64 * (uint32_t)((E + 63) / 64 ? (E + 63) / 64 : 1);
    const uint32_t L1 = 64 * ((L0 / 64 + 63) / 64);
    static bool pattr = false;
    if (!pattr) {
      allow_smem(k_pl_fit_par<1>, 4096 * 4);
      allow_smem(k_pl_fit_par<2>, (kParLeaves + kParLeaves / 64) * 4);
      pattr = true;
    }
    const unsigned thr = kFitWarps * 32;
    ProfSpan ps;
    prof_begin(&ps, st);
    if (L0 <= 4096)
      k_pl_fit_par<1><<<1, thr, (size_t)L0 * 4, st>>>(t.lev[0], (uint32_t)E, L0, 0, req, nreq, nhf, fit);
    else
      k_pl_fit_par<2><<<1, thr, (size_t)(L0 + L1) * 4, st>>>(t.lev[0], (uint32_t)E, L0, L1, req, nreq, nhf, fit);
    prof_end(&ps, kProfPlaceFit, st);
  } else {
    k_pl_fit<<<1, 32, 0, st>>>(t, req, nreq, nhf, fit);
  }
  k_pl_finish<<<grid_n(nreq), 256, 0, st>>>(req, nreq, nhf, fit, ext_hi, mreq, gva_out);
  g_launches += 2;
  if (cudaGetLastError() != cudaSuccess) return -5;
  return mmap_install(dg, hg, mreq, nreq, hf, nhf, status, st, true);
}

}  // namespace cvd
