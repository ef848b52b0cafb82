// cvd_kernels.cu -- translation, planning and levelled-run kernels (sm_103a).
//
// Paper: Sec. 4.2 -- the CVD backend services copy_from_user/copy_to_user on
// a guest user buffer by walking the guest page tables in software
// (gVA -> gPA), turning the gPA into a host address through KVM's memslots,
// once per page, and then copying; Sec. 6.2 -- these are redirected kernel
// memory routines called by an unmodified host driver.
//
// B300 design: guest arenas, page tables, requests and staging all resident
// in HBM.  One warp plans one request (lanes walk pages in parallel, a ballot
// picks the first fault); the copy engines (cvd_copy.cu) then move the bytes
// of the planned work list.  This file holds translation, the scans, the
// planner and the levelled run engine.
#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <utility>

#include "cvd_internal.h"

namespace cvd {

unsigned long long g_launches = 0;

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms;
}

// ---------------------------------------------------------------------------
// a1/a2: translate (persistent grid, top levels in smem; each thread keeps
// N walks in flight -- kTranslateWalks; kTranslateWalksPae / Ept for PAE and EPT guests --
// on gVAs i, i + stride, ... so that every warp-wide load stays coalesced)
// ---------------------------------------------------------------------------
constexpr int kTranslateWalks = 2;
// PAE walks (3 levels, fewer instructions) and 2-D walks behind an EPT
// (long, with their own staged tables) run fastest one per thread: PAE
// 141.5 vs 135.3 G walks/s with two, EPT 46.8 vs 42.3 G, while 4-level
// memslot walks gain from two (95.3 vs 87.1 G).
constexpr int kTranslateWalksPae = 1;
constexpr int kTranslateWalksEpt = 1;

template <int N, int PM>
__global__ void __launch_bounds__(256) k_translate(const DevGuest* __restrict__ gp, const uint64_t* __restrict__ gva, uint64_t n,
                                                   int write, uint64_t* __restrict__ gpa, uint64_t* __restrict__ hpa,
                                                   uint32_t* __restrict__ code) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DevGuest& G = *gp;
  TopCache* tc = reinterpret_cast<TopCache*>(smem);
  // staging reads the top tables through the memslots themselves: the unit
  // table is staged only after it
  stage_top<pm_units(PM) ? kSdSlots : SdOf<PM>::v>(tc, G);
  if (PM == kPmEpt || PM == kPmEptT) stage_ept(tc, G, reinterpret_cast<EptTop*>(smem + kTopCacheBytes));
  if (PM == kPmEptT) stage_ept_units(tc, G, reinterpret_cast<EptTop*>(smem + kTopCacheBytes));
  if (pm_units(PM)) stage_units(tc, G);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += N * stride) {
    uint64_t va[N];
    WalkOut w[N];
#pragma unroll
    for (int k = 0; k < N; k++) {
      const uint64_t j = i + k * stride;
      va[k] = j < n ? __ldcs(gva + j) : (1ull << 63) | 1ull;   // past the end: non-canonical, no table read
    }
    walk_multi<N, PM>(G, tc, va, write != 0, w);
#pragma unroll
    for (int k = 0; k < N; k++) {
      const uint64_t j = i + k * stride;
      if (j < n) {
        __stcs(gpa + j, w[k].gpa);
        __stcs(hpa + j, w[k].hpa);
        __stcs(code + j, w[k].code);
      }
    }
  }
}

using TranslateFn = void (*)(const DevGuest*, const uint64_t*, uint64_t, int, uint64_t*, uint64_t*, uint32_t*);

// The translate instantiation for a guest (walk selector, unit-table length)
// and the dynamic shared memory it is launched with.
TranslateFn translate_kernel(uint32_t sel, uint32_t nunits, size_t* smem) {
  if (sel == kWalkEpt) {
    *smem = kTopCacheBytes + kEptTopBytes + kEptUnitBytes;
    return k_translate<kTranslateWalksEpt, kPmEptT>;
  }
  if (nunits) {   // memslots on 2 MiB boundaries: lookups through the unit deltas
    *smem = kTopCacheBytes + unit_stage_bytes(nunits);
    return sel == kPagingPae ? k_translate<kTranslateWalksPae, kPmPaeU> : k_translate<kTranslateWalks, kPmX86U>;
  }
  *smem = sizeof(TopCache);
  return sel == kPagingPae ? k_translate<kTranslateWalksPae, kPmPae> : k_translate<kTranslateWalks, kPmX86>;
}

// Resident blocks per SM of a translate instantiation (at most 8), cached
// per (kernel, shared memory); 0 if the query fails.
unsigned translate_blocks(TranslateFn fn, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, size_t>, unsigned> cache;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(reinterpret_cast<const void*>(fn), smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, 256, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const unsigned r = (unsigned)(b < 8 ? b : 8);   // launch_translate starts at most 8 blocks per SM
  cache[key] = r;
  return r;
}

void translate_shape(uint32_t sel, uint32_t paging, uint32_t nunits, uint32_t* threads_per_sm,
                     uint32_t* walks_per_thread) {
  if (translate_staged_ok(sel, paging, nunits)) {
    translate_staged_shape(sel, paging, nunits, threads_per_sm, walks_per_thread);
    return;
  }
  size_t sm = 0;
  const TranslateFn fn = translate_kernel(sel, nunits, &sm);
  *threads_per_sm = translate_blocks(fn, sm) * 256;
  *walks_per_thread = sel == kWalkEpt ? kTranslateWalksEpt : sel == kPagingPae ? kTranslateWalksPae : kTranslateWalks;
}

cudaError_t launch_translate(const DevGuest* g, uint32_t sel, uint32_t paging, uint32_t nunits, const uint64_t* gva,
                             uint64_t n, bool write, uint64_t* gpa, uint64_t* hpa, uint32_t* code, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  if (translate_staged_ok(sel, paging, nunits))
    return launch_translate_staged(g, sel, paging, nunits, gva, n, write, gpa, hpa, code, st);
  size_t sm = 0;
  const TranslateFn fn = translate_kernel(sel, nunits, &sm);
  // one resident wave (a second, partial wave would run under-occupied)
  const unsigned res = translate_blocks(fn, sm);
  const uint64_t want = (n + 255) / 256;
  const uint64_t cap = (uint64_t)num_sms() * (res ? res : 1);
  fn<<<(unsigned)(want < cap ? want : cap), 256, sm, st>>>(g, gva, n, write ? 1 : 0, gpa, hpa, code);
  g_launches++;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan over (u64, u64) pairs; out[n] = totals.
// ---------------------------------------------------------------------------
constexpr int kScanT = 256, kScanI = 8, kScanTile = kScanT * kScanI;

__device__ __forceinline__ ulonglong2 add2(ulonglong2 a, ulonglong2 b) { return make_ulonglong2(a.x + b.x, a.y + b.y); }

// block-wide exclusive scan of one pair per thread; *total = block sum
__device__ ulonglong2 block_excl_scan(ulonglong2 v, ulonglong2* total) {
  __shared__ ulonglong2 ws[33];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  ulonglong2 inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    unsigned long long tx = __shfl_up_sync(0xffffffffu, inc.x, d);
    unsigned long long ty = __shfl_up_sync(0xffffffffu, inc.y, d);
    if (lane >= d) { inc.x += tx; inc.y += ty; }
  }
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    ulonglong2 s = lane < nw ? ws[lane] : make_ulonglong2(0, 0);
    ulonglong2 si = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      unsigned long long tx = __shfl_up_sync(0xffffffffu, si.x, d);
      unsigned long long ty = __shfl_up_sync(0xffffffffu, si.y, d);
      if (lane >= d) { si.x += tx; si.y += ty; }
    }
    if (lane < nw) ws[lane] = make_ulonglong2(si.x - s.x, si.y - s.y);
    if (lane == nw - 1) ws[32] = si;
  }
  __syncthreads();
  ulonglong2 base = ws[wid];
  *total = ws[32];
  __syncthreads();
  return make_ulonglong2(base.x + inc.x - v.x, base.y + inc.y - v.y);
}

__global__ void __launch_bounds__(kScanT) k_scan_reduce(const ulonglong2* __restrict__ in, uint64_t n,
                                                        ulonglong2* __restrict__ bsum) {
  uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  ulonglong2 acc = make_ulonglong2(0, 0);
  for (int i = threadIdx.x; i < kScanTile; i += kScanT) {
    uint64_t k = base + i;
    if (k < n) acc = add2(acc, in[k]);
  }
  ulonglong2 tot;
  block_excl_scan(acc, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(ulonglong2* bsum, uint64_t nb, ulonglong2* total_out) {
  ulonglong2 carry = make_ulonglong2(0, 0);
  for (uint64_t start = 0; start < nb; start += blockDim.x) {
    uint64_t k = start + threadIdx.x;
    ulonglong2 v = k < nb ? bsum[k] : make_ulonglong2(0, 0);
    ulonglong2 tot;
    ulonglong2 ex = block_excl_scan(v, &tot);
    if (k < nb) bsum[k] = add2(carry, ex);
    carry = add2(carry, tot);
  }
  if (threadIdx.x == 0) *total_out = carry;
}

__global__ void __launch_bounds__(kScanT) k_scan_apply(const ulonglong2* __restrict__ in, ulonglong2* __restrict__ out,
                                                       uint64_t n, const ulonglong2* __restrict__ boff) {
  uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanI;
  ulonglong2 v[kScanI];
  ulonglong2 s = make_ulonglong2(0, 0);
#pragma unroll
  for (int i = 0; i < kScanI; i++) {
    v[i] = (base + i < n) ? in[base + i] : make_ulonglong2(0, 0);
    s = add2(s, v[i]);
  }
  ulonglong2 tot;
  ulonglong2 ex = block_excl_scan(s, &tot);
  ex = add2(ex, boff[blockIdx.x]);
#pragma unroll
  for (int i = 0; i < kScanI; i++) {
    if (base + i < n) out[base + i] = ex;
    ex = add2(ex, v[i]);
  }
}

__global__ void k_zero_pair(ulonglong2* p) { *p = make_ulonglong2(0, 0); }

// One tile (n <= kScanTile): the exclusive scan and the total in one launch
// (the tile layout of k_scan_apply, with no block offsets).
__global__ void __launch_bounds__(kScanT) k_scan_single(const ulonglong2* __restrict__ in, ulonglong2* __restrict__ out,
                                                        uint64_t n) {
  const uint64_t base = (uint64_t)threadIdx.x * kScanI;
  ulonglong2 v[kScanI];
  ulonglong2 s = make_ulonglong2(0, 0);
#pragma unroll
  for (int i = 0; i < kScanI; i++) {
    v[i] = (base + i < n) ? in[base + i] : make_ulonglong2(0, 0);
    s = add2(s, v[i]);
  }
  ulonglong2 tot;
  ulonglong2 ex = block_excl_scan(s, &tot);
#pragma unroll
  for (int i = 0; i < kScanI; i++) {
    if (base + i < n) out[base + i] = ex;
    ex = add2(ex, v[i]);
  }
  if (threadIdx.x == 0) out[n] = tot;
}

size_t scan_tmp_elems(uint64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1; }

cudaError_t launch_scan_pairs(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t* tmp, cudaStream_t st) {
  const ulonglong2* i2 = reinterpret_cast<const ulonglong2*>(in);
  ulonglong2* o2 = reinterpret_cast<ulonglong2*>(out);
  ulonglong2* t2 = reinterpret_cast<ulonglong2*>(tmp);
  if (n == 0) {
    k_zero_pair<<<1, 1, 0, st>>>(o2);
    g_launches++;
    return cudaGetLastError();
  }
  uint64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 1) {
    k_scan_single<<<1, kScanT, 0, st>>>(i2, o2, n);
    g_launches++;
    return cudaGetLastError();
  }
  k_scan_reduce<<<(unsigned)nb, kScanT, 0, st>>>(i2, n, t2);
  k_scan_top<<<1, 1024, 0, st>>>(t2, nb, o2 + n);
  k_scan_apply<<<(unsigned)nb, kScanT, 0, st>>>(i2, o2, n, t2);
  g_launches += 3;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a6: request sizing + validation (warp per request)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_req_sizes(BatchArgs a) {
  int lane = threadIdx.x & 31;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.counter[1] = 0;   // k_plan's request counter
    a.counter[2] = 0;   // long-segment list length
    a.counter[3] = 0;   // a levelled call's conflict flag and marked-request count (two u32)
  }
  uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = w; r < a.nreq; r += nw) {
    Req q = a.req[r];
    uint32_t dir = a.dir_override >= 0 ? (uint32_t)a.dir_override : q.dir;
    uint32_t guest = a.dir_override >= 0 ? 0u : q.guest;
    bool bad = dir > 1 || guest >= a.nguests || (uint64_t)q.seg_begin + q.seg_count > a.nseg;
    uint64_t L = 0;
    if (!bad) {
      uint64_t part = 0;
      for (uint32_t k = lane; k < q.seg_count; k += 32) {
        uint64_t l = a.seg[q.seg_begin + k].len;
        part = (part + l < part) ? ~0ull : part + l;
      }
      L = warp_sat_sum(part);
    }
    uint32_t code = bad ? kBadReq : ((L > a.stg_bytes || q.host_off > a.stg_bytes - L) ? kHostBuf : kOk);
    if (lane == 0) {
      a.fkey[r] = ~0ull;   // no fault found yet
      a.lcount[r] = 0;
      a.pairs_in[2 * r] = code == kOk ? q.seg_count : 0;
      a.pairs_in[2 * r + 1] = code == kOk ? L + kReqWeight : 0;   // balancing position, see kReqWeight
      Result o;
      o.done = 0; o.fault_gva = 0; o.fault_code = code; o.pad = 0;
      a.res[r] = o;
    }
  }
}

// ---------------------------------------------------------------------------
// a6: planner.  One warp per request (requests taken 4 at a time from a
// counter): stream offsets (warp scan), first fault (segment checks, then page
// walks: lane-local for segments of <= 2 pages, the pages of all 3-64-page
// segments of a 32-segment group walked together, longer segments warp-
// cooperatively), then per-segment work records.  Segments of more than
// kLongPages pages are not walked by their warp: their pages go to a list in
// blocks that k_long_scan walks across the whole grid, each block lowering
// the request's fault key (stream offset << 12 | code) with atomicMin; the
// warp that walks a request's last block settles it.
// ---------------------------------------------------------------------------
constexpr uint64_t kNoFault = ~0ull;

struct Fault1 { uint64_t off, gva; uint32_t code; };

// First fault inside [gva, gva+len) (already range-checked), warp cooperative:
// lane k walks the k-th page from pos; the walked spans cover [pos, max end)
// without gaps (each span reaches at least its page end), so the first
// faulting lane holds the first faulting byte.  off = ~0 if none.
template <int PM>
__device__ Fault1 seg_first_fault(const DevGuest& G, const TopCache* tc, uint64_t gva, uint64_t len,
                                  bool write, int lane) {
  Fault1 f;
  f.off = ~0ull; f.gva = 0; f.code = 0;
  uint64_t end = gva + len;
  uint64_t pos = gva;
  while (pos < end) {
    uint64_t va = lane == 0 ? pos : (pos & ~4095ull) + (uint64_t)lane * 4096;
    bool active = va < end;
    WalkOut w;
    w.code = kOk; w.span = 0;
    if (active) w = walk_t<PM>(G, tc, va, write);
    unsigned m = __ballot_sync(0xffffffffu, active && w.code != kOk);
    if (m) {
      int fl = __ffs(m) - 1;
      uint64_t fva = __shfl_sync(0xffffffffu, va, fl);
      uint32_t c = __shfl_sync(0xffffffffu, w.code, fl);
      f.off = fva - gva; f.gva = fva; f.code = c;
      return f;
    }
    uint64_t e = active ? va + w.span : 0;
    pos = warp_max(e);
  }
  return f;
}

// Segments of up to this many 4 KiB pages are walked together: the pages of
// every such segment of a 32-segment group are enumerated across the warp in
// stream order and walked 32 at a time, so the first faulting item of the
// first round with a fault is the group's first faulting byte among them.
constexpr uint32_t kPlanBatchPages = 64;
// Requests a planner warp takes from the shared counter at a time.
constexpr uint32_t kPlanGrab = 4;
// Segments longer than kLongPages pages are not walked by their request's
// warp: their pages go to the long-segment list in blocks of kLongBlock pages,
// which k_long_scan walks across the whole grid (a 33 MB frame is 8,100 pages;
// shorter segments are cheaper inline, where a round crosses a whole 2 MiB leaf).

template <bool STAGE, int PM>
__global__ void __launch_bounds__(256, 4) k_plan(BatchArgs a) {   // 4 blocks (32 warps) per SM: walks are latency-bound
  extern __shared__ __align__(16) unsigned char smem[];
  TopCache* tc = nullptr;
  if (STAGE) {
    tc = reinterpret_cast<TopCache*>(smem);
    stage_top<SdOf<PM>::v>(tc, *a.single);
    if (PM == kPmEpt) stage_ept(tc, *a.single, reinterpret_cast<EptTop*>(smem + kTopCacheBytes));
  }
  int lane = threadIdx.x & 31;
  for (;;) {
    uint64_t r0 = 0;
    if (lane == 0) r0 = atomicAdd(&a.counter[1], (unsigned long long)kPlanGrab);
    r0 = __shfl_sync(0xffffffffu, r0, 0);
    if (r0 >= a.nreq) break;
    const uint64_t r1 = r0 + kPlanGrab < a.nreq ? r0 + kPlanGrab : a.nreq;
  for (uint64_t r = r0; r < r1; r++) {
    Req q = a.req[r];
    ReqWork rwk;
    rwk.host_off = q.host_off;
    rwk.nsw = 0;
    uint32_t pre = a.res[r].fault_code;
    uint64_t sb = a.pairs_out[2 * r];
    if (pre == kOk && sb + q.seg_count > a.nseg) {
      pre = kBadReq;
      if (lane == 0) a.res[r].fault_code = kBadReq;
    }
    uint32_t dir = a.dir_override >= 0 ? (uint32_t)a.dir_override : q.dir;
    uint32_t guest = a.dir_override >= 0 ? 0u : q.guest;
    rwk.sb = sb;
    rwk.guest_dir = (guest << 1) | (dir & 1);
    if (pre != kOk) {
      if (lane == 0) a.rw[r] = rwk;
      continue;
    }
    const DevGuest& G = STAGE ? *a.single : *a.guests[guest];
    const TopCache* t = STAGE ? tc : nullptr;
    bool write = dir == 1;
    uint64_t L = a.pairs_in[2 * r + 1] - kReqWeight;
    bool deferred = false;   // some long segment went to the long-segment list
    // pass 1: first fault
    Fault1 best;
    best.off = ~0ull; best.gva = 0; best.code = 0;
    uint64_t carry = 0;
    for (uint32_t g0 = 0; g0 < q.seg_count; g0 += 32) {
      if (best.off != ~0ull && best.off < carry) break;
      uint32_t j = g0 + lane;
      bool valid = j < q.seg_count;
      Seg s = valid ? a.seg[q.seg_begin + j] : Seg{0, 0};
      uint64_t incl = warp_incl_scan(s.len, lane);
      uint64_t soff = carry + incl - s.len;
      carry += __shfl_sync(0xffffffffu, incl, 31);
      Fault1 mine;
      mine.off = ~0ull; mine.gva = 0; mine.code = 0;
      uint32_t npg = 0;        // pages of a segment walked in the batched rounds
      bool large = false;      // walked alone, warp cooperative
      if (valid && s.len > 0) {
        if (!va_canonical(G, s.gva)) { mine.off = soff; mine.gva = s.gva; mine.code = kNonCanonical; }
        else if (s.gva >= va_top(G) || s.len > va_top(G) - s.gva) { mine.off = soff; mine.gva = s.gva; mine.code = kRange; }
        else {
          uint64_t n = ((s.gva + s.len - 1) >> 12) - (s.gva >> 12) + 1;
          if (n <= 2) {
            WalkOut w1 = walk_t<PM>(G, t, s.gva, write);
            if (w1.code != kOk) { mine.off = soff; mine.gva = s.gva; mine.code = w1.code; }
            else if (w1.span < s.len) {
              uint64_t va2 = s.gva + w1.span;
              WalkOut w2 = walk_t<PM>(G, t, va2, write);
              if (w2.code != kOk) { mine.off = soff + w1.span; mine.gva = va2; mine.code = w2.code; }
            }
          } else if (n <= kPlanBatchPages) {
            npg = (uint32_t)n;
          } else {
            large = true;
          }
        }
      }
      // batched rounds over the pages of the mid-sized segments
      uint32_t pincl = npg;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        uint32_t v = __shfl_up_sync(0xffffffffu, pincl, d);
        if (lane >= d) pincl += v;
      }
      const uint32_t ptotal = __shfl_sync(0xffffffffu, pincl, 31);
      for (uint32_t base = 0; base < ptotal; base += 32) {
        const uint32_t item = base + lane;
        int lo = 0, hi = 31;   // owner = smallest lane whose inclusive count exceeds item
#pragma unroll
        for (int it = 0; it < 5; it++) {
          int mid = (lo + hi) >> 1;
          uint32_t v = __shfl_sync(0xffffffffu, pincl, mid);
          if (v > item) hi = mid; else lo = mid + 1;
        }
        const uint32_t before = __shfl_sync(0xffffffffu, pincl - npg, lo);
        const uint64_t og = __shfl_sync(0xffffffffu, s.gva, lo);
        const uint64_t oo = __shfl_sync(0xffffffffu, soff, lo);
        const uint32_t k = item - before;
        const uint64_t va = k == 0 ? og : (og & ~4095ull) + (uint64_t)k * 4096;
        bool bad = false;
        uint32_t code = kOk;
        if (item < ptotal) {
          WalkOut w = walk_t<PM>(G, t, va, write);
          bad = w.code != kOk;
          code = w.code;
        }
        unsigned m = __ballot_sync(0xffffffffu, bad);
        if (m) {
          int fl = __ffs(m) - 1;
          uint64_t fva = __shfl_sync(0xffffffffu, va, fl);
          uint64_t foff = __shfl_sync(0xffffffffu, oo + (va - og), fl);
          uint32_t fc = __shfl_sync(0xffffffffu, code, fl);
          int fo = __shfl_sync(0xffffffffu, lo, fl);
          if (lane == fo) { mine.off = foff; mine.gva = fva; mine.code = fc; }
          break;
        }
      }
      uint64_t gmin = warp_min(mine.off);
      unsigned lm = __ballot_sync(0xffffffffu, large);
      while (lm) {
        int l = __ffs(lm) - 1;
        lm &= lm - 1;
        uint64_t lsoff = __shfl_sync(0xffffffffu, soff, l);
        if (gmin != ~0ull && gmin < lsoff) break;   // later in the stream than a known fault
        uint64_t lg = __shfl_sync(0xffffffffu, s.gva, l);
        uint64_t ll = __shfl_sync(0xffffffffu, s.len, l);
        const uint64_t lpages = ((lg + ll - 1) >> 12) - (lg >> 12) + 1;
        if (lpages > kLongPages) {   // to the long-segment list, unless it is full
          const uint64_t nb = (lpages + kLongBlock - 1) / kLongBlock;
          uint64_t at = 0;
          if (lane == 0) at = atomicAdd(&a.counter[2], (unsigned long long)nb);
          at = __shfl_sync(0xffffffffu, at, 0);
          if (at + nb <= a.long_cap) {
            if (lane == 0) atomicAdd(&a.lcount[r], (unsigned int)nb);
            for (uint64_t k = lane; k < nb; k += 32) {
              LongItem it;
              it.req = (uint32_t)r; it.seg = g0 + (uint32_t)l; it.page0 = (uint32_t)(k * kLongBlock);
              it.npages = (uint32_t)(lpages - k * kLongBlock < kLongBlock ? lpages - k * kLongBlock : kLongBlock);
              a.long_items[at + k] = it;
            }
            deferred = true;
            continue;
          }
          for (uint64_t k = lane; k < nb && at + k < a.long_cap; k += 32) {   // reserved, unused: null entries
            LongItem it;
            it.req = ~0u; it.seg = 0; it.page0 = 0; it.npages = 0;
            a.long_items[at + k] = it;
          }
        }
        Fault1 f = seg_first_fault<PM>(G, t, lg, ll, write, lane);
        if (f.off != ~0ull) {
          if (lane == l) { mine.off = lsoff + f.off; mine.gva = f.gva; mine.code = f.code; }
          break;
        }
      }
      gmin = warp_min(mine.off);
      if (gmin != ~0ull && gmin < best.off) {
        unsigned who = __ballot_sync(0xffffffffu, mine.off == gmin);
        int wl = __ffs(who) - 1;
        best.off = gmin;
        best.gva = __shfl_sync(0xffffffffu, mine.gva, wl);
        best.code = __shfl_sync(0xffffffffu, mine.code, wl);
      }
    }
    uint64_t done = best.off == ~0ull ? L : best.off;
    if (lane == 0) {
      Result o;
      o.done = done; o.fault_gva = best.off == ~0ull ? 0 : best.gva;
      o.fault_code = best.off == ~0ull ? kOk : best.code; o.pad = 0;
      a.res[r] = o;
      rwk.nsw = q.seg_count;
      a.rw[r] = rwk;
      if (deferred && best.off != ~0ull)   // k_long_scan settles the result once the list is walked
        atomicMin(&a.fkey[r], (unsigned long long)((best.off << 12) | best.code));
    }
    // pass 2: work records
    carry = 0;
    for (uint32_t g0 = 0; g0 < q.seg_count; g0 += 32) {
      uint32_t j = g0 + lane;
      bool valid = j < q.seg_count;
      Seg s = valid ? a.seg[q.seg_begin + j] : Seg{0, 0};
      uint64_t incl = warp_incl_scan(s.len, lane);
      uint64_t soff = carry + incl - s.len;
      carry += __shfl_sync(0xffffffffu, incl, 31);
      if (valid) {
        SegWork sw;
        sw.gva = s.gva; sw.soff = soff; sw.len = s.len;
        sw.ncopy = done <= soff ? 0 : (done - soff < s.len ? done - soff : s.len);
        a.sw[sb + j] = sw;
      }
    }
  }
  }
}


// Settle a request whose long segments were all walked: the result from the
// merged fault key, the faulting gVA, and ncopy of the segments at and after
// the fault (k_plan wrote them for its own first fault, which is no earlier).
__device__ void settle_request(const BatchArgs& a, uint64_t r, int lane) {
  const ReqWork rw = a.rw[r];
  const uint64_t key = *reinterpret_cast<volatile unsigned long long*>(&a.fkey[r]);
  if (key == kNoFault) return;   // no fault anywhere: k_plan's result stands
  const uint64_t done = key >> 12;
  uint64_t fgva = 0;
  for (uint32_t g0 = 0; g0 < rw.nsw; g0 += 32) {
    const uint32_t j = g0 + lane;
    if (j < rw.nsw) {
      SegWork s = a.sw[rw.sb + j];
      if (s.soff <= done && done < s.soff + s.len) fgva = s.gva + (done - s.soff);   // the faulting byte's segment
      if (s.soff + s.len > done) {
        s.ncopy = done <= s.soff ? 0 : done - s.soff;
        a.sw[rw.sb + j] = s;
      }
    }
  }
  fgva = warp_max(fgva);   // the one lane whose segment holds the faulting byte (others hold 0)
  if (lane == 0) {
    Result o;
    o.done = done; o.fault_gva = fgva; o.fault_code = (uint32_t)(key & 4095); o.pad = 0;
    a.res[r] = o;
  }
}

// Walk one block of a deferred long segment; the first faulting byte lowers
// the request's fault key.  A block wholly after a fault already known is
// skipped.  Each block then counts its request down; the warp that retires
// the last block settles the request (after a fence, so that every other
// block's key update is visible to it).
template <bool STAGE, int PM>
__global__ void __launch_bounds__(256) k_long_scan(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint64_t n0 = *reinterpret_cast<volatile unsigned long long*>(&a.counter[2]);
  const uint64_t n = n0 < a.long_cap ? n0 : a.long_cap;
  if ((uint64_t)blockIdx.x * (blockDim.x >> 5) >= n) return;   // no entry for this block
  TopCache* tc = nullptr;
  if (STAGE) {
    tc = reinterpret_cast<TopCache*>(smem);
    stage_top<SdOf<PM>::v>(tc, *a.single);
    if (PM == kPmEpt) stage_ept(tc, *a.single, reinterpret_cast<EptTop*>(smem + kTopCacheBytes));
  }
  const int lane = threadIdx.x & 31;
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = gw; i < n; i += nw) {
    const LongItem it = a.long_items[i];
    if (it.req == ~0u) continue;   // slot of a reservation that did not fit (walked inline)
    const ReqWork rw = a.rw[it.req];
    const SegWork s = a.sw[rw.sb + it.seg];
    const DevGuest& G = STAGE ? *a.single : *a.guests[rw.guest_dir >> 1];
    const TopCache* t = STAGE ? tc : nullptr;
    const bool write = rw.guest_dir & 1;
    const uint64_t pbase = s.gva & ~4095ull;
    const uint64_t first = it.page0 == 0 ? s.soff : s.soff + (pbase + (uint64_t)it.page0 * 4096 - s.gva);
    const uint64_t known = *reinterpret_cast<volatile unsigned long long*>(&a.fkey[it.req]);
    if ((known >> 12) > first) {
      // [pos, end): the block's bytes of the segment.  Lane k walks the k-th
      // page from pos; every walked span reaches at least its page end, so the
      // spans cover [pos, max end) without gaps and the first faulting lane
      // holds the first faulting byte; a round that faults nowhere moves pos
      // past the farthest span (one round crosses a whole 2 MiB leaf).
      uint64_t pos = it.page0 == 0 ? s.gva : pbase + (uint64_t)it.page0 * 4096;
      const uint64_t bend = pbase + (uint64_t)(it.page0 + it.npages) * 4096;
      const uint64_t end = bend < s.gva + s.len ? bend : s.gva + s.len;
      while (pos < end) {
        const uint64_t va = lane == 0 ? pos : (pos & ~4095ull) + (uint64_t)lane * 4096;
        const bool active = va < end;
        uint64_t key = kNoFault, reach = 0;
        if (active) {
          const WalkOut wo = walk_t<PM>(G, t, va, write);
          if (wo.code != kOk) key = ((s.soff + (va - s.gva)) << 12) | wo.code;
          else reach = va + wo.span;
        }
        const uint64_t m = warp_min(key);
        if (m != kNoFault) {
          if (lane == 0) atomicMin(&a.fkey[it.req], (unsigned long long)m);
          break;
        }
        pos = warp_max(reach);
      }
    }
    unsigned int left = 0;
    if (lane == 0) {
      __threadfence();
      left = atomicSub(&a.lcount[it.req], 1u);
    }
    left = __shfl_sync(0xffffffffu, left, 0);
    if (left == 1) {
      __threadfence();
      settle_request(a, it.req, lane);
    }
  }
}

cudaError_t launch_plan_sizes(const BatchArgs& a, cudaStream_t st) {
  unsigned blocks = (unsigned)num_sms() * 8;
  const uint64_t want = ((uint64_t)a.nreq + 7) / 8;
  if (want < blocks) blocks = (unsigned)(want ? want : 1);
  k_req_sizes<<<blocks, 256, 0, st>>>(a);
  g_launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_scan_pairs(a.pairs_in, a.pairs_out, a.nreq, a.scan_tmp, st);
}

cudaError_t launch_plan(const BatchArgs& a, cudaStream_t st) {
  const cudaError_t e = launch_plan_sizes(a, st);
  return e != cudaSuccess ? e : launch_plan_walk(a, st);
}

cudaError_t launch_plan_walk(const BatchArgs& a, cudaStream_t st) {
  const int sms = num_sms();
  // one resident wave: every block stages the top tables once, then warps
  // take requests from the counter until none is left.  A single-guest launch
  // compiles its walks for the guest's paging format.
  static const unsigned rx = resident_blocks(k_plan<true, kPmX86>, 256, sizeof(TopCache));
  static const unsigned rp = resident_blocks(k_plan<true, kPmPae>, 256, sizeof(TopCache));
  static const unsigned ry = resident_blocks(k_plan<true, kPmEpt>, 256, kTopCacheBytes + kEptTopBytes);
  static const unsigned ra = resident_blocks(k_plan<false, kPmAny>, 256, 0);
  static const unsigned re = resident_blocks(k_plan<false, kPmEpt>, 256, 0);
  const bool one = a.nguests == 1, pae = one && a.single_paging == kPagingPae;
  const bool ept = a.single_paging == kWalkEpt, any1 = one && ept;
  unsigned pb = (unsigned)sms * (!one ? (ept ? re : ra) : (any1 ? ry : (pae ? rp : rx)));
  const uint64_t pwant = ((uint64_t)a.nreq + 8 * kPlanGrab - 1) / (8 * kPlanGrab);
  if (pwant < pb) pb = (unsigned)(pwant ? pwant : 1);
  if (!one && ept) k_plan<false, kPmEpt><<<pb, 256, 0, st>>>(a);
  else if (!one) k_plan<false, kPmAny><<<pb, 256, 0, st>>>(a);
  else if (any1) k_plan<true, kPmEpt><<<pb, 256, kTopCacheBytes + kEptTopBytes, st>>>(a);
  else if (pae) k_plan<true, kPmPae><<<pb, 256, sizeof(TopCache), st>>>(a);
  else k_plan<true, kPmX86><<<pb, 256, sizeof(TopCache), st>>>(a);
  g_launches++;
  if (a.no_long) return cudaGetLastError();   // the caller checked: no segment spans over kLongPages pages
  static const unsigned lx = resident_blocks(k_long_scan<true, kPmX86>, 256, sizeof(TopCache));
  static const unsigned lp = resident_blocks(k_long_scan<true, kPmPae>, 256, sizeof(TopCache));
  static const unsigned ly = resident_blocks(k_long_scan<true, kPmEpt>, 256, kTopCacheBytes + kEptTopBytes);
  static const unsigned la = resident_blocks(k_long_scan<false, kPmAny>, 256, 0);
  static const unsigned le = resident_blocks(k_long_scan<false, kPmEpt>, 256, 0);
  const unsigned lb = (unsigned)sms * (!one ? (ept ? le : la) : (any1 ? ly : (pae ? lp : lx)));
  if (!one && ept) k_long_scan<false, kPmEpt><<<lb, 256, 0, st>>>(a);
  else if (!one) k_long_scan<false, kPmAny><<<lb, 256, 0, st>>>(a);
  else if (any1) k_long_scan<true, kPmEpt><<<lb, 256, kTopCacheBytes + kEptTopBytes, st>>>(a);
  else if (pae) k_long_scan<true, kPmPae><<<lb, 256, sizeof(TopCache), st>>>(a);
  else k_long_scan<true, kPmX86><<<lb, 256, sizeof(TopCache), st>>>(a);
  g_launches++;
  return cudaGetLastError();
}

// Set every dynamic-shared-memory attribute up front, so that no attribute
// call happens for the first time inside a stream capture.
void prepare_kernels() {
  static bool done = false;
  if (done) return;
  size_t sm = sizeof(TopCache);
  allow_smem(k_translate<kTranslateWalks, kPmX86>, sm);
  allow_smem(k_translate<kTranslateWalksPae, kPmPae>, sm);
  allow_smem(k_plan<true, kPmX86>, sm);
  allow_smem(k_plan<true, kPmPae>, sm);
  allow_smem(k_long_scan<true, kPmX86>, sm);
  allow_smem(k_long_scan<true, kPmPae>, sm);
  allow_smem(k_translate<kTranslateWalksEpt, kPmEptT>, kTopCacheBytes + kEptTopBytes + kEptUnitBytes);
  allow_smem(k_translate<kTranslateWalks, kPmX86U>, kTopCacheBytes + unit_stage_bytes(kUnitSlots));
  allow_smem(k_translate<kTranslateWalksPae, kPmPaeU>, kTopCacheBytes + unit_stage_bytes(kUnitSlots));
  allow_smem(k_plan<true, kPmEpt>, kTopCacheBytes + kEptTopBytes);
  allow_smem(k_long_scan<true, kPmEpt>, kTopCacheBytes + kEptTopBytes);
  prepare_copy_kernels();
  prepare_translate_staged();
  num_sms();
  done = true;
}

// ---------------------------------------------------------------------------
// a7: levelled engine -- explicit run list (in stream order) for the host
// leveller, then one copy launch per level.
// ---------------------------------------------------------------------------
// Walk the copy part of every segment of request r, merging host-contiguous
// pages into runs; plus one zero-fill run for a faulted copy-from request.
// EMIT=false counts runs into counts[2r]; EMIT=true writes them at offs[2r].
// Emit run dst <- src (src 0: zero fill) of n bytes as pieces of at most
// kRunPiece bytes (one warp copies one piece: a long run on one warp would
// hold its level back), advancing the request's run count.
__device__ __forceinline__ void emit_run(bool emit, Run* runs, uint64_t base, uint64_t* cnt, uint64_t dst, uint64_t src,
                                         uint64_t n, int lane) {
  for (uint64_t o = 0; o < n; o += kRunPiece) {
    if (emit && lane == 0) {
      Run ru;
      ru.dst = dst + o; ru.src = src ? src + o : 0; ru.len = n - o < kRunPiece ? n - o : kRunPiece; ru.pad = 0;
      runs[base + *cnt] = ru;
    }
    (*cnt)++;
  }
}

// only (optional): the requests to list (the marked ones of a levelled call,
// whose work the mark pass took from rw.nsw: seg_count stands in for it).
template <bool EMIT>
__global__ void __launch_bounds__(256) k_runs(BatchArgs a, uint64_t* counts, const uint64_t* offs, Run* runs,
                                              const uint8_t* only) {
  int lane = threadIdx.x & 31;
  uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = w; r < a.nreq; r += nw) {
    ReqWork rw = a.rw[r];
    if (only) rw.nsw = only[r] ? a.req[r].seg_count : 0;
    uint64_t cnt = 0;
    uint64_t out = EMIT ? offs[2 * r] : 0;
    if (rw.nsw) {
      const DevGuest& G = *a.guests[rw.guest_dir >> 1];
      bool to_guest = rw.guest_dir & 1;
      uint64_t L = 0, done = 0;
      for (uint32_t j = 0; j < rw.nsw; j++) {
        SegWork s = a.sw[rw.sb + j];
        L = s.soff + s.len;
        done += s.ncopy;
        uint64_t end = s.gva + s.ncopy, pos = s.gva;
        uint64_t pend_va = 0, pend_h = 0, pend_n = 0;
        while (pos < end) {
          uint64_t va = lane == 0 ? pos : (pos & ~4095ull) + (uint64_t)lane * 4096;
          bool active = va < end;
          WalkOut wk;
          wk.code = kOk; wk.span = 0; wk.hpa = 0;
          if (active) wk = walk(G, nullptr, va, to_guest);
          unsigned bad = __ballot_sync(0xffffffffu, active && wk.code != kOk);
          uint64_t stop = end;
          if (bad) stop = __shfl_sync(0xffffffffu, va, __ffs(bad) - 1);
          unsigned act = __ballot_sync(0xffffffffu, active && va < stop);
          uint64_t np = pos;
          while (act) {
            int k = __ffs(act) - 1;
            act &= act - 1;
            uint64_t kva = __shfl_sync(0xffffffffu, va, k);
            uint64_t kh = __shfl_sync(0xffffffffu, wk.hpa, k);
            uint64_t ks = __shfl_sync(0xffffffffu, wk.span, k);
            uint64_t kend = kva + ks < stop ? kva + ks : stop;
            if (kend <= np) continue;
            uint64_t h = kh + (np - kva);
            uint64_t n = kend - np;
            if (pend_n && pend_h + pend_n == h) {
              pend_n += n;
            } else {
              if (pend_n) {
                uint64_t g = (uint64_t)(uintptr_t)(G.pool + pend_h);
                uint64_t sp = (uint64_t)(uintptr_t)(a.stg + rw.host_off + s.soff + (pend_va - s.gva));
                emit_run(EMIT, runs, out, &cnt, to_guest ? g : sp, to_guest ? sp : g, pend_n, lane);
              }
              pend_va = np; pend_h = h; pend_n = n;
            }
            np = kend;
          }
          if (bad || np == pos) break;
          pos = np;
        }
        if (pend_n) {
          uint64_t g = (uint64_t)(uintptr_t)(G.pool + pend_h);
          uint64_t sp = (uint64_t)(uintptr_t)(a.stg + rw.host_off + s.soff + (pend_va - s.gva));
          emit_run(EMIT, runs, out, &cnt, to_guest ? g : sp, to_guest ? sp : g, pend_n, lane);
        }
      }
      if (!to_guest && done < L)
        emit_run(EMIT, runs, out, &cnt, (uint64_t)(uintptr_t)(a.stg + rw.host_off + done), 0, L - done, lane);
    }
    if (!EMIT && lane == 0) { counts[2 * r] = cnt; counts[2 * r + 1] = 0; }
  }
}

cudaError_t launch_runs(const BatchArgs& a, bool emit, uint64_t* counts, const uint64_t* offs, Run* runs,
                        cudaStream_t st, const uint8_t* only) {
  unsigned blocks = (unsigned)num_sms() * 8;
  uint64_t want = ((uint64_t)a.nreq + 7) / 8;
  if (want < blocks) blocks = (unsigned)(want ? want : 1);
  if (emit) k_runs<true><<<blocks, 256, 0, st>>>(a, counts, offs, runs, only);
  else k_runs<false><<<blocks, 256, 0, st>>>(a, counts, offs, runs, only);
  g_launches++;
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_run_copy(const Run* __restrict__ runs, uint64_t n) {
  int lane = threadIdx.x & 31;
  uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = w; i < n; i += nw) {
    Run r = runs[i];
    uint8_t* d = reinterpret_cast<uint8_t*>((uintptr_t)r.dst);
    if (r.src) warp_copy<16, 2>(d, reinterpret_cast<const uint8_t*>((uintptr_t)r.src), r.len, lane);
    else warp_zero<16>(d, r.len, lane);
  }
}

// ---------------------------------------------------------------------------
// a7: levelled calls on the device.  Two requests conflict when they touch a
// common staging byte or a common guest host byte with one of them writing
// it.  Pass 1 (beside the planner) puts every guest page each request may
// touch into a hash table, keyed by the device frame the page starts in, and
// marks the pages that two requests touch with a writer among them (a
// copy-to request touching a page twice marks it too: its segments would
// otherwise be copied in parallel).  Pass 2 marks every request that
// touches a marked frame -- or every request, when the staging ranges are
// not in order without overlap or the table ran full.  Unmarked requests
// conflict with no other request, so they run in one parallel launch; the
// marked ones then run one after another in index order (k_ordered_copy):
// the sequential semantics, with no host round trip.
// ---------------------------------------------------------------------------

constexpr unsigned long long kHzConflict = 1ull << 39;   // vals: the frame is touched with a conflict

__device__ __forceinline__ uint64_t hz_hash(uint64_t frame, uint32_t shift, uint64_t mask) {
  return ((frame * 0x9E3779B97F4A7C15ull) >> shift) & mask;   // Fibonacci hashing
}

// Insert (frame, request r, writes w) into the epoch-tagged open-addressing
// table (keys[i] = epoch << 40 | frame, vals[i] = epoch << 40 | conflict << 39
// | r << 1 | w; a slot whose epoch is not the current one is empty, so the
// table is never cleared between calls).  The first request to touch a frame
// owns it; a later touch conflicts when it comes from another request and
// either writes, or from the owner itself writing again (bit 2 of *flag then
// tells the mark pass it has work).  A probe sequence that runs out sets bit
// 1 of *flag.
__device__ __forceinline__ void hz_insert(unsigned long long* keys, unsigned long long* vals, uint64_t mask,
                                          uint32_t shift, uint64_t epoch, uint64_t frame, uint64_t r, uint32_t w,
                                          unsigned int* flag) {
  const unsigned long long key = (epoch << 40) | frame;
  uint64_t h = hz_hash(frame, shift, mask);
  for (int probe = 0; probe < 64; probe++) {
    unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(&keys[h]);
    while ((k >> 40) != epoch) {   // empty or left from an earlier call: claim it
      const unsigned long long old = atomicCAS(&keys[h], k, key);
      if (old == k) { k = key; break; }
      k = old;
    }
    if (k == key) {
      const unsigned long long mine = (epoch << 40) | (r << 1) | w;
      unsigned long long v = *reinterpret_cast<volatile unsigned long long*>(&vals[h]);
      for (;;) {
        if ((v >> 40) != epoch) {
          const unsigned long long old = atomicCAS(&vals[h], v, mine);
          if (old == v) return;   // first touch of the frame
          v = old;
          continue;
        }
        const bool other = ((v >> 1) & 0xFFFFFFFFull) != r;
        if ((other && ((v & 1) || w)) || (!other && w)) {
          atomicOr(&vals[h], kHzConflict);
          atomicOr(flag, 4u);   // some frame conflicts: the mark pass has work
        }
        return;
      }
    }
    h = (h + 1) & mask;
  }
  atomicOr(flag, 2u);
}

// Whether the frame is marked (it was inserted in this epoch by pass 1).
__device__ __forceinline__ bool hz_marked(const unsigned long long* keys, const unsigned long long* vals, uint64_t mask,
                                          uint32_t shift, uint64_t epoch, uint64_t frame) {
  const unsigned long long key = (epoch << 40) | frame;
  uint64_t h = hz_hash(frame, shift, mask);
  for (int probe = 0; probe < 64; probe++) {
    const unsigned long long k = keys[h];
    if (k == key) return (vals[h] & kHzConflict) != 0;
    if ((k >> 40) != epoch) return true;   // not found: cannot happen after pass 1; stay safe
    h = (h + 1) & mask;
  }
  return true;
}

// The frame key of a guest page: the 4 KiB frame of device memory the page's
// first byte lies in.  Every access to a guest page gives the same key
// whatever its first byte, and distinct guest pages give distinct keys when
// the guests' pools do not overlap (a pool need not be 4 KiB-aligned: the
// pages of a view into a larger allocation still start 4 KiB apart).
__device__ __forceinline__ uint64_t hz_key(const DevGuest& G, uint64_t hpa, uint64_t va) {
  return ((uint64_t)(uintptr_t)(G.pool + hpa) - (va & 4095)) >> 12;
}

// The keys of the pages of [gva, end) (already range-checked) that translate,
// one page per lane, 32 pages a round; fn(key) for each, which returns true
// to stop (then the call returns true).  All lanes call it.
template <class F>
__device__ __forceinline__ bool hz_range(const DevGuest& G, bool to_guest, uint64_t gva, uint64_t end, int lane,
                                         F fn) {
  for (uint64_t pos = gva; pos < end; pos = (pos & ~4095ull) + 32ull * 4096) {
    const uint64_t va = lane == 0 ? pos : (pos & ~4095ull) + (uint64_t)lane * 4096;
    bool hit = false;
    if (va < end) {
      const WalkOut wo = walk(G, nullptr, va, to_guest);
      if (wo.code == kOk) hit = fn(hz_key(G, wo.hpa, va));
    }
    if (__any_sync(0xffffffffu, hit)) return true;
  }
  return false;
}

// The keys of the copied part of every segment of request r (the planner's
// ncopy).
template <class F>
__device__ __forceinline__ void hz_frames(const BatchArgs& a, const ReqWork& rw, int lane, F fn) {
  const DevGuest& G = *a.guests[rw.guest_dir >> 1];
  const bool to_guest = rw.guest_dir & 1;
  for (uint32_t j = 0; j < rw.nsw; j++) {
    const SegWork s = a.sw[rw.sb + j];
    if (hz_range(G, to_guest, s.gva, s.gva + s.ncopy, lane, fn)) return;
  }
}

// Pass 1: one warp per request inserts the keys of every page of its
// segments that translates, read from the request itself (not from the
// plan, so the pass runs beside the planner).  That is a superset of the
// pages the request copies (the planner stops a request at its first fault);
// a superset can only add conflicts, never hide one.  A request the sizing
// kernel refused (BADREQ, HOSTBUF: its pair holds 0) copies nothing and
// inserts nothing, so an accepted request's pages are bounded by its staging
// range; a segment that fails its range checks ends the request's copy, and
// its insertions.
__global__ void __launch_bounds__(256) k_hz_insert(BatchArgs a, unsigned long long* keys, unsigned long long* vals,
                                                   uint64_t mask, uint32_t shift, uint64_t epoch, unsigned int* flag) {
  const int lane = threadIdx.x & 31;
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = w0; r < a.nreq; r += nw) {
    const Req q = a.req[r];
    const uint32_t dir = a.dir_override >= 0 ? (uint32_t)a.dir_override : q.dir;
    const uint32_t guest = a.dir_override >= 0 ? 0u : q.guest;
    if (dir > 1 || guest >= a.nguests || (uint64_t)q.seg_begin + q.seg_count > a.nseg) continue;
    if (a.pairs_in[2 * r + 1] == 0) continue;   // refused by the sizing kernel
    const DevGuest& G = *a.guests[guest];
    for (uint32_t j = 0; j < q.seg_count; j++) {
      const Seg s = a.seg[q.seg_begin + j];
      if (!s.len) continue;
      if (!va_canonical(G, s.gva) || s.gva >= va_top(G) || s.len > va_top(G) - s.gva) break;
      hz_range(G, dir == 1, s.gva, s.gva + s.len, lane, [&](uint64_t key) {
        hz_insert(keys, vals, mask, shift, epoch, key, r, dir, flag);
        return false;
      });
    }
  }
}

// Pass 2: one warp per request; a request touching a marked frame (or every
// request, when *flag has bit 0 or 1) is marked for the ordered pass: mark[r] = 1,
// its work taken from the parallel launch (nsw = 0; the ordered pass reads
// seg_count from the request), and counted in *nmarked.
__global__ void __launch_bounds__(256) k_hz_mark(BatchArgs a, const unsigned long long* keys,
                                                 const unsigned long long* vals, uint64_t mask, uint32_t shift,
                                                 uint64_t epoch, const unsigned int* flag, uint8_t* mark,
                                                 unsigned int* nmarked) {
  const int lane = threadIdx.x & 31;
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  if (w0 == 0 && lane == 0) a.counter[0] = 0;   // the parallel copy's work counter (it follows this pass)
  const unsigned int f = *flag;
  const bool all = (f & 3u) != 0;
  if (!all && !(f & 4u)) {   // no frame conflicts: nothing to mark
    for (uint64_t r = w0; r < a.nreq; r += nw)
      if (lane == 0) mark[r] = 0;
    return;
  }
  for (uint64_t r = w0; r < a.nreq; r += nw) {
    ReqWork rw = a.rw[r];
    bool m = false;
    if (rw.nsw) {
      if (all) {
        m = true;
      } else {
        hz_frames(a, rw, lane, [&](uint64_t frame) {
          const bool hit = hz_marked(keys, vals, mask, shift, epoch, frame);
          if (hit) m = true;
          return hit;
        });
        m = __any_sync(0xffffffffu, m);
      }
    }
    if (lane == 0) {
      mark[r] = m ? 1 : 0;
      if (m) {
        rw.nsw = 0;
        a.rw[r] = rw;
        atomicAdd(nmarked, 1u);
      }
    }
  }
}

// Staging: the requests' ranges [host_off, host_off + L) must lie in
// increasing order without overlap (an exclusive max-scan of the range ends
// in request order); a request whose range starts before the end of an
// earlier one sets bit 0 of *flag (every request then runs in order).  One
// block.
__global__ void __launch_bounds__(1024) k_hz_staging(BatchArgs a, unsigned int* flag) {
  __shared__ uint64_t wmax[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  uint64_t carry = 0;   // largest range end of the earlier chunks
  bool bad = false;
  for (uint64_t base = 0; base < a.nreq; base += blockDim.x) {
    const uint64_t r = base + threadIdx.x;
    uint64_t off = 0, end = 0;
    if (r < a.nreq) {
      const uint64_t p = a.pairs_in[2 * r + 1];   // L + kReqWeight for a request the sizing accepted
      if (p > kReqWeight) { off = a.req[r].host_off; end = off + (p - kReqWeight); }
    }
    uint64_t v = end;   // inclusive max-scan within the warp
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t t = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d && t > v) v = t;
    }
    const uint64_t lane_excl = __shfl_up_sync(0xffffffffu, v, 1);
    if (lane == 31) wmax[wid] = v;
    __syncthreads();
    if (wid == 0) {   // exclusive max-scan of the warp maxima
      uint64_t x = lane < nwarp ? wmax[lane] : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t t = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d && t > x) x = t;
      }
      const uint64_t ex = __shfl_up_sync(0xffffffffu, x, 1);
      if (lane < nwarp) wmax[lane] = lane == 0 ? 0 : ex;
    }
    __syncthreads();
    uint64_t before = carry;
    if (wmax[wid] > before) before = wmax[wid];
    if (lane > 0 && lane_excl > before) before = lane_excl;
    if (end > off && off < before) bad = true;
    __syncthreads();
    // the chunk's largest end: the last warp's exclusive prefix and its own maximum
    const uint64_t last = __shfl_sync(0xffffffffu, v, 31);
    if (wid == nwarp - 1 && lane == 0) wmax[0] = last > wmax[nwarp - 1] ? last : wmax[nwarp - 1];
    __syncthreads();
    if (wmax[0] > carry) carry = wmax[0];
    __syncthreads();
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1u);
}

static uint32_t hz_shift(uint64_t cap) {
  uint32_t shift = 64;
  for (uint64_t c = cap; c > 1; c >>= 1) shift--;
  return shift;
}

static unsigned hz_blocks(uint32_t nreq) {
  unsigned blocks = (unsigned)num_sms() * 8;
  const uint64_t want = ((uint64_t)nreq + 7) / 8;
  if (want < blocks) blocks = (unsigned)(want ? want : 1);
  return blocks;
}

cudaError_t launch_hz_insert(const BatchArgs& a, unsigned long long* keys, unsigned long long* vals, uint64_t cap,
                             uint64_t epoch, bool staging_disjoint, unsigned int* flag, cudaStream_t st) {
  const uint32_t shift = hz_shift(cap);
  k_hz_insert<<<hz_blocks(a.nreq), 256, 0, st>>>(a, keys, vals, cap - 1, shift, epoch, flag);
  g_launches++;
  if (!staging_disjoint) {
    k_hz_staging<<<1, 1024, 0, st>>>(a, flag);
    g_launches++;
  }
  return cudaGetLastError();
}

cudaError_t launch_hz_mark(const BatchArgs& a, const unsigned long long* keys, const unsigned long long* vals,
                           uint64_t cap, uint64_t epoch, const unsigned int* flag, uint8_t* mark, unsigned int* nmarked,
                           cudaStream_t st) {
  k_hz_mark<<<hz_blocks(a.nreq), 256, 0, st>>>(a, keys, vals, cap - 1, hz_shift(cap), epoch, flag, mark, nmarked);
  g_launches++;
  return cudaGetLastError();
}

// A serving wave's inputs in one launch, read from mapped pinned host memory:
// the first n16 16-byte words of the wave's descriptor block (requests and
// segments) copied into device memory, and the runs (a copy-to request's
// source bytes gathered into its staging range) copied by one warp each, the
// warp reading the run's record from the host block.
__global__ void __launch_bounds__(256) k_wave_in(const uint4* __restrict__ h, uint4* __restrict__ d, uint64_t n16,
                                                 const Run* __restrict__ h_runs, uint64_t nruns) {
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = t; i < n16; i += nt) d[i] = h[i];
  const int lane = threadIdx.x & 31;
  for (uint64_t i = t >> 5; i < nruns; i += nt >> 5) {
    const Run r = h_runs[i];
    uint8_t* dst = reinterpret_cast<uint8_t*>((uintptr_t)r.dst);
    if (r.src) warp_copy<16, 2>(dst, reinterpret_cast<const uint8_t*>((uintptr_t)r.src), r.len, lane);
    else warp_zero<16>(dst, r.len, lane);
  }
}

cudaError_t launch_wave_in(const void* h_block, void* d_block, uint64_t n16, const Run* h_runs, uint64_t nruns,
                           cudaStream_t st) {
  if (!n16 && !nruns) return cudaSuccess;
  const uint64_t want = std::max<uint64_t>((n16 + 255) / 256, (nruns + 7) / 8);
  const unsigned blocks = (unsigned)std::min<uint64_t>(std::max<uint64_t>(want, 1), (uint64_t)num_sms() * 8);
  k_wave_in<<<blocks, 256, 0, st>>>(static_cast<const uint4*>(h_block), static_cast<uint4*>(d_block), n16, h_runs,
                                    nruns);
  g_launches++;
  return cudaGetLastError();
}

cudaError_t launch_run_copy(const Run* runs, uint64_t n, cudaStream_t st) {
  if (!n) return cudaSuccess;
  unsigned blocks = (unsigned)num_sms() * 8;
  uint64_t want = (n + 7) / 8;
  if (want < blocks) blocks = (unsigned)want;
  k_run_copy<<<blocks, 256, 0, st>>>(runs, n);
  g_launches++;
  return cudaGetLastError();
}

}  // namespace cvd
