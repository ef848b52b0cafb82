// cvd_kernels.cu -- translation, planning and copy kernels (sm_103a).
//
// Paper: Sec. 4.2 -- the CVD backend services copy_from_user/copy_to_user on
// a guest user buffer by walking the guest page tables in software
// (gVA -> gPA), turning the gPA into a host address through KVM's memslots,
// once per page, and then copying; Sec. 6.2 -- these are redirected kernel
// memory routines called by an unmodified host driver.
//
// B300 design: guest arenas, page tables, requests and staging all resident
// in HBM.  One warp plans one request (lanes walk pages in parallel, a ballot
// picks the first fault); a persistent grid copies a byte-balanced work list
// (fixed-size chunks of the concatenated request streams, taken from an
// atomic counter).  Two copy engines move the bytes: engine 0 realigns 16-byte
// vector loads in registers; engine 1 (default) streams each warp's pieces
// through a ring of shared-memory stages filled by bulk (TMA) copies.
#include <cstdio>
#include "cvd_internal.h"

namespace cvd {

unsigned long long g_launches = 0;

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

template <class K>
static void allow_smem(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Resident blocks per SM of a kernel at its launch shape (queried once).
template <class K>
static unsigned resident_blocks(K kernel, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  return (unsigned)n;
}

// ---------------------------------------------------------------------------
// a1/a2: translate (persistent grid, top levels in smem; each thread keeps
// kTranslateWalks walks in flight, gVAs i, i + stride, ... so that every
// warp-wide load stays coalesced)
// ---------------------------------------------------------------------------
constexpr int kTranslateWalks = 2;

template <int N>
__global__ void __launch_bounds__(256) k_translate(const DevGuest* __restrict__ gp, const uint64_t* __restrict__ gva, uint64_t n,
                                                   int write, uint64_t* __restrict__ gpa, uint64_t* __restrict__ hpa,
                                                   uint32_t* __restrict__ code) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DevGuest& G = *gp;
  TopCache* tc = reinterpret_cast<TopCache*>(smem);
  stage_top(tc, G);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += N * stride) {
    uint64_t va[N];
    WalkOut w[N];
#pragma unroll
    for (int k = 0; k < N; k++) {
      const uint64_t j = i + k * stride;
      va[k] = j < n ? __ldcs(gva + j) : (1ull << 63) | 1ull;   // past the end: non-canonical, no table read
    }
    walk_multi<N>(G, tc, va, write != 0, w);
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

void translate_shape(uint32_t* threads_per_sm, uint32_t* walks_per_thread) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_translate<kTranslateWalks>, 256, sizeof(TopCache)) !=
      cudaSuccess) {
    cudaGetLastError();
    b = 0;
  }
  if (b > 8) b = 8;   // launch_translate starts at most 8 blocks per SM
  *threads_per_sm = (uint32_t)b * 256;
  *walks_per_thread = kTranslateWalks;
}

cudaError_t launch_translate(const DevGuest* g, const uint64_t* gva, uint64_t n, bool write, uint64_t* gpa,
                             uint64_t* hpa, uint32_t* code, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  // one resident wave (a second, partial wave would run under-occupied)
  static const unsigned res = resident_blocks(k_translate<kTranslateWalks>, 256, sizeof(TopCache));
  uint64_t want = (n + 255) / 256;
  uint64_t cap = (uint64_t)num_sms() * (res < 8 ? res : 8);
  unsigned blocks = (unsigned)(want < cap ? want : cap);
  k_translate<kTranslateWalks><<<blocks, 256, sizeof(TopCache), st>>>(g, gva, n, write ? 1 : 0, gpa, hpa, code);
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
  if (blockIdx.x == 0 && threadIdx.x == 0) a.counter[1] = 0;   // k_plan's request counter
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
      a.pairs_in[2 * r] = code == kOk ? q.seg_count : 0;
      a.pairs_in[2 * r + 1] = code == kOk ? L + kReqWeight : 0;   // balancing position, see kReqWeight
      Result o;
      o.done = 0; o.fault_gva = 0; o.fault_code = code; o.pad = 0;
      a.res[r] = o;
    }
  }
}

// ---------------------------------------------------------------------------
// a6: planner.  One warp per request: stream offsets (warp scan), first fault
// (segment checks, then page walks: lane-local for segments of <= 2 pages,
// warp-cooperative for longer ones; a ballot picks the first faulting lane),
// then per-segment work records.
// ---------------------------------------------------------------------------
struct Fault1 { uint64_t off, gva; uint32_t code; };

// First fault inside [gva, gva+len) (already range-checked), warp cooperative:
// lane k walks the k-th page from pos; the walked spans cover [pos, max end)
// without gaps (each span reaches at least its page end), so the first
// faulting lane holds the first faulting byte.  off = ~0 if none.
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
    if (active) w = walk(G, tc, va, write);
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

template <bool STAGE>
__global__ void __launch_bounds__(256) k_plan(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  TopCache* tc = nullptr;
  if (STAGE) {
    tc = reinterpret_cast<TopCache*>(smem);
    stage_top(tc, *a.single);
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
        if (!canonical(s.gva)) { mine.off = soff; mine.gva = s.gva; mine.code = kNonCanonical; }
        else if (s.gva >= kUserTop || s.len > kUserTop - s.gva) { mine.off = soff; mine.gva = s.gva; mine.code = kRange; }
        else {
          uint64_t n = ((s.gva + s.len - 1) >> 12) - (s.gva >> 12) + 1;
          if (n <= 2) {
            WalkOut w1 = walk(G, t, s.gva, write);
            if (w1.code != kOk) { mine.off = soff; mine.gva = s.gva; mine.code = w1.code; }
            else if (w1.span < s.len) {
              uint64_t va2 = s.gva + w1.span;
              WalkOut w2 = walk(G, t, va2, write);
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
          WalkOut w = walk(G, t, va, write);
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
        Fault1 f = seg_first_fault(G, t, lg, ll, write, lane);
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


cudaError_t launch_plan(const BatchArgs& a, cudaStream_t st) {
  int sms = num_sms();
  unsigned blocks = (unsigned)sms * 8;
  uint64_t want = ((uint64_t)a.nreq + 7) / 8;
  if (want < blocks) blocks = (unsigned)(want ? want : 1);
  k_req_sizes<<<blocks, 256, 0, st>>>(a);
  g_launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_scan_pairs(a.pairs_in, a.pairs_out, a.nreq, a.scan_tmp, st);
  if (e != cudaSuccess) return e;
  // one resident wave: every block stages the top tables once, then warps
  // take requests from the counter until none is left
  static const unsigned res1 = resident_blocks(k_plan<true>, 256, sizeof(TopCache));
  static const unsigned res0 = resident_blocks(k_plan<false>, 256, 0);
  unsigned pb = (unsigned)sms * (a.nguests == 1 ? res1 : res0);
  uint64_t pwant = ((uint64_t)a.nreq + 8 * kPlanGrab - 1) / (8 * kPlanGrab);
  if (pwant < pb) pb = (unsigned)(pwant ? pwant : 1);
  if (a.nguests == 1) k_plan<true><<<pb, 256, sizeof(TopCache), st>>>(a);
  else k_plan<false><<<pb, 256, 0, st>>>(a);
  g_launches++;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a3/a4/a8: persistent byte-balanced copy engine (hazard-free batches)
// ---------------------------------------------------------------------------
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

// Copy part [a0, a1) of a segment (segment-local offsets), warp cooperative:
// lanes translate up to 32 pages at once, host-contiguous pieces are merged
// into runs, each run is moved by warp_copy.
template <int VEC, int U>
__device__ void copy_piece(const DevGuest& G, const TopCache* tc, const SegWork& s, uint64_t stg_base,
                           uint8_t* stg, bool to_guest, uint64_t a0, uint64_t a1, int lane) {
  uint64_t end = s.gva + a1;
  uint64_t pos = s.gva + a0;
  uint64_t pend_va = 0, pend_h = 0, pend_n = 0;
  while (pos < end) {
    uint64_t va = lane == 0 ? pos : (pos & ~4095ull) + (uint64_t)lane * 4096;
    bool active = va < end;
    WalkOut w;
    w.code = kOk; w.span = 0; w.hpa = 0;
    if (active) w = walk(G, tc, va, to_guest);
    unsigned bad = __ballot_sync(0xffffffffu, active && w.code != kOk);
    uint64_t stop = end;
    if (bad) stop = __shfl_sync(0xffffffffu, va, __ffs(bad) - 1);   // tables changed under us: stop there
    unsigned act = __ballot_sync(0xffffffffu, active && (va < stop));
    uint64_t np = pos;
    while (act) {
      int k = __ffs(act) - 1;
      act &= act - 1;
      uint64_t kva = __shfl_sync(0xffffffffu, va, k);
      uint64_t kh = __shfl_sync(0xffffffffu, w.hpa, k);
      uint64_t ks = __shfl_sync(0xffffffffu, w.span, k);
      uint64_t kend = kva + ks < stop ? kva + ks : stop;
      if (kend <= np) continue;
      uint64_t h = kh + (np - kva);
      uint64_t n = kend - np;
      if (pend_n && pend_h + pend_n == h) {
        pend_n += n;
      } else {
        if (pend_n) {
          uint8_t* gp = G.pool + pend_h;
          uint8_t* sp = stg + stg_base + (pend_va - s.gva);
          if (to_guest) warp_copy<VEC, U>(gp, sp, pend_n, lane);
          else warp_copy<VEC, U>(sp, gp, pend_n, lane);
        }
        pend_va = np; pend_h = h; pend_n = n;
      }
      np = kend;
    }
    if (bad || np == pos) break;
    pos = np;
  }
  if (pend_n) {
    uint8_t* gp = G.pool + pend_h;
    uint8_t* sp = stg + stg_base + (pend_va - s.gva);
    if (to_guest) warp_copy<VEC, U>(gp, sp, pend_n, lane);
    else warp_copy<VEC, U>(sp, gp, pend_n, lane);
  }
}

// Lane-local copy of a small segment (whole copy part + zero part).
__device__ void copy_small(const DevGuest& G, const TopCache* tc, const SegWork& s, uint64_t stg_base, uint8_t* stg,
                           bool to_guest) {
  uint64_t off = 0;
  while (off < s.ncopy) {
    WalkOut w = walk(G, tc, s.gva + off, to_guest);
    if (w.code != kOk) break;
    uint64_t n = s.ncopy - off < w.span ? s.ncopy - off : w.span;
    uint8_t* gp = G.pool + w.hpa;
    uint8_t* sp = stg + stg_base + off;
    if (to_guest) for (uint64_t i = 0; i < n; i++) gp[i] = sp[i];
    else for (uint64_t i = 0; i < n; i++) sp[i] = gp[i];
    off += n;
  }
  if (!to_guest)
    for (uint64_t i = s.ncopy; i < s.len; i++) stg[stg_base + i] = 0;
}

template <int VEC, int U, bool STAGE>
__global__ void __launch_bounds__(256, 2) k_copy(BatchArgs a, uint64_t chunk, uint64_t small) {
  extern __shared__ __align__(16) unsigned char smem[];
  TopCache* tc = nullptr;
  if (STAGE) {
    tc = reinterpret_cast<TopCache*>(smem);
    stage_top(tc, *a.single);
  }
  int lane = threadIdx.x & 31;
  const uint64_t total = a.pairs_out[2 * (uint64_t)a.nreq + 1];
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (;;) {
    uint64_t cs, ce;
    if (!next_chunk(a.counter, total, chunk, nwarps, lane, &cs, &ce)) break;
    uint64_t r = find_req(a.pairs_out, a.nreq, cs, lane);
    uint64_t b = cs;
    while (b < ce && r < a.nreq) {
      uint64_t Rr = a.pairs_out[2 * r + 1];
      uint64_t Rn = (r + 1 < a.nreq) ? a.pairs_out[2 * (r + 1) + 1] : total;
      if (Rn <= b) { r++; continue; }
      ReqWork rw = a.rw[r];
      const uint64_t lo = Rr + kReqWeight;               // stream position of the request's byte 0
      const uint64_t we = ce < Rn ? ce : Rn;
      const uint64_t wa = b > lo ? b - lo : 0, wb = we > lo ? we - lo : 0;
      if (rw.nsw && wa < wb) {
        uint32_t gi = rw.guest_dir >> 1;
        bool to_guest = rw.guest_dir & 1;
        const DevGuest& G = STAGE ? *a.single : *a.guests[gi];
        const TopCache* t = STAGE ? tc : nullptr;
        for (uint32_t g0 = 0; g0 < rw.nsw; g0 += 32) {
          uint32_t j = g0 + lane;
          bool valid = j < rw.nsw;
          SegWork s;
          if (valid) s = a.sw[rw.sb + j];
          else { s.gva = 0; s.soff = ~0ull; s.len = 0; s.ncopy = 0; }
          uint64_t last_end = valid ? s.soff + s.len : 0;
          if (warp_max(last_end) <= wa) continue;                 // group before the window
          uint64_t first = __shfl_sync(0xffffffffu, s.soff, 0);
          if (first >= wb) break;                                // group after the window
          bool is_small = valid && s.len <= small;
          if (is_small && s.len > 0 && s.soff >= wa && s.soff < wb)
            copy_small(G, t, s, rw.host_off + s.soff, a.stg, to_guest);
          unsigned lm = __ballot_sync(0xffffffffu, valid && !is_small && s.soff < wb && s.soff + s.len > wa);
          while (lm) {
            int l = __ffs(lm) - 1;
            lm &= lm - 1;
            SegWork ls;
            ls.gva = __shfl_sync(0xffffffffu, s.gva, l);
            ls.soff = __shfl_sync(0xffffffffu, s.soff, l);
            ls.len = __shfl_sync(0xffffffffu, s.len, l);
            ls.ncopy = __shfl_sync(0xffffffffu, s.ncopy, l);
            uint64_t pa = wa > ls.soff ? wa - ls.soff : 0;
            uint64_t pb = wb - ls.soff < ls.len ? wb - ls.soff : ls.len;
            uint64_t sbase = rw.host_off + ls.soff;
            uint64_t c1 = pb < ls.ncopy ? pb : ls.ncopy;
            if (pa < c1) copy_piece<VEC, U>(G, t, ls, sbase, a.stg, to_guest, pa, c1, lane);
            if (!to_guest) {
              uint64_t z0 = pa > ls.ncopy ? pa : ls.ncopy;
              if (z0 < pb) warp_zero<VEC>(a.stg + sbase + z0, pb - z0, lane);
            }
          }
        }
      }
      b = ce < Rn ? ce : Rn;
      r++;
    }
  }
}

template <int VEC, int U>
static cudaError_t launch_copy_t(const BatchArgs& a, const CopyParams& p, cudaStream_t st) {
  unsigned threads = p.warps_per_block * 32;
  unsigned blocks = (unsigned)num_sms() * p.blocks_per_sm;
  if (a.nguests == 1)
    k_copy<VEC, U, true><<<blocks, threads, sizeof(TopCache), st>>>(a, p.chunk_bytes, p.small_bytes);
  else
    k_copy<VEC, U, false><<<blocks, threads, 0, st>>>(a, p.chunk_bytes, p.small_bytes);
  g_launches++;
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Copy engine 1: per-warp ring of shared-memory stages filled by bulk (TMA)
// copies.  The copy loop (segment bookkeeping, page walks) appends host runs
// dst <- src to a small per-warp queue in shared memory; when the queue is
// full, and at the end, one streaming routine moves the queued runs: each run
// is cut into pieces of <= stage_bytes; lane 0 issues one cp.async.bulk
// global->shared of the piece's 16-byte-aligned source window, completing on
// the slot's mbarrier; when the ring or the slots are full the oldest piece
// is consumed: lanes rebuild 16-byte destination-aligned words from two
// 16-byte shared loads (funnel shift by the relative misalignment) and store
// them.  Pieces stay in flight across calls, so their loads overlap the walks
// that produce the next runs.  Inside the streaming routine the ring state is
// held in registers and the per-piece path makes no call; between calls it
// lives in the warp's control block in shared memory.  (Per-piece calls that
// pass the state through local memory cost several microseconds a piece:
// with most of the SM's unified L1/shared storage given to the rings, local
// memory goes to L2.)  Every wait is bounded; a wait that gives up sets an
// error bit in the device error word and the piece is skipped.
// ---------------------------------------------------------------------------
struct Piece { uint64_t dst, src; uint32_t len, off; };   // in flight; off: window offset in the ring

// Runs a warp queues before streaming them.
constexpr uint32_t kQueueRuns = 16;

// Per-warp control block at the start of the warp's shared-memory region,
// followed by bar[K] (u64), desc[K] (Piece), q[kQueueRuns] (Run) and, at the
// next 128-byte boundary, the byte ring.
struct WarpPipe {
  uint32_t head, tail, phase;   // pieces in flight [head, tail); per-slot parity bits
  uint32_t rd, wr;              // ring bytes of the pieces in flight: [rd, wr), wrapping
  uint32_t nq;                  // queued runs
  uint32_t ring, K, stage, pad;
  unsigned int* err;
};
static_assert(sizeof(WarpPipe) <= 64, "WarpPipe control block");

__host__ __device__ constexpr uint32_t round128(uint32_t x) { return (x + 127u) & ~127u; }
__host__ __device__ constexpr uint32_t wp_ring_off(uint32_t K) { return round128(64u + 32u * K + 32u * kQueueRuns); }

__device__ __forceinline__ uint64_t* wp_bar(WarpPipe* w) {
  return reinterpret_cast<uint64_t*>(reinterpret_cast<uint8_t*>(w) + 64);
}
__device__ __forceinline__ Piece* wp_desc(WarpPipe* w, uint32_t K) {
  return reinterpret_cast<Piece*>(reinterpret_cast<uint8_t*>(w) + 64 + 8 * K);
}
__device__ __forceinline__ Run* wp_queue(WarpPipe* w, uint32_t K) {
  return reinterpret_cast<Run*>(reinterpret_cast<uint8_t*>(w) + 64 + 32 * K);
}

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(saddr(dst_smem)), "l"(src), "r"(bytes), "r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: try_wait suspends for a hardware-defined time per attempt;
// 2^22 attempts is far beyond any completion time of a 16 KiB copy.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < (1u << 22); i++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// One loop for every relative misalignment: output word i is bytes
// [4(q+i) + r, 4(q+i) + r + 4) of the 32-byte pair of aligned shared words;
// q is warp-uniform, so the word select costs a few predicated moves and the
// kernel keeps one compact copy of the loop.
__device__ __forceinline__ void consume(const uint8_t* slot, const Piece& pc, int lane) {
  uint8_t* d = reinterpret_cast<uint8_t*>((uintptr_t)pc.dst);
  const uint8_t* sm = slot + (pc.src & 15);
  uint32_t n = pc.len;
  uint32_t head = (16u - (uint32_t)(pc.dst & 15)) & 15u;
  if (head > n) head = n;
  if ((uint32_t)lane < head) d[lane] = sm[lane];
  d += head; sm += head; n -= head;
  const uint32_t nvec = n >> 4;
  const uint32_t off = (uint32_t)(sm - slot);
  const uint8_t* al = slot + (off & ~15u);
  const uint32_t sh = off & 15u, q = sh >> 2, r = sh & 3u;
#pragma unroll 2   // two iterations' shared loads in flight
  for (uint32_t v = lane; v < nvec; v += 32) {
    uint4 x = *reinterpret_cast<const uint4*>(al + 16u * v);
    uint4 y = sh ? *reinterpret_cast<const uint4*>(al + 16u * v + 16u) : x;
    uint32_t w0 = x.x, w1 = x.y, w2 = x.z, w3 = x.w, w4 = y.x, w5 = y.y, w6 = y.z, w7 = y.w;
    if (q & 2) { w0 = w2; w1 = w3; w2 = w4; w3 = w5; w4 = w6; w5 = w7; }
    if (q & 1) { w0 = w1; w1 = w2; w2 = w3; w3 = w4; w4 = w5; }
    uint4 out;
    out.x = fsh(w0, w1, r);
    out.y = fsh(w1, w2, r);
    out.z = fsh(w2, w3, r);
    out.w = fsh(w3, w4, r);
    __stcs(reinterpret_cast<uint4*>(d + 16u * v), out);
  }
  const uint32_t done = nvec * 16u;
  if ((uint32_t)lane < n - done) d[done + lane] = sm[done + lane];
}

// Stream the queued runs through the ring; with drain, also consume every
// piece still in flight.  A piece's source window takes contiguous ring bytes
// (wrapping to offset 0 when the tail is too short); the oldest piece is
// consumed whenever the next window or descriptor slot does not fit.  All
// lanes call it.
__device__ __noinline__ void wp_stream(WarpPipe* w, bool drain, int lane) {
  const uint32_t K = w->K, ring = w->ring, stage = w->stage, nq = w->nq;
  uint64_t* bar = wp_bar(w);
  Piece* desc = wp_desc(w, K);
  const Run* q = wp_queue(w, K);
  uint8_t* buf = reinterpret_cast<uint8_t*>(w) + wp_ring_off(K);
  uint32_t head = w->head, tail = w->tail, phase = w->phase, rd = w->rd, wr = w->wr;
  uint32_t i = 0;   // current run
  uint64_t o = 0;   // its bytes already issued
  for (;;) {
    if (i < nq) {
      const Run r = q[i];
      const uint64_t src = r.src + o, dst = r.dst + o;
      const uint32_t len = r.len - o < stage ? (uint32_t)(r.len - o) : stage;
      const uint64_t a0 = src & ~15ull;
      const uint32_t wb = (uint32_t)(((src + len + 15) & ~15ull) - a0);
      uint32_t at = ~0u;
      if (tail - head < K) {
        if (head == tail) at = 0;
        else if (wr > rd) {            // occupied [rd, wr): free [wr, ring) and [0, rd)
          if (ring - wr >= wb) at = wr;
          else if (rd >= wb) at = 0;
        } else if (wr < rd) {          // wrapped: free [wr, rd)
          if (rd - wr >= wb) at = wr;
        }
      }
      if (at != ~0u) {
        const uint32_t s = tail % K;
        if (lane == 0) {
          Piece pc;
          pc.dst = dst; pc.src = src; pc.len = len; pc.off = at;
          desc[s] = pc;
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // ring bytes were read by the generic proxy
          mbar_expect_tx(&bar[s], wb);
          bulk_g2s(buf + at, reinterpret_cast<const void*>((uintptr_t)a0), wb, &bar[s]);
        }
        __syncwarp();
        wr = at + wb;
        tail++;
        o += len;
        if (o >= r.len) { i++; o = 0; }
        continue;
      }
    } else if (!drain || head == tail) {
      break;
    }
    // no room for the next piece (or draining): consume the oldest one
    const uint32_t s = head % K;
    const Piece pc = desc[s];
    const bool ok = mbar_wait_bounded(&bar[s], (phase >> s) & 1u);
    phase ^= 1u << s;
    if (ok) consume(buf + pc.off, pc, lane);
    else if (lane == 0) atomicOr(w->err, kErrWaitTimeout);
    __syncwarp();
    head++;
    if (head == tail) rd = wr = 0;
    else rd = desc[head % K].off;
  }
  if (lane == 0) {
    w->head = head; w->tail = tail; w->phase = phase; w->rd = rd; w->wr = wr; w->nq = 0;
  }
  __syncwarp();
}

// Queue the host run dst <- src (n bytes); a run contiguous on both sides with
// the last queued one extends it.  Streams the queue when it is full.  All
// lanes call it with identical arguments.
__device__ __forceinline__ void wp_add(WarpPipe* w, uint64_t dst, uint64_t src, uint64_t n, int lane) {
  if (!n) return;
  const uint32_t K = w->K, nq = w->nq;
  Run* q = wp_queue(w, K);
  if (nq) {
    const Run last = q[nq - 1];
    if (last.dst + last.len == dst && last.src + last.len == src) {
      __syncwarp();
      if (lane == 0) q[nq - 1].len = last.len + n;
      __syncwarp();
      return;
    }
  }
  __syncwarp();
  if (lane == 0) {
    Run r;
    r.dst = dst; r.src = src; r.len = n; r.pad = 0;
    q[nq] = r;
    w->nq = nq + 1;
  }
  __syncwarp();
  if (nq + 1 == kQueueRuns) wp_stream(w, false, lane);
}

__device__ __noinline__ WalkOut walk_ni(const DevGuest& G, const TopCache* tc, uint64_t va, bool write) {
  return walk(G, tc, va, write);
}

// Queue part [a0, a1) of a segment (warp cooperative): lanes translate up to
// 32 pages at once; each host-contiguous piece becomes a run.
__device__ __noinline__ void copy_piece_q(WarpPipe* wp, const DevGuest& G, const TopCache* tc, SegWork s,
                                          uint64_t stg_base, uint8_t* stg, bool to_guest, uint64_t a0, uint64_t a1,
                                          int lane) {
  const uint64_t end = s.gva + a1;
  uint64_t pos = s.gva + a0;
  while (pos < end) {
    uint64_t va = lane == 0 ? pos : (pos & ~4095ull) + (uint64_t)lane * 4096;
    bool active = va < end;
    WalkOut w;
    w.code = kOk; w.span = 0; w.hpa = 0;
    if (active) w = walk_ni(G, tc, va, to_guest);
    unsigned bad = __ballot_sync(0xffffffffu, active && w.code != kOk);
    uint64_t stop = end;
    if (bad) stop = __shfl_sync(0xffffffffu, va, __ffs(bad) - 1);
    unsigned act = __ballot_sync(0xffffffffu, active && (va < stop));
    uint64_t np = pos;
    while (act) {
      int k = __ffs(act) - 1;
      act &= act - 1;
      uint64_t kva = __shfl_sync(0xffffffffu, va, k);
      uint64_t kh = __shfl_sync(0xffffffffu, w.hpa, k);
      uint64_t ks = __shfl_sync(0xffffffffu, w.span, k);
      uint64_t kend = kva + ks < stop ? kva + ks : stop;
      if (kend <= np) continue;
      const uint64_t gp = (uint64_t)(uintptr_t)(G.pool + kh + (np - kva));
      const uint64_t sp = (uint64_t)(uintptr_t)(stg + stg_base + (np - s.gva));
      wp_add(wp, to_guest ? gp : sp, to_guest ? sp : gp, kend - np, lane);
      np = kend;
    }
    if (bad || np == pos) break;
    pos = np;
  }
}

__device__ __noinline__ void copy_small_ni(const DevGuest& G, const TopCache* tc, const SegWork& s, uint64_t stg_base,
                                           uint8_t* stg, bool to_guest) {
  copy_small(G, tc, s, stg_base, stg, to_guest);
}

// Segments whose copy part spans at most this many 4 KiB pages are translated
// together: one parallel walk round covers the pages of every short segment
// of a 32-segment group, instead of one serial round per segment.
constexpr uint32_t kShortPages = 8;

// Queue copy parts [gva+pa, gva+c1) of the lanes with mine = true, batched:
// the pages of all of them are enumerated across the warp (item i -> owner
// lane by a shuffle binary search over the inclusive page-count scan), walked
// in parallel, then queued in order.
__device__ __noinline__ void copy_group_short(WarpPipe* wp, const DevGuest& G, const TopCache* tc, uint64_t gva,
                                              uint64_t soff, bool mine, uint64_t pa, uint64_t c1, uint64_t host_off,
                                              uint8_t* stg, bool to_guest, int lane) {
  const uint64_t start = gva + pa, end = gva + c1;
  const uint32_t np = mine ? (uint32_t)(((end - 1) >> 12) - (start >> 12) + 1) : 0u;
  uint32_t incl = np;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += t;
  }
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
  for (uint32_t base = 0; base < total; base += 32) {
    const uint32_t item = base + lane;
    int lo = 0, hi = 31;   // owner = smallest lane whose inclusive count exceeds item
#pragma unroll
    for (int it = 0; it < 5; it++) {
      int mid = (lo + hi) >> 1;
      uint32_t v = __shfl_sync(0xffffffffu, incl, mid);
      if (v > item) hi = mid; else lo = mid + 1;
    }
    const int L = lo;
    const uint32_t before = __shfl_sync(0xffffffffu, incl - np, L);
    const uint64_t ostart = __shfl_sync(0xffffffffu, start, L);
    const uint32_t k = item - before;
    const uint64_t va = k == 0 ? ostart : (ostart & ~4095ull) + (uint64_t)k * 4096;
    const bool active = item < total;
    WalkOut w;
    w.code = kOk; w.hpa = 0; w.span = 0;
    if (active) w = walk_ni(G, tc, va, to_guest);
    const uint32_t nit = total - base < 32 ? total - base : 32;
    for (uint32_t j = 0; j < nit; j++) {
      const int jl = __shfl_sync(0xffffffffu, L, j);
      const uint64_t jva = __shfl_sync(0xffffffffu, va, j);
      const uint64_t jh = __shfl_sync(0xffffffffu, w.hpa, j);
      const uint32_t jc = __shfl_sync(0xffffffffu, w.code, j);
      const uint64_t jend = __shfl_sync(0xffffffffu, end, jl);
      const uint64_t jgva = __shfl_sync(0xffffffffu, gva, jl);
      const uint64_t jsoff = __shfl_sync(0xffffffffu, soff, jl);
      if (jc != kOk) continue;   // tables changed under the call: unspecified, skip
      const uint64_t pe = (jva & ~4095ull) + 4096;
      const uint64_t n = (pe < jend ? pe : jend) - jva;
      const uint64_t sp = (uint64_t)(uintptr_t)(stg + host_off + jsoff + (jva - jgva));
      const uint64_t gp = (uint64_t)(uintptr_t)(G.pool + jh);
      wp_add(wp, to_guest ? gp : sp, to_guest ? sp : gp, n, lane);
    }
  }
}

template <bool STAGE>
__global__ void __launch_bounds__(1024) k_copy_tma(BatchArgs a, uint64_t chunk, uint64_t small, uint32_t K,
                                                   uint32_t stage, uint32_t ring) {
  extern __shared__ __align__(16) unsigned char smem[];
  TopCache* tc = nullptr;
  unsigned char* base = smem;
  if (STAGE) {
    tc = reinterpret_cast<TopCache*>(smem);
    stage_top(tc, *a.single);
    base += round128((uint32_t)sizeof(TopCache));
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  WarpPipe* wp = reinterpret_cast<WarpPipe*>(base + (size_t)wid * (wp_ring_off(K) + ring));
  if (lane == 0) {
    wp->head = wp->tail = wp->phase = 0;
    wp->rd = wp->wr = 0;
    wp->nq = 0;
    wp->ring = ring; wp->K = K; wp->stage = stage; wp->pad = 0;
    wp->err = a.err;
  }
  if ((uint32_t)lane < K) mbar_init(&wp_bar(wp)[lane], 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncwarp();

  const uint64_t total = a.pairs_out[2 * (uint64_t)a.nreq + 1];
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (;;) {
    uint64_t cs, ce;
    if (!next_chunk(a.counter, total, chunk, nwarps, lane, &cs, &ce)) break;
    uint64_t r = find_req(a.pairs_out, a.nreq, cs, lane);
    uint64_t b = cs;
    while (b < ce && r < a.nreq) {
      uint64_t Rr = a.pairs_out[2 * r + 1];
      uint64_t Rn = (r + 1 < a.nreq) ? a.pairs_out[2 * (r + 1) + 1] : total;
      if (Rn <= b) { r++; continue; }
      ReqWork rw = a.rw[r];
      const uint64_t lo = Rr + kReqWeight;               // stream position of the request's byte 0
      const uint64_t we = ce < Rn ? ce : Rn;
      const uint64_t wa = b > lo ? b - lo : 0, wb = we > lo ? we - lo : 0;
      if (rw.nsw && wa < wb) {
        uint32_t gi = rw.guest_dir >> 1;
        bool to_guest = rw.guest_dir & 1;
        const DevGuest& G = STAGE ? *a.single : *a.guests[gi];
        const TopCache* t = STAGE ? tc : nullptr;
        for (uint32_t g0 = 0; g0 < rw.nsw; g0 += 32) {
          uint32_t j = g0 + lane;
          bool valid = j < rw.nsw;
          SegWork s;
          if (valid) s = a.sw[rw.sb + j];
          else { s.gva = 0; s.soff = ~0ull; s.len = 0; s.ncopy = 0; }
          uint64_t last_end = valid ? s.soff + s.len : 0;
          if (warp_max(last_end) <= wa) continue;
          uint64_t first = __shfl_sync(0xffffffffu, s.soff, 0);
          if (first >= wb) break;
          bool is_small = valid && s.len <= small;
          if (is_small && s.len > 0 && s.soff >= wa && s.soff < wb)
            copy_small_ni(G, t, s, rw.host_off + s.soff, a.stg, to_guest);
          // this lane's part of its segment inside the window
          const bool ov = valid && !is_small && s.soff < wb && s.soff + s.len > wa;
          uint64_t pa = 0, pb = 0, c1 = 0;
          if (ov) {
            pa = wa > s.soff ? wa - s.soff : 0;
            pb = wb - s.soff < s.len ? wb - s.soff : s.len;
            c1 = pb < s.ncopy ? pb : s.ncopy;
          }
          const bool cp = ov && pa < c1;
          const bool shortseg = cp && (((s.gva + c1 - 1) >> 12) - ((s.gva + pa) >> 12) + 1) <= kShortPages;
          if (__any_sync(0xffffffffu, shortseg))
            copy_group_short(wp, G, t, s.gva, s.soff, shortseg, pa, c1, rw.host_off, a.stg, to_guest, lane);
          unsigned lm = __ballot_sync(0xffffffffu, cp && !shortseg);
          while (lm) {
            int l = __ffs(lm) - 1;
            lm &= lm - 1;
            SegWork ls;
            ls.gva = __shfl_sync(0xffffffffu, s.gva, l);
            ls.soff = __shfl_sync(0xffffffffu, s.soff, l);
            ls.len = __shfl_sync(0xffffffffu, s.len, l);
            ls.ncopy = __shfl_sync(0xffffffffu, s.ncopy, l);
            uint64_t lpa = __shfl_sync(0xffffffffu, pa, l), lc1 = __shfl_sync(0xffffffffu, c1, l);
            copy_piece_q(wp, G, t, ls, rw.host_off + ls.soff, a.stg, to_guest, lpa, lc1, lane);
          }
          if (!to_guest) {   // zero-fill after a fault (copy from guest)
            uint64_t z0 = pa > s.ncopy ? pa : s.ncopy;
            unsigned zm = __ballot_sync(0xffffffffu, ov && z0 < pb);
            while (zm) {
              int l = __ffs(zm) - 1;
              zm &= zm - 1;
              uint64_t lz0 = __shfl_sync(0xffffffffu, z0, l), lpb = __shfl_sync(0xffffffffu, pb, l);
              uint64_t lsoff = __shfl_sync(0xffffffffu, s.soff, l);
              warp_zero<16>(a.stg + rw.host_off + lsoff + lz0, lpb - lz0, lane);
            }
          }
        }
      }
      b = ce < Rn ? ce : Rn;
      r++;
    }
  }
  wp_stream(wp, true, lane);   // drain: no copy may be in flight at exit
}

size_t copy_smem_bytes(const CopyParams& p, bool staged) {
  if (p.engine == 0) return staged ? sizeof(TopCache) : 0;
  uint32_t per_warp = wp_ring_off(p.stages) + p.ring_bytes;
  return (staged ? round128((uint32_t)sizeof(TopCache)) : 0) + (size_t)p.warps_per_block * per_warp;
}

static cudaError_t launch_copy_tma(const BatchArgs& a, const CopyParams& p, cudaStream_t st) {
  unsigned threads = p.warps_per_block * 32;
  unsigned blocks = (unsigned)num_sms() * p.blocks_per_sm;
  size_t sm = copy_smem_bytes(p, a.nguests == 1);
  if (a.nguests == 1)
    k_copy_tma<true><<<blocks, threads, sm, st>>>(a, p.chunk_bytes, p.small_bytes, p.stages, p.stage_bytes,
                                                 p.ring_bytes);
  else
    k_copy_tma<false><<<blocks, threads, sm, st>>>(a, p.chunk_bytes, p.small_bytes, p.stages, p.stage_bytes,
                                                  p.ring_bytes);
  g_launches++;
  return cudaGetLastError();
}

// Set every dynamic-shared-memory attribute up front, so that no attribute
// call happens for the first time inside a stream capture.
void prepare_kernels() {
  static bool done = false;
  if (done) return;
  size_t sm = sizeof(TopCache);
  allow_smem(k_translate<kTranslateWalks>, sm);
  allow_smem(k_plan<true>, sm);
  allow_smem(k_copy<16, 1, true>, sm);
  allow_smem(k_copy<16, 2, true>, sm);
  allow_smem(k_copy<16, 4, true>, sm);
  allow_smem(k_copy<8, 4, true>, sm);
  allow_smem(k_copy<8, 2, true>, sm);
  allow_smem(k_copy<4, 4, true>, sm);
  allow_smem(k_copy_tma<true>, 227 * 1024);
  allow_smem(k_copy_tma<false>, 227 * 1024);
  num_sms();
  done = true;
}

bool copy_params_supported(const CopyParams& p) {
  if (p.engine > 1) return false;
  if (p.engine == 1) {
    if (p.stages < 1 || p.stages > 32 || p.stage_bytes < 512 || p.stage_bytes > 32768 || (p.stage_bytes & 15))
      return false;
    if ((p.ring_bytes & 127) || p.ring_bytes < round128(p.stage_bytes + 32)) return false;
    if (p.warps_per_block < 1 || p.warps_per_block > 32) return false;
    return copy_smem_bytes(p, true) <= 227 * 1024;
  }
  switch (p.vec_bytes * 10 + p.unroll) {
    case 161: case 162: case 164: case 84: case 82: case 44: return true;
    default: return false;
  }
}

cudaError_t launch_copy(const BatchArgs& a, const CopyParams& p, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (p.engine == 1) return launch_copy_tma(a, p, st);
  switch (p.vec_bytes * 10 + p.unroll) {
    case 161: return launch_copy_t<16, 1>(a, p, st);
    case 162: return launch_copy_t<16, 2>(a, p, st);
    case 164: return launch_copy_t<16, 4>(a, p, st);
    case 84: return launch_copy_t<8, 4>(a, p, st);
    case 82: return launch_copy_t<8, 2>(a, p, st);
    case 44: return launch_copy_t<4, 4>(a, p, st);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// a7: levelled engine -- explicit run list (in stream order) for the host
// leveller, then one copy launch per level.
// ---------------------------------------------------------------------------
// Walk the copy part of every segment of request r, merging host-contiguous
// pages into runs; plus one zero-fill run for a faulted copy-from request.
// EMIT=false counts runs into counts[2r]; EMIT=true writes them at offs[2r].
template <bool EMIT>
__global__ void __launch_bounds__(256) k_runs(BatchArgs a, uint64_t* counts, const uint64_t* offs, Run* runs) {
  int lane = threadIdx.x & 31;
  uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = w; r < a.nreq; r += nw) {
    ReqWork rw = a.rw[r];
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
                if (EMIT && lane == 0) {
                  uint64_t g = (uint64_t)(uintptr_t)(G.pool + pend_h);
                  uint64_t sp = (uint64_t)(uintptr_t)(a.stg + rw.host_off + s.soff + (pend_va - s.gva));
                  Run ru; ru.dst = to_guest ? g : sp; ru.src = to_guest ? sp : g; ru.len = pend_n; ru.pad = 0;
                  runs[out + cnt] = ru;
                }
                cnt++;
              }
              pend_va = np; pend_h = h; pend_n = n;
            }
            np = kend;
          }
          if (bad || np == pos) break;
          pos = np;
        }
        if (pend_n) {
          if (EMIT && lane == 0) {
            uint64_t g = (uint64_t)(uintptr_t)(G.pool + pend_h);
            uint64_t sp = (uint64_t)(uintptr_t)(a.stg + rw.host_off + s.soff + (pend_va - s.gva));
            Run ru; ru.dst = to_guest ? g : sp; ru.src = to_guest ? sp : g; ru.len = pend_n; ru.pad = 0;
            runs[out + cnt] = ru;
          }
          cnt++;
        }
      }
      if (!to_guest && done < L) {
        if (EMIT && lane == 0) {
          Run ru;
          ru.dst = (uint64_t)(uintptr_t)(a.stg + rw.host_off + done);
          ru.src = 0; ru.len = L - done; ru.pad = 0;
          runs[out + cnt] = ru;
        }
        cnt++;
      }
    }
    if (!EMIT && lane == 0) { counts[2 * r] = cnt; counts[2 * r + 1] = 0; }
  }
}

cudaError_t launch_runs(const BatchArgs& a, bool emit, uint64_t* counts, const uint64_t* offs, Run* runs,
                        cudaStream_t st) {
  unsigned blocks = (unsigned)num_sms() * 8;
  uint64_t want = ((uint64_t)a.nreq + 7) / 8;
  if (want < blocks) blocks = (unsigned)(want ? want : 1);
  if (emit) k_runs<true><<<blocks, 256, 0, st>>>(a, counts, offs, runs);
  else k_runs<false><<<blocks, 256, 0, st>>>(a, counts, offs, runs);
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
