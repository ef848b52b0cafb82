// cvd_copy.cu -- the copy engines of the batched copy path (sm_103a).
//
// Paper: Sec. 4.2 -- copy_from_user / copy_to_user on a guest user buffer,
// translated once per page (gVA -> gPA through the guest's tables, gPA ->
// host through KVM's memslots), then copied; Sec. 6.2 -- redirected kernel
// memory routines called by an unmodified host driver.
//
// B300 design: a persistent grid copies the planner's byte-balanced work list
// (windows of the concatenated request streams taken from a shared cursor).
// Engine 0 realigns 16-byte vector loads in registers; engine 1 (default)
// queues each warp's host runs and streams them through a shared-memory ring
// filled by bulk (TMA) copies.
#include <cstdio>
#include "cvd_internal.h"
#include "cvd_mbar.cuh"

namespace cvd {

// ---------------------------------------------------------------------------
// a3/a4/a8: persistent byte-balanced copy engine (hazard-free batches)
// ---------------------------------------------------------------------------
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
template <int PM>
__device__ void copy_small(const DevGuest& G, const TopCache* tc, const SegWork& s, uint64_t stg_base, uint8_t* stg,
                           bool to_guest) {
  uint64_t off = 0;
  while (off < s.ncopy) {
    WalkOut w = walk_t<PM>(G, tc, s.gva + off, to_guest);
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
            copy_small<kPmEpt>(G, t, s, rw.host_off + s.soff, a.stg, to_guest);
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

// The ordered pass of a levelled call: the requests the device conflict check
// marked, one after another in index order, by one block whose warps share
// each request's pages (a warp per page: walk, then the page's piece of the
// copied part; the zero-filled tail of a copy from guest likewise).  The
// block synchronises after every request, and after every segment of a copy
// to guest (two of its segments may write the same bytes; the later one
// wins), so every write of an earlier request or segment is visible to a
// later one.  nsw comes from the request's seg_count: the mark pass took it
// from the parallel launch.
constexpr int kOrderedWarps = 16;

__global__ void __launch_bounds__(kOrderedWarps * 32) k_ordered_copy(BatchArgs a, const uint8_t* __restrict__ mark,
                                                                     const unsigned int* __restrict__ nmarked) {
  if (*nmarked == 0) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (uint64_t r = 0; r < a.nreq; r++) {
    if (!mark[r]) continue;
    const ReqWork rw = a.rw[r];
    const uint32_t nsw = a.req[r].seg_count;
    const DevGuest& G = *a.guests[rw.guest_dir >> 1];
    const bool to_guest = rw.guest_dir & 1;
    uint32_t k = 0;   // running page index over the request (copy from guest: one pool of pages)
    for (uint32_t j = 0; j < nsw; j++) {
      const SegWork sg = a.sw[rw.sb + j];
      const uint64_t sbase = rw.host_off + sg.soff;
      const uint64_t end = sg.gva + sg.ncopy;
      const uint64_t npg = sg.ncopy ? ((end - 1) >> 12) - (sg.gva >> 12) + 1 : 0;
      for (uint64_t p = 0; p < npg; p++, k++) {
        if ((k % kOrderedWarps) != (uint32_t)wid) continue;
        const uint64_t va = p == 0 ? sg.gva : (sg.gva & ~4095ull) + p * 4096;
        const uint64_t pe = (va & ~4095ull) + 4096 < end ? (va & ~4095ull) + 4096 : end;
        const WalkOut w = walk(G, nullptr, va, to_guest);
        if (w.code != kOk) continue;   // tables changed under the call: unspecified, skip
        uint8_t* gp = G.pool + w.hpa;
        uint8_t* sp = a.stg + sbase + (va - sg.gva);
        if (to_guest) warp_copy<16, 2>(gp, sp, pe - va, lane);
        else warp_copy<16, 2>(sp, gp, pe - va, lane);
      }
      if (!to_guest && sg.ncopy < sg.len) {   // zero-filled tail, in 4 KiB pieces over the warps
        const uint64_t z = sg.len - sg.ncopy, nz = (z + 4095) / 4096;
        for (uint64_t q = 0; q < nz; q++, k++)
          if ((k % kOrderedWarps) == (uint32_t)wid)
            warp_zero<16>(a.stg + sbase + sg.ncopy + q * 4096, z - q * 4096 < 4096 ? z - q * 4096 : 4096, lane);
      }
      if (to_guest) __syncthreads();
    }
    __syncthreads();
  }
}

cudaError_t launch_ordered_copy(const BatchArgs& a, const uint8_t* mark, const unsigned int* nmarked, cudaStream_t st) {
  k_ordered_copy<<<1, kOrderedWarps * 32, 0, st>>>(a, mark, nmarked);
  g_launches++;
  return cudaGetLastError();
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

template <int PM>
__device__ __noinline__ WalkOut walk_ni(const DevGuest& G, const TopCache* tc, uint64_t va, bool write) {
  return walk_t<PM>(G, tc, va, write);
}

// Queue part [a0, a1) of a segment (warp cooperative): lanes translate up to
// 32 pages at once; each host-contiguous piece becomes a run.
template <int PM>
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
    if (active) w = walk_ni<PM>(G, tc, va, to_guest);
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

template <int PM>
__device__ __noinline__ void copy_small_ni(const DevGuest& G, const TopCache* tc, const SegWork& s, uint64_t stg_base,
                                           uint8_t* stg, bool to_guest) {
  copy_small<PM>(G, tc, s, stg_base, stg, to_guest);
}

// Segments whose copy part spans at most this many 4 KiB pages are translated
// together: one parallel walk round covers the pages of every short segment
// of a 32-segment group, instead of one serial round per segment.
constexpr uint32_t kShortPages = 8;

// Queue copy parts [gva+pa, gva+c1) of the lanes with mine = true, batched:
// the pages of all of them are enumerated across the warp (item i -> owner
// lane by a shuffle binary search over the inclusive page-count scan), walked
// in parallel, then queued in order.
template <int PM>
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
    if (active) w = walk_ni<PM>(G, tc, va, to_guest);
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

// MAXT: the largest block the instantiation is launched with.  Blocks of up
// to 16 warps (the default) compile for 512 threads, which leaves 128
// registers per thread (64 at 1024): the chunk/segment loop no longer spills
// to local memory.  On the batching workload k_copy went from 0.85 of the
// measured copy peak (20 warps, 64 registers) to 0.88 (20 warps, 96) and
// 0.91 (16 warps, 128); 12 warps with 168 registers fell to 0.80.
constexpr int kCopyNarrow = 512;

// ept_stage (EPT launches): the EPT's top levels are staged after the top
// cache when the host found room for them.
template <bool STAGE, int PM, int MAXT>
__global__ void __launch_bounds__(MAXT) k_copy_tma(BatchArgs a, uint64_t chunk, uint64_t small, uint32_t K,
                                                   uint32_t stage, uint32_t ring, uint32_t ept_stage) {
  extern __shared__ __align__(16) unsigned char smem[];
  TopCache* tc = nullptr;
  unsigned char* base = smem;
  if (STAGE) {
    tc = reinterpret_cast<TopCache*>(smem);
    stage_top<SdOf<PM>::v>(tc, *a.single);
    base += round128((uint32_t)sizeof(TopCache));
    if (PM == kPmEpt && ept_stage) {
      stage_ept(tc, *a.single, reinterpret_cast<EptTop*>(base));
      base += kEptTopBytes;
    }
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
            copy_small_ni<PM>(G, t, s, rw.host_off + s.soff, a.stg, to_guest);
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
            copy_group_short<PM>(wp, G, t, s.gva, s.soff, shortseg, pa, c1, rw.host_off, a.stg, to_guest, lane);
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
            copy_piece_q<PM>(wp, G, t, ls, rw.host_off + ls.soff, a.stg, to_guest, lpa, lc1, lane);
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

template <bool STAGE, int PM>
static void launch_tma_t(const BatchArgs& a, const CopyParams& p, unsigned blocks, unsigned threads, size_t sm,
                         cudaStream_t st) {
  // an EPT launch stages the EPT's top levels when they fit beside the rings
  const uint32_t ept = (PM == kPmEpt && STAGE && sm + kEptTopBytes <= 227 * 1024) ? 1u : 0u;
  if (ept) sm += kEptTopBytes;
  if (threads <= (unsigned)kCopyNarrow)
    k_copy_tma<STAGE, PM, kCopyNarrow><<<blocks, threads, sm, st>>>(a, p.chunk_bytes, p.small_bytes, p.stages,
                                                                    p.stage_bytes, p.ring_bytes, ept);
  else
    k_copy_tma<STAGE, PM, 1024><<<blocks, threads, sm, st>>>(a, p.chunk_bytes, p.small_bytes, p.stages,
                                                             p.stage_bytes, p.ring_bytes, ept);
}

static cudaError_t launch_copy_tma(const BatchArgs& a, const CopyParams& p, cudaStream_t st) {
  unsigned threads = p.warps_per_block * 32;
  const int sms = num_sms() - (int)a.spare_sms;
  unsigned blocks = (unsigned)(sms > 0 ? sms : 1) * p.blocks_per_sm;
  size_t sm = copy_smem_bytes(p, a.nguests == 1);
  // a single-guest launch compiles its walks for the guest's paging format
  if (a.nguests != 1 && a.single_paging == kWalkEpt) launch_tma_t<false, kPmEpt>(a, p, blocks, threads, sm, st);
  else if (a.nguests != 1) launch_tma_t<false, kPmAny>(a, p, blocks, threads, sm, st);
  else if (a.single_paging == kPagingPae) launch_tma_t<true, kPmPae>(a, p, blocks, threads, sm, st);
  else if (a.single_paging == kWalkEpt) launch_tma_t<true, kPmEpt>(a, p, blocks, threads, sm, st);
  else launch_tma_t<true, kPmX86>(a, p, blocks, threads, sm, st);
  g_launches++;
  return cudaGetLastError();
}

// Shared-memory attributes of the copy kernels, set before any stream capture.
void prepare_copy_kernels() {
  size_t sm = sizeof(TopCache);
  allow_smem(k_copy<16, 1, true>, sm);
  allow_smem(k_copy<16, 2, true>, sm);
  allow_smem(k_copy<16, 4, true>, sm);
  allow_smem(k_copy<8, 4, true>, sm);
  allow_smem(k_copy<8, 2, true>, sm);
  allow_smem(k_copy<4, 4, true>, sm);
  allow_smem(k_copy_tma<true, kPmX86, kCopyNarrow>, 227 * 1024);
  allow_smem(k_copy_tma<true, kPmPae, kCopyNarrow>, 227 * 1024);
  allow_smem(k_copy_tma<true, kPmEpt, kCopyNarrow>, 227 * 1024);
  allow_smem(k_copy_tma<false, kPmEpt, kCopyNarrow>, 227 * 1024);
  allow_smem(k_copy_tma<false, kPmAny, kCopyNarrow>, 227 * 1024);
  allow_smem(k_copy_tma<true, kPmX86, 1024>, 227 * 1024);
  allow_smem(k_copy_tma<true, kPmPae, 1024>, 227 * 1024);
  allow_smem(k_copy_tma<true, kPmEpt, 1024>, 227 * 1024);
  allow_smem(k_copy_tma<false, kPmEpt, 1024>, 227 * 1024);
  allow_smem(k_copy_tma<false, kPmAny, 1024>, 227 * 1024);
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

cudaError_t launch_copy(const BatchArgs& a, const CopyParams& p, cudaStream_t st, bool counter_zeroed) {
  if (!counter_zeroed) {
    const cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
  }
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

}  // namespace cvd
