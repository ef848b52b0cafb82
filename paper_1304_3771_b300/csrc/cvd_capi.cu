// cvd_capi.cu -- extern "C" boundary of libcvd.so (declared in include/cvd.h)
// plus the host runtime behind it: guest handles, per-stream scratch, the
// hazard leveller for sequential semantics, the CUDA-graph cache and the
// copy-engine autotuner.
//
// Paper: the calls stand for the kernel memory routines that a host driver
// calls while servicing a forwarded file operation and that the CVD backend
// redirects to the guest process's memory (Sec. 4.2, Sec. 6.2); the guest
// handle keeps the page-table root captured when the guest process first
// called (Sec. 6.3).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <memory>
#include <mutex>
#include <tuple>
#include <new>
#include <vector>

#include "../../include/cvd.h"
#include "cvd_internal.h"

using namespace cvd;

int cvd::check_batch_args(cvd_guest* const* guests, uint32_t nguests, const void* req, uint32_t nreq,
                          const void* seg, uint64_t nseg, const void* stg, uint64_t stg_bytes, const void* res) {
  if (nguests == 0 || nguests > CVD_MAX_GUESTS_PER_BATCH || !guests) return CVD_EINVAL;
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t s0 = (uint64_t)(uintptr_t)stg;
  for (uint32_t i = 0; i < nguests; i++) {
    if (!guests[i] || guests[i]->device != dev) return CVD_EINVAL;
    const DevGuest& h = guests[i]->host;
    const uint64_t p0 = (uint64_t)(uintptr_t)h.pool;
    if (stg && stg_bytes && p0 < s0 + stg_bytes && s0 < p0 + h.pool_bytes) return CVD_EINVAL;
  }
  // Guests whose pools overlap must start a multiple of 4 KiB apart (the same
  // guest twice, say): the levelled calls' conflict check keys a guest page by
  // the device frame it starts in, which other aliasing would not match.
  for (uint32_t i = 0; i < nguests; i++)
    for (uint32_t j = i + 1; j < nguests; j++) {
      const DevGuest& a = guests[i]->host;
      const DevGuest& b = guests[j]->host;
      const uint64_t a0 = (uint64_t)(uintptr_t)a.pool, b0 = (uint64_t)(uintptr_t)b.pool;
      if (a0 < b0 + b.pool_bytes && b0 < a0 + a.pool_bytes && ((a0 - b0) & 4095)) return CVD_EINVAL;
    }
  if (nreq && (!req || !res)) return CVD_EINVAL;
  if (nseg && !seg) return CVD_EINVAL;
  if (stg_bytes && !stg) return CVD_EINVAL;
  // stream positions are sums of staging-bounded lengths: keep them in u64
  if (nreq && stg_bytes + kReqWeight > (1ull << 62) / nreq) return CVD_EINVAL;
  if (stg_bytes >= (1ull << 52)) return CVD_EINVAL;   // fault keys hold request offsets in 52 bits
  return CVD_OK;
}

namespace {

thread_local int t_last_cuda = 0;

int cuda_fail(cudaError_t e) {
  t_last_cuda = (int)e;
  cudaGetLastError();   // do not leave a non-sticky error for the next launch check
  return CVD_ECUDA;
}
#define CK(x)                                    \
  do {                                           \
    cudaError_t _e = (x);                        \
    if (_e != cudaSuccess) return cuda_fail(_e); \
  } while (0)

// Device buffer that only grows.  Growing frees the old buffer (cudaFree
// waits for the device), so a call that grows scratch synchronises.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  bool grow(size_t bytes, bool* moved) {
    if (bytes <= cap) return true;
    size_t nb = std::max(bytes + bytes / 4, (size_t)4096);
    void* q = nullptr;
    if (cudaMalloc(&q, nb) != cudaSuccess) { cudaGetLastError(); return false; }
    if (p) cudaFree(p);
    p = q;
    cap = nb;
    if (moved) *moved = true;
    return true;
  }
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

// Pinned host buffer that only grows.
struct PinBuf {
  void* p = nullptr;
  size_t cap = 0;
  bool grow(size_t bytes) {
    if (bytes <= cap) return true;
    size_t nb = std::max(bytes + bytes / 4, (size_t)4096);
    void* q = nullptr;
    if (cudaHostAlloc(&q, nb, cudaHostAllocDefault) != cudaSuccess) { cudaGetLastError(); return false; }
    if (p) cudaFreeHost(p);
    p = q;
    cap = nb;
    return true;
  }
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

using GraphKey = std::tuple<std::vector<uint64_t>, uint64_t, uint64_t, uint64_t, uint64_t, uint64_t, uint64_t,
                            uint64_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, int>;

// ---- host leveller -------------------------------------------------------
// Byte-exact levels of a run list: level(run) = 1 + the highest level of an
// earlier run that touches a common byte with one of the two writing it (0
// if none).  Runs are in stream order of the call (requests in index order,
// bytes in order), so executing levels in order reproduces sequential
// semantics.  Every run's byte ranges (destination: written, source: read)
// are sorted by address and swept into clusters of overlapping ranges; only
// a cluster holding two or more ranges, one of them written, can order
// anything, and a run with no range in such a cluster stays at level 0.
// Within those clusters the distinct range ends cut the bytes into
// elementary intervals, each holding the highest writer and reader level
// seen so far, and the runs are levelled in stream order over them.
struct RangeRec { uint64_t a, b; uint32_t run, write; };

// Host scratch of the leveller, kept across calls so that repeated calls do
// not fault fresh pages in.
struct LevelScratch {
  std::vector<RangeRec> iv, tmp;
  std::vector<uint32_t> cnt, rec_of, cl_of, span_lo, span_hi;
  std::vector<uint64_t> cl_lo, cl_end, pts, pt_lo;
  std::vector<char> mark;
  std::vector<int> W, R;
};

// Stable LSD radix sort of the records by start address, 11-bit digits over
// the bits in which the starts differ.
void sort_by_start(LevelScratch& S) {
  std::vector<RangeRec>& v = S.iv;
  const size_t n = v.size();
  if (n < 2) return;
  uint64_t lo = ~0ull, hi = 0;
  for (const RangeRec& r : v) { lo = std::min(lo, r.a); hi = std::max(hi, r.a); }
  const uint64_t span = hi - lo;
  int bits = 0;
  while (bits < 64 && (span >> bits)) bits++;
  S.tmp.resize(n);
  RangeRec* src = v.data();
  RangeRec* dst = S.tmp.data();
  S.cnt.resize(2048);
  uint32_t* cnt = S.cnt.data();
  for (int shift = 0; shift < bits; shift += 11) {
    std::fill(cnt, cnt + 2048, 0u);
    for (size_t i = 0; i < n; i++) cnt[((src[i].a - lo) >> shift) & 2047]++;
    uint32_t sum = 0;
    for (uint32_t d = 0; d < 2048; d++) { const uint32_t c = cnt[d]; cnt[d] = sum; sum += c; }
    for (size_t i = 0; i < n; i++) dst[cnt[((src[i].a - lo) >> shift) & 2047]++] = src[i];
    std::swap(src, dst);
  }
  if (src != v.data()) std::copy(src, src + n, v.data());
}

// Levels of the runs in stream order: level(run) = 1 + the highest level of
// an earlier run touching a common byte with one of the two writing it (0
// when none); *marked gets the number of runs that can conflict at all.
// lev[i] gets run i's level; returns the highest level.
int level_runs(LevelScratch& S, const Run* runs, uint64_t n, int* lev, uint64_t* marked_out) {
  std::vector<RangeRec>& iv = S.iv;
  iv.clear();
  for (uint64_t i = 0; i < n; i++) {
    lev[i] = 0;
    if (!runs[i].len) continue;
    iv.push_back({runs[i].dst, runs[i].dst + runs[i].len, (uint32_t)i, 1u});
    if (runs[i].src) iv.push_back({runs[i].src, runs[i].src + runs[i].len, (uint32_t)i, 0u});
  }
  sort_by_start(S);
  // clusters of overlapping ranges; the conflicting ones hold >= 2 ranges and a writer
  S.rec_of.assign(2 * n, ~0u);
  S.mark.assign(n, 0);
  S.cl_lo.clear();
  S.cl_end.clear();
  uint64_t marked = 0;
  size_t c0 = 0;
  while (c0 < iv.size()) {
    size_t c1 = c0 + 1;
    uint64_t end = iv[c0].b;
    uint32_t w = iv[c0].write;
    while (c1 < iv.size() && iv[c1].a < end) {
      end = std::max(end, iv[c1].b);
      w |= iv[c1].write;
      c1++;
    }
    if (c1 - c0 >= 2 && w) {
      S.cl_lo.push_back(c0);
      S.cl_end.push_back(c1);
      for (size_t k = c0; k < c1; k++) {
        S.rec_of[2 * (uint64_t)iv[k].run + iv[k].write] = (uint32_t)k;
        if (!S.mark[iv[k].run]) { S.mark[iv[k].run] = 1; marked++; }
      }
    }
    c0 = c1;
  }
  *marked_out = marked;
  if (!marked) return 0;
  // elementary intervals of each conflicting cluster: its distinct endpoints
  const size_t ncl = S.cl_lo.size();
  S.pts.clear();
  S.pt_lo.resize(ncl + 1);
  for (size_t c = 0; c < ncl; c++) {
    S.pt_lo[c] = S.pts.size();
    const size_t s0 = S.pts.size();
    for (size_t k = S.cl_lo[c]; k < S.cl_end[c]; k++) { S.pts.push_back(iv[k].a); S.pts.push_back(iv[k].b); }
    std::sort(S.pts.begin() + s0, S.pts.end());
    S.pts.erase(std::unique(S.pts.begin() + s0, S.pts.end()), S.pts.end());
  }
  S.pt_lo[ncl] = S.pts.size();
  S.span_lo.resize(iv.size());
  S.span_hi.resize(iv.size());
  for (size_t c = 0; c < ncl; c++) {
    const uint64_t* p0 = S.pts.data() + S.pt_lo[c];
    const uint64_t* p1 = S.pts.data() + S.pt_lo[c + 1];
    for (size_t k = S.cl_lo[c]; k < S.cl_end[c]; k++) {
      S.span_lo[k] = (uint32_t)(std::lower_bound(p0, p1, iv[k].a) - S.pts.data());
      S.span_hi[k] = (uint32_t)(std::lower_bound(p0, p1, iv[k].b) - S.pts.data());
    }
  }
  // the highest writer / reader level on each elementary interval, in stream order
  S.W.assign(S.pts.size(), -1);
  S.R.assign(S.pts.size(), -1);
  int* W = S.W.data();
  int* R = S.R.data();
  int maxl = 0;
  for (uint64_t i = 0; i < n; i++) {
    if (!S.mark[i]) continue;
    const uint32_t kd = S.rec_of[2 * i + 1], ks = S.rec_of[2 * i];
    int L = 0;
    if (kd != ~0u)
      for (uint32_t e = S.span_lo[kd]; e < S.span_hi[kd]; e++) L = std::max(L, std::max(W[e], R[e]) + 1);
    if (ks != ~0u)
      for (uint32_t e = S.span_lo[ks]; e < S.span_hi[ks]; e++) L = std::max(L, W[e] + 1);
    if (kd != ~0u)
      for (uint32_t e = S.span_lo[kd]; e < S.span_hi[kd]; e++) W[e] = std::max(W[e], L);
    if (ks != ~0u)
      for (uint32_t e = S.span_lo[ks]; e < S.span_hi[ks]; e++) R[e] = std::max(R[e], L);
    lev[i] = L;
    maxl = std::max(maxl, L);
  }
  return maxl;
}

struct Workspace {
  std::mutex mu;
  DevBuf pairs_in, pairs_out, scan_tmp, rw, sw, counter, guests, err, fkey, lcount, long_items;
  DevBuf run_counts, run_offs, runs, runs_sorted;   // run lists (checked calls, marked requests)
  PinBuf h_runs, h_sorted;             // their pinned host copies
  LevelScratch lvs;                    // the host leveller's scratch
  std::vector<int> lev;                // levels of the runs
  // levelled calls: frame table (keys, vals) of hz_cap slots, tagged with a
  // per-call epoch so it is never cleared; [flag, marked count]; request marks
  DevBuf hz_keys, hz_vals, marks;
  PinBuf hz_host;
  uint64_t hz_cap = 0, hz_epoch = 0;
  bool levels_on_device = false;       // the last levelled call's marked count is in the counter block
  // host-buffer batches: two device slots (a batch's inputs go into one
  // while the previous batch's outputs leave the other), private copy streams
  struct HostSlot { DevBuf req, seg, stg, res; cudaEvent_t in = nullptr, res_done = nullptr, free = nullptr; };
  HostSlot hs[2];
  cudaStream_t up = nullptr, down = nullptr, res = nullptr;   // inputs, write-backs, results
  std::vector<uint64_t> guest_list;    // DevGuest* currently in `guests`
  uint32_t last_levels = 0;
  cudaStream_t cap = nullptr;          // private stream graphs are captured on
  // levelled calls: a second stream on which the conflict insert pass runs
  // beside the planner, and the ordered pass beside the parallel copy
  // (fork and join events, created with the stream)
  cudaStream_t aux = nullptr;
  cudaEvent_t fork_ev[2] = {nullptr, nullptr}, join_ev[2] = {nullptr, nullptr};
  std::map<GraphKey, cudaGraphExec_t> graphs;
  void drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
  }
};

// Library state is kept per (device, stream): the legacy default stream is
// the same handle on every device, and scratch, cached graphs and guest
// arrays belong to one device.
using StreamKey = std::pair<int, cudaStream_t>;
StreamKey stream_key(cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  return {dev, st};
}

std::mutex g_mu;
std::map<StreamKey, std::unique_ptr<Workspace>> g_ws;

// Copy-engine parameters per device (cvd_set_copy_params / cvd_tune set the
// current device's; defaults elsewhere).
std::mutex g_params_mu;
std::map<int, CopyParams> g_params;
CopyParams current_params() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_params_mu);
  auto it = g_params.find(dev);
  return it == g_params.end() ? CopyParams() : it->second;
}
void set_current_params(const CopyParams& p) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_params_mu);
  g_params[dev] = p;
}

// kernel timing (cvd_profile_*): kind 0 a batch call (a..b planner, b..c
// copy), otherwise a single launch (a..b) of that ProfKind
struct ProfRec { cudaEvent_t a, b, c; int kind = 0; };
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;

Workspace& workspace(cudaStream_t st) {
  const StreamKey key = stream_key(st);
  std::lock_guard<std::mutex> lk(g_mu);
  auto& p = g_ws[key];
  if (!p) p.reset(new Workspace());
  return *p;
}

bool overlaps(uint64_t a0, uint64_t a1, uint64_t b0, uint64_t b1) { return a0 < b1 && b0 < a1; }

struct Call {
  cvd_guest* const* guests;
  uint32_t nguests;
  const cvd_req* req;
  uint32_t nreq;
  const cvd_seg* seg;
  uint64_t nseg;
  void* stg;
  uint64_t stg_bytes;
  cvd_result* res;
  uint32_t flags;
  int dir_override;
};

int validate(const Call& c) {
  return check_batch_args(c.guests, c.nguests, c.req, c.nreq, c.seg, c.nseg, c.stg, c.stg_bytes, c.res);
}

// The guest pointers of a batch, passed by value: a launch captures its
// parameters, so the upload is stream-ordered with no host buffer to keep
// alive and no synchronisation.
struct GuestList { const DevGuest* g[CVD_MAX_GUESTS_PER_BATCH]; uint32_t n; };

__global__ void k_store_guests(const DevGuest** dst, GuestList gl) {
  if (threadIdx.x < gl.n) dst[threadIdx.x] = gl.g[threadIdx.x];
}

// Long-segment list entries for a batch over a staging buffer of the given
// size: long segments (> 1 MiB) of requests with disjoint staging ranges need
// at most two entries per 1 MiB of staging; a batch that needs more walks the
// rest inline.
size_t long_cap(uint64_t stg_bytes) {
  return (size_t)std::min<uint64_t>(1u << 22, 2 * (stg_bytes / ((uint64_t)kLongBlock * 4096)) + 4096);
}

// Size scratch and fill BatchArgs.  *moved reports a scratch reallocation.
int prepare(Workspace& ws, const Call& c, BatchArgs* a, bool* moved, cudaStream_t st) {
  bool mv = false;
  size_t np = 2 * ((size_t)c.nreq + 1);
  if (!ws.pairs_in.grow(np * 8, &mv) || !ws.pairs_out.grow(np * 8, &mv) ||
      !ws.scan_tmp.grow(2 * scan_tmp_elems(c.nreq) * 8, &mv) ||
      !ws.rw.grow(std::max<size_t>(c.nreq, 1) * sizeof(ReqWork), &mv) ||
      !ws.fkey.grow(std::max<size_t>(c.nreq, 1) * 8, &mv) || !ws.lcount.grow(std::max<size_t>(c.nreq, 1) * 4, &mv) ||
      !ws.long_items.grow(long_cap(c.stg_bytes) * sizeof(LongItem), &mv) ||
      !ws.sw.grow(std::max<size_t>(c.nseg, 1) * sizeof(SegWork), &mv) || !ws.counter.grow(256, &mv) ||
      !ws.guests.grow(CVD_MAX_GUESTS_PER_BATCH * sizeof(void*), &mv))
    return CVD_ENOMEM;
  if (!ws.err.p) {
    if (!ws.err.grow(256, &mv)) return CVD_ENOMEM;
    CK(cudaMemsetAsync(ws.err.p, 0, 256, st));
  }
  std::vector<uint64_t> gl(c.nguests);
  for (uint32_t i = 0; i < c.nguests; i++) gl[i] = (uint64_t)(uintptr_t)c.guests[i]->dev;
  if (mv || gl != ws.guest_list) {
    GuestList p;
    p.n = c.nguests;
    for (uint32_t i = 0; i < c.nguests; i++) p.g[i] = c.guests[i]->dev;
    k_store_guests<<<1, CVD_MAX_GUESTS_PER_BATCH, 0, st>>>(ws.guests.as<const DevGuest*>(), p);
    g_launches++;
    CK(cudaGetLastError());
    ws.guest_list = gl;
    mv = true;   // cached graphs read the guest array: drop them
  }
  if (mv) ws.drop_graphs();
  *moved = mv;
  a->req = reinterpret_cast<const Req*>(c.req);
  a->nreq = c.nreq;
  a->seg = reinterpret_cast<const Seg*>(c.seg);
  a->nseg = c.nseg;
  a->guests = ws.guests.as<const DevGuest*>();
  a->nguests = c.nguests;
  a->single = c.nguests == 1 ? c.guests[0]->dev : nullptr;
  a->single_paging = 0;
  for (uint32_t i = 0; i < c.nguests; i++)
    if (c.guests[i]->host.ept) a->single_paging = kWalkEpt;
  if (c.nguests == 1) a->single_paging = walk_selector(c.guests[0]->host);
  a->dir_override = c.dir_override;
  a->stg = reinterpret_cast<uint8_t*>(c.stg);
  a->stg_bytes = c.stg_bytes;
  a->res = reinterpret_cast<Result*>(c.res);
  a->pairs_in = ws.pairs_in.as<uint64_t>();
  a->pairs_out = ws.pairs_out.as<uint64_t>();
  a->scan_tmp = ws.scan_tmp.as<uint64_t>();
  a->rw = ws.rw.as<ReqWork>();
  a->sw = ws.sw.as<SegWork>();
  a->counter = ws.counter.as<unsigned long long>();
  a->fkey = ws.fkey.as<unsigned long long>();
  a->lcount = ws.lcount.as<unsigned int>();
  a->long_items = ws.long_items.as<LongItem>();
  a->long_cap = long_cap(c.stg_bytes);
  a->err = ws.err.as<unsigned int>();
  a->spare_sms = 0;
  return CVD_OK;
}

// Internal flag (never accepted from callers): the caller guarantees that the
// requests' staging ranges are pairwise disjoint (the serving loop, whose
// staging allocator hands out disjoint ranges).
constexpr uint32_t kBatchStagingDisjoint = 1u << 16;
// Internal flag: the caller checked that no segment spans over kLongPages
// pages, so the long-segment pass has nothing to walk and is not launched.
constexpr uint32_t kBatchNoLong = 1u << 17;

// Frame-table sizes of the levelled calls' conflict check (slots; 16 bytes
// each).
constexpr uint64_t kHzMinCap = 1ull << 16, kHzMaxCap = 1ull << 24;

// Marked requests a public levelled call runs in the device's ordered pass;
// with more, their byte-exact levels are computed on the host.  The ordered
// pass costs ~10 us per request (one block walks and copies them one after
// another); the host path ~0.3-0.6 ms in all (two more synchronisations and
// the leveller), so it wins from a few dozen requests on (measured on B300:
// 150 marked requests 1.6 ms on the device, 0.36 ms through the host).
constexpr uint32_t kOrderedMaxMarked = 32;

// Levels of the marked requests' runs on the host: list their runs on the
// device (count, scan, emit: two synchronisations), mark the runs that
// overlap another with a writer (sort-and-sweep), level those with the
// byte-exact leveller, and copy level by level.  The unmarked requests are
// already copied (they conflict with none of these).
int level_marked_on_host(Workspace& ws, const BatchArgs& a, cudaStream_t st) {
  const uint8_t* only = ws.marks.as<uint8_t>();
  bool mv = false;
  size_t np = 2 * ((size_t)a.nreq + 1);
  if (!ws.run_counts.grow(np * 8, &mv) || !ws.run_offs.grow(np * 8, &mv) || !ws.h_runs.grow(64)) return CVD_ENOMEM;
  if (mv) ws.drop_graphs();
  CK(launch_runs(a, false, ws.run_counts.as<uint64_t>(), nullptr, nullptr, st, only));
  CK(launch_scan_pairs(ws.run_counts.as<uint64_t>(), ws.run_offs.as<uint64_t>(), a.nreq, a.scan_tmp, st));
  uint64_t* tot = ws.h_runs.as<uint64_t>();
  CK(cudaMemcpyAsync(tot, ws.run_offs.as<uint64_t>() + 2 * (uint64_t)a.nreq, 16, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const uint64_t nruns = tot[0];
  if (nruns == 0) return CVD_OK;
  if (!ws.runs.grow(nruns * sizeof(Run), &mv) || !ws.runs_sorted.grow(nruns * sizeof(Run), &mv) ||
      !ws.h_runs.grow(nruns * sizeof(Run)) || !ws.h_sorted.grow(nruns * sizeof(Run)))
    return CVD_ENOMEM;
  if (mv) ws.drop_graphs();
  CK(launch_runs(a, true, nullptr, ws.run_offs.as<uint64_t>(), ws.runs.as<Run>(), st, only));
  Run* runs = ws.h_runs.as<Run>();
  CK(cudaMemcpyAsync(runs, ws.runs.p, nruns * sizeof(Run), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<int>& lev = ws.lev;
  lev.resize(nruns);
  uint64_t nmarked = 0;
  const int maxl = level_runs(ws.lvs, runs, nruns, lev.data(), &nmarked);
  std::vector<uint64_t> cnt(maxl + 2, 0);
  for (uint64_t i = 0; i < nruns; i++) cnt[lev[i] + 1]++;
  for (int l = 1; l <= maxl + 1; l++) cnt[l] += cnt[l - 1];
  Run* sorted = ws.h_sorted.as<Run>();
  std::vector<uint64_t> pos(cnt.begin(), cnt.end() - 1);
  for (uint64_t i = 0; i < nruns; i++) sorted[pos[lev[i]]++] = runs[i];
  // pinned source: the copy completes before the next call touches the
  // buffer (that call synchronises the stream before it writes it)
  CK(cudaMemcpyAsync(ws.runs_sorted.p, sorted, nruns * sizeof(Run), cudaMemcpyHostToDevice, st));
  for (int l = 0; l <= maxl; l++)
    CK(launch_run_copy(ws.runs_sorted.as<Run>() + cnt[l], cnt[l + 1] - cnt[l], st));
  ws.last_levels = (uint32_t)(maxl + 2);   // the parallel launch, then the levels of the marked runs
  return CVD_OK;
}

// A levelled call's conflict flag and marked-request count: two u32 in word 3
// of the workspace's counter block, which the plan's sizing kernel zeroes.
unsigned int* hz_flag_of(Workspace& ws) { return reinterpret_cast<unsigned int*>(ws.counter.as<unsigned long long>() + 3); }

// Run on ws.aux, after everything enqueued so far on st, what `body`
// enqueues; `join` makes st wait for it (before whatever st gets next).
template <class F>
cudaError_t fork_aux(Workspace& ws, int k, cudaStream_t st, F body) {
  if (!ws.aux) {   // the stream is set only once its events exist
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; i++) {
      if (!ws.fork_ev[i]) e = cudaEventCreateWithFlags(&ws.fork_ev[i], cudaEventDisableTiming);
      if (e == cudaSuccess && !ws.join_ev[i]) e = cudaEventCreateWithFlags(&ws.join_ev[i], cudaEventDisableTiming);
    }
    cudaStream_t aux = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    ws.aux = aux;
  }
  cudaError_t e = cudaEventRecord(ws.fork_ev[k], st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ws.aux, ws.fork_ev[k], 0);
  if (e == cudaSuccess) e = body(ws.aux);
  if (e == cudaSuccess) e = cudaEventRecord(ws.join_ev[k], ws.aux);
  return e;
}
cudaError_t join_aux(Workspace& ws, int k, cudaStream_t st) { return cudaStreamWaitEvent(st, ws.join_ev[k], 0); }

// A levelled call after its plan's sizing: the conflict insert pass on a
// second stream beside the planner's walk, then the conflict marks and the
// unmarked requests in one parallel copy launch, all on the device.  Then the
// marked requests: with `decide` (public calls), one synchronisation reads
// how many there are -- none: done; up to kOrderedMaxMarked: the device's
// ordered pass; more: levelled on the host.  Without it (the serving loop,
// where conflicts are rare), the ordered pass is enqueued with no host round
// trip, on the second stream beside the parallel copy (the two touch no
// common guest page and, the staging ranges being disjoint, no common
// staging byte).  The frame table holds twice the pages the call can touch
// (its guest bytes are at most the staging bytes when the staging ranges are
// disjoint, plus a partial page at both ends of every segment); a call that
// overflows it anyway marks every request.
int level_on_device(Workspace& ws, const BatchArgs& a, bool staging_disjoint, bool decide, const CopyParams& p,
                    cudaStream_t st) {
  bool mv = false;
  const uint64_t frames = a.stg_bytes / 4096 + 2 * a.nseg + 64;
  uint64_t cap = kHzMinCap;
  while (cap < 2 * frames && cap < kHzMaxCap) cap <<= 1;
  if (cap > ws.hz_cap) {
    if (!ws.hz_keys.grow(cap * 8, &mv) || !ws.hz_vals.grow(cap * 8, &mv)) return CVD_ENOMEM;
    CK(cudaMemsetAsync(ws.hz_keys.p, 0, cap * 8, st));
    CK(cudaMemsetAsync(ws.hz_vals.p, 0, cap * 8, st));
    ws.hz_cap = cap;
    ws.hz_epoch = 0;
  }
  if (++ws.hz_epoch >= (1ull << 24)) {   // epochs wrap: start over from an empty table
    CK(cudaMemsetAsync(ws.hz_keys.p, 0, ws.hz_cap * 8, st));
    CK(cudaMemsetAsync(ws.hz_vals.p, 0, ws.hz_cap * 8, st));
    ws.hz_epoch = 1;
  }
  if (!ws.marks.grow((size_t)a.nreq + 256, &mv) || !ws.hz_host.grow(64)) return CVD_ENOMEM;
  unsigned int* flag = hz_flag_of(ws);   // [0] flag, [1] marked requests: zeroed by the plan's sizing kernel
  unsigned long long* keys = ws.hz_keys.as<unsigned long long>();
  unsigned long long* vals = ws.hz_vals.as<unsigned long long>();
  const uint64_t hcap = ws.hz_cap, epoch = ws.hz_epoch;
  CK(fork_aux(ws, 0, st, [&](cudaStream_t s2) {
    return launch_hz_insert(a, keys, vals, hcap, epoch, staging_disjoint, flag, s2);
  }));
  CK(launch_plan_walk(a, st));
  CK(join_aux(ws, 0, st));
  CK(launch_hz_mark(a, keys, vals, hcap, epoch, flag, ws.marks.as<uint8_t>(), flag + 1, st));
  if (!decide) {
    uint8_t* marks = ws.marks.as<uint8_t>();
    CK(fork_aux(ws, 1, st, [&](cudaStream_t s2) { return launch_ordered_copy(a, marks, flag + 1, s2); }));
    CK(launch_copy(a, p, st, true));
    CK(join_aux(ws, 1, st));
    ws.levels_on_device = true;
    return CVD_OK;
  }
  CK(launch_copy(a, p, st, true));
  unsigned int* h = ws.hz_host.as<unsigned int>();
  CK(cudaMemcpyAsync(h, flag + 1, 4, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const unsigned int marked = *h;
  ws.levels_on_device = false;
  ws.last_levels = marked ? 2 : 1;
  if (marked == 0) return CVD_OK;
  if (marked <= kOrderedMaxMarked) {
    CK(launch_ordered_copy(a, ws.marks.as<uint8_t>(), flag + 1, st));
    return CVD_OK;
  }
  return level_marked_on_host(ws, a, st);
}

// CVD_BATCH_CHECK: plan, build the run list (one synchronisation for its
// length, one for its bytes), mark the runs that overlap another run with a
// writer by a sort-and-sweep of their ranges, and level the marked ones with
// the byte-exact leveller.  ws.last_levels gets the number of levels.
int plan_and_level(Workspace& ws, const BatchArgs& a, cudaStream_t st) {
  CK(launch_plan(a, st));
  bool mv = false;
  size_t np = 2 * ((size_t)a.nreq + 1);
  if (!ws.run_counts.grow(np * 8, &mv) || !ws.run_offs.grow(np * 8, &mv)) return CVD_ENOMEM;
  if (mv) ws.drop_graphs();
  CK(launch_runs(a, false, ws.run_counts.as<uint64_t>(), nullptr, nullptr, st));
  CK(launch_scan_pairs(ws.run_counts.as<uint64_t>(), ws.run_offs.as<uint64_t>(), a.nreq, a.scan_tmp, st));
  if (!ws.h_runs.grow(64)) return CVD_ENOMEM;
  uint64_t* tot = ws.h_runs.as<uint64_t>();
  CK(cudaMemcpyAsync(tot, ws.run_offs.as<uint64_t>() + 2 * (uint64_t)a.nreq, 16, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const uint64_t nruns = tot[0];
  ws.levels_on_device = false;
  if (nruns == 0) { ws.last_levels = 0; return CVD_OK; }
  if (!ws.runs.grow(nruns * sizeof(Run), &mv) || !ws.h_runs.grow(nruns * sizeof(Run))) return CVD_ENOMEM;
  if (mv) ws.drop_graphs();
  CK(launch_runs(a, true, nullptr, ws.run_offs.as<uint64_t>(), ws.runs.as<Run>(), st));
  Run* runs = ws.h_runs.as<Run>();
  CK(cudaMemcpyAsync(runs, ws.runs.p, nruns * sizeof(Run), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  ws.lev.resize(nruns);
  uint64_t nmarked = 0;
  const int maxl = level_runs(ws.lvs, runs, nruns, ws.lev.data(), &nmarked);
  ws.last_levels = nmarked ? (uint32_t)(maxl + 1) : 1;
  return CVD_OK;
}

int run_batch(const Call& c, cudaStream_t st) {
  int v = validate(c);
  if (v) return v;
  if (c.nreq == 0) return CVD_OK;
  prepare_kernels();
  Workspace& ws = workspace(st);
  std::lock_guard<std::mutex> lk(ws.mu);
  BatchArgs a;
  bool moved = false;
  int rc = prepare(ws, c, &a, &moved, st);
  if (rc) return rc;
  a.no_long = (c.flags & kBatchNoLong) ? 1u : 0u;
  CopyParams p = current_params();
  if (c.flags & CVD_BATCH_HAZARD_FREE) {
    if (c.flags & CVD_BATCH_CHECK) {
      rc = plan_and_level(ws, a, st);
      if (rc) return rc;
      if (ws.last_levels > 1) return CVD_EHAZARD;
    }
    if (c.flags & CVD_BATCH_GRAPH) {
      GraphKey key{ws.guest_list, (uint64_t)(uintptr_t)c.req, c.nreq, (uint64_t)(uintptr_t)c.seg, c.nseg,
                   (uint64_t)(uintptr_t)c.stg, c.stg_bytes, (uint64_t)(uintptr_t)c.res, p.vec_bytes, p.unroll,
                   p.chunk_bytes, p.blocks_per_sm, p.warps_per_block, p.small_bytes,
                   (int)(c.dir_override + 4 * (p.engine + 4 * (p.stages + 64 * p.stage_bytes))) ^
                       (int)(p.ring_bytes << 7)};
      auto it = ws.graphs.find(key);
      if (it == ws.graphs.end()) {
        // Capture on a private stream (the caller's may be the legacy default
        // stream, which cannot be captured); the graph runs on the caller's.
        if (!ws.cap) CK(cudaStreamCreateWithFlags(&ws.cap, cudaStreamNonBlocking));
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(ws.cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = launch_plan(a, ws.cap);
        cudaError_t e2 = e1 == cudaSuccess ? launch_copy(a, p, ws.cap) : e1;
        cudaError_t e3 = cudaStreamEndCapture(ws.cap, &g);
        if (e2 != cudaSuccess) return cuda_fail(e2);
        if (e3 != cudaSuccess) return cuda_fail(e3);
        cudaGraphExec_t ex;
        cudaError_t e4 = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e4 != cudaSuccess) return cuda_fail(e4);
        it = ws.graphs.emplace(key, ex).first;
      } else {
        g_launches += 6;   // replay: k_req_sizes, 3 scan kernels, k_plan, k_copy
      }
      CK(cudaGraphLaunch(it->second, st));
      return CVD_OK;
    }
    ProfRec pr{nullptr, nullptr, nullptr};
    bool prof = false;
    {
      std::lock_guard<std::mutex> pl(g_prof_mu);
      prof = g_prof_on;
    }
    if (prof) {
      CK(cudaEventCreate(&pr.a));
      CK(cudaEventCreate(&pr.b));
      CK(cudaEventCreate(&pr.c));
      CK(cudaEventRecord(pr.a, st));
    }
    CK(launch_plan(a, st));
    if (prof) CK(cudaEventRecord(pr.b, st));
    CK(launch_copy(a, p, st));
    if (prof) {
      CK(cudaEventRecord(pr.c, st));
      std::lock_guard<std::mutex> pl(g_prof_mu);
      g_prof.push_back(pr);
    }
    return CVD_OK;
  }
  // Levelled call: plan, then mark the conflicting requests and copy the
  // others on the device; the serving loop (disjoint staging) also orders
  // the marked ones on the device, other callers decide after one sync.
  CK(launch_plan_sizes(a, st));
  const bool serving = (c.flags & kBatchStagingDisjoint) != 0;
  return level_on_device(ws, a, serving, !serving, p, st);
}

}  // namespace

// Levelled batch whose staging ranges the caller guarantees disjoint (the
// serving loop); otherwise cvd_copy_batch without flags.
int cvd::copy_batch_staging_disjoint(cvd_guest* const* guests, uint32_t nguests, const cvd_req* d_req, uint32_t nreq,
                                     const cvd_seg* d_seg, uint64_t nseg, void* d_host_buf, uint64_t host_buf_bytes,
                                     cvd_result* d_res, bool no_long, cudaStream_t st) {
  Call c{guests, nguests, d_req, nreq, d_seg, nseg, d_host_buf, host_buf_bytes, d_res,
         kBatchStagingDisjoint | (no_long ? kBatchNoLong : 0u), -1};
  return run_batch(c, st);
}

namespace {

cvd_copy_params to_abi(const CopyParams& p) {
  cvd_copy_params q;
  q.vec_bytes = p.vec_bytes; q.unroll = p.unroll; q.chunk_bytes = p.chunk_bytes;
  q.blocks_per_sm = p.blocks_per_sm; q.warps_per_block = p.warps_per_block; q.small_bytes = p.small_bytes;
  q.engine = p.engine; q.stages = p.stages; q.stage_bytes = p.stage_bytes; q.ring_bytes = p.ring_bytes;
  return q;
}

CopyParams from_abi(const cvd_copy_params& q) {
  CopyParams p;
  p.vec_bytes = q.vec_bytes; p.unroll = q.unroll; p.chunk_bytes = q.chunk_bytes;
  p.blocks_per_sm = q.blocks_per_sm; p.warps_per_block = q.warps_per_block; p.small_bytes = q.small_bytes;
  p.engine = q.engine; p.stages = q.stages; p.stage_bytes = q.stage_bytes; p.ring_bytes = q.ring_bytes;
  return p;
}

// ---- planned-ahead device batches (cvd_copy_batches) ---------------------
// Two scratch slots and two library streams per caller stream: batch k is
// planned into slot k & 1 on a low-priority planning stream and copied on a
// high-priority copy stream, so pending copy blocks are dispatched before
// pending planning blocks when both wait for SM resources.  The caller's
// stream orders the call: both library streams wait for its work at entry,
// and it waits for the last copy at exit.
struct Pipe {
  std::mutex mu;
  Workspace w[2];
  cudaStream_t ps = nullptr, cs = nullptr;
  cudaEvent_t start = nullptr, end = nullptr, plan_done[2] = {nullptr, nullptr}, copy_done[2] = {nullptr, nullptr};
};
std::map<StreamKey, std::unique_ptr<Pipe>> g_pipes;

Pipe& pipe_for(cudaStream_t st) {
  const StreamKey key = stream_key(st);
  std::lock_guard<std::mutex> lk(g_mu);
  auto& p = g_pipes[key];
  if (!p) p.reset(new Pipe());
  return *p;
}

int run_batches_dev(cvd_guest* const* guests, uint32_t nguests, const cvd_dev_batch* b, uint32_t nb, void* stg,
                    uint64_t stg_bytes, cudaStream_t st) {
  for (uint32_t k = 0; k < nb; k++) {
    Call c{guests, nguests, b[k].d_req, b[k].nreq, b[k].d_seg, b[k].nseg, stg, stg_bytes, b[k].d_res,
           CVD_BATCH_HAZARD_FREE, -1};
    int v = validate(c);
    if (v) return v;
  }
  prepare_kernels();
  Pipe& P = pipe_for(st);
  std::lock_guard<std::mutex> lk(P.mu);
  if (!P.ps) {
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    CK(cudaStreamCreateWithPriority(&P.ps, cudaStreamNonBlocking, least));
    CK(cudaStreamCreateWithPriority(&P.cs, cudaStreamNonBlocking, greatest));
    CK(cudaEventCreateWithFlags(&P.start, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&P.end, cudaEventDisableTiming));
    for (int i = 0; i < 2; i++) {
      CK(cudaEventCreateWithFlags(&P.plan_done[i], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&P.copy_done[i], cudaEventDisableTiming));
    }
  }
  bool prof = false;
  {
    std::lock_guard<std::mutex> pl(g_prof_mu);
    prof = g_prof_on;
  }
  const CopyParams p = current_params();
  CK(cudaEventRecord(P.start, st));
  CK(cudaStreamWaitEvent(P.ps, P.start, 0));   // inputs made ready on the caller's stream
  CK(cudaStreamWaitEvent(P.cs, P.start, 0));
  for (uint32_t k = 0; k < nb; k++) {
    if (b[k].nreq == 0) continue;
    const int slot = k & 1;
    Workspace& ws = P.w[slot];
    std::lock_guard<std::mutex> wl(ws.mu);
    Call c{guests, nguests, b[k].d_req, b[k].nreq, b[k].d_seg, b[k].nseg, stg, stg_bytes, b[k].d_res,
           CVD_BATCH_HAZARD_FREE, -1};
    CK(cudaStreamWaitEvent(P.ps, P.copy_done[slot], 0));   // the slot's previous copy is done with it
    BatchArgs a;
    bool moved = false;
    int rc = prepare(ws, c, &a, &moved, P.ps);
    if (rc) {   // nothing of this batch launched: the caller's stream still joins the copies in flight
      CK(cudaEventRecord(P.end, P.cs));
      CK(cudaStreamWaitEvent(st, P.end, 0));
      return rc;
    }
    ProfRec pr{nullptr, nullptr, nullptr};
    if (prof) {
      CK(cudaEventCreate(&pr.a));
      CK(cudaEventCreate(&pr.b));
      CK(cudaEventCreate(&pr.c));
      CK(cudaEventRecord(pr.a, P.ps));
    }
    CK(launch_plan(a, P.ps));
    CK(cudaEventRecord(P.plan_done[slot], P.ps));
    CK(cudaStreamWaitEvent(P.cs, P.plan_done[slot], 0));
    // leave SMs to the next batch's planning (none after the last batch)
    bool more = false;
    for (uint32_t k2 = k + 1; k2 < nb && !more; k2++) more = b[k2].nreq > 0;
    a.spare_sms = more ? kPlanAheadSms : 0;
    if (prof) CK(cudaEventRecord(pr.b, P.cs));
    CK(launch_copy(a, p, P.cs));
    if (prof) {
      CK(cudaEventRecord(pr.c, P.cs));
      std::lock_guard<std::mutex> pl(g_prof_mu);
      g_prof.push_back(pr);
    }
    CK(cudaEventRecord(P.copy_done[slot], P.cs));
  }
  CK(cudaEventRecord(P.end, P.cs));
  CK(cudaStreamWaitEvent(st, P.end, 0));
  return CVD_OK;
}

// ---- host-buffer transfers (cvd_copy_batch_host) ---------------------------
// [start, end) byte ranges of the host staging buffer, sorted and merged.
using Ranges = std::vector<std::pair<uint64_t, uint64_t>>;

// Stream length of request i from the host segment array (saturating), or
// false when its descriptors fall outside the array.
bool host_req_len(const cvd_req& q, const cvd_seg* seg, uint64_t nseg, uint64_t* L) {
  if ((uint64_t)q.seg_begin + q.seg_count > nseg) return false;
  uint64_t t = 0;
  for (uint32_t k = 0; k < q.seg_count; k++) {
    uint64_t l = seg[q.seg_begin + k].len;
    t = t + l < t ? ~0ull : t + l;
  }
  *L = t;
  return true;
}

// Sort and merge; ranges closer than `gap` bytes join (the bytes between them
// travel too).
Ranges merge_ranges(Ranges r, uint64_t gap) {
  std::sort(r.begin(), r.end());
  Ranges out;
  for (auto& x : r) {
    if (x.first >= x.second) continue;
    if (!out.empty() && x.first <= out.back().second + gap) out.back().second = std::max(out.back().second, x.second);
    else out.push_back(x);
  }
  return out;
}

// True when [a, b) lies inside one range of the sorted, merged set r.
bool covered(const Ranges& r, uint64_t a, uint64_t b) {
  auto it = std::upper_bound(r.begin(), r.end(), std::pair<uint64_t, uint64_t>(a, ~(uint64_t)0));
  if (it == r.begin()) return false;
  --it;
  return it->first <= a && b <= it->second;
}

bool params_ok(const cvd_copy_params& q) {
  CopyParams p = from_abi(q);
  if (q.chunk_bytes < 4096 || q.chunk_bytes > (1u << 20) || (q.chunk_bytes & (q.chunk_bytes - 1))) return false;
  if (q.blocks_per_sm < 1 || q.blocks_per_sm > 16) return false;
  if (q.small_bytes > 4096) return false;
  if (q.engine == 0) {
    if (q.warps_per_block != 4 && q.warps_per_block != 8) return false;
    CopyParams v = p;
    v.engine = 0;
    return copy_params_supported(v);
  }
  return copy_params_supported(p);
}

// Autotuner search space.  Engine 0 (single-batch tuning only): vector width
// / unroll / chunk / grid.  Engine 1: (warps, pieces in flight, largest piece,
// ring bytes) -- a ring of k x (stage + 16) bytes holds k misaligned pieces
// of the largest size -- by chunk (warps per segment: a segment's bytes are
// split over chunk-sized windows) and, for whole steps, by the largest
// segment copied lane-locally instead of through the bulk-copy ring.
std::vector<CopyParams> tune_candidates(const CopyParams& base, bool step) {
  std::vector<CopyParams> cands;
  static const uint32_t chunks[] = {16u << 10, 64u << 10, 256u << 10};
  if (!step) {
    static const uint32_t vu[][2] = {{16, 1}, {16, 2}, {16, 4}, {8, 4}, {4, 4}};
    for (auto& x : vu)
      for (uint32_t ch : chunks)
        for (uint32_t b : {2u, 4u}) {
          CopyParams p = base;
          p.engine = 0; p.vec_bytes = x[0]; p.unroll = x[1]; p.chunk_bytes = ch; p.blocks_per_sm = b;
          p.warps_per_block = 8;
          cands.push_back(p);
        }
  }
  static const uint32_t ring[][4] = {{32, 4, 4096, 4224},  {32, 8, 2048, 4224},  {28, 8, 2048, 6272},
                                     {24, 6, 4096, 8320},  {20, 8, 4096, 8320},  {16, 8, 4096, 8320},
                                     {16, 16, 4096, 8320}, {16, 12, 2048, 6272}, {16, 8, 4096, 12416},
                                     {12, 8, 8192, 16512}, {6, 8, 16384, 32896}};
  static const uint32_t smalls_step[] = {64u, 256u, 1024u};
  const uint32_t smalls_one[] = {base.small_bytes};
  for (auto& x : ring)
    for (uint32_t ch : chunks) {
      if (step && ch == (16u << 10)) continue;
      for (uint32_t sm : step ? std::vector<uint32_t>(smalls_step, smalls_step + 3)
                              : std::vector<uint32_t>(smalls_one, smalls_one + 1)) {
        CopyParams p = base;
        p.engine = 1; p.warps_per_block = x[0]; p.stages = x[1]; p.stage_bytes = x[2]; p.ring_bytes = x[3];
        p.chunk_bytes = ch; p.blocks_per_sm = 1; p.small_bytes = sm;
        if (copy_params_supported(p)) cands.push_back(p);
      }
    }
  return cands;
}

// Tuning cache: (GPU name, shape) -> best parameters and time, kept for the
// process and, when CVD_TUNE_CACHE names a file, in that file (one entry
// per line, appended).
struct TuneKey {
  std::string gpu;
  uint32_t nguests, sel, nb, lreq, lseg, lstg;
  bool operator<(const TuneKey& o) const {
    return std::tie(gpu, nguests, sel, nb, lreq, lseg, lstg) <
           std::tie(o.gpu, o.nguests, o.sel, o.nb, o.lreq, o.lseg, o.lstg);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<CopyParams, float>> g_tune_cache;
bool g_tune_file_read = false;

uint32_t log2_bucket(uint64_t x) {
  uint32_t b = 0;
  while (x > 1) { x >>= 1; b++; }
  return b;
}

void tune_cache_read_file() {
  if (g_tune_file_read) return;
  g_tune_file_read = true;
  const char* path = getenv("CVD_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char gpu[256];
  TuneKey k;
  CopyParams p;
  float ms;
  while (fscanf(f, " %255[^\t]\t%u %u %u %u %u %u %u %u %u %u %u %u %u %u %u %u %f", gpu, &k.nguests, &k.sel,
                &k.nb, &k.lreq, &k.lseg, &k.lstg, &p.vec_bytes, &p.unroll, &p.chunk_bytes, &p.blocks_per_sm,
                &p.warps_per_block, &p.small_bytes, &p.engine, &p.stages, &p.stage_bytes, &p.ring_bytes, &ms) == 18) {
    k.gpu = gpu;
    if (copy_params_supported(p)) g_tune_cache[k] = {p, ms};
  }
  fclose(f);
}

void tune_cache_append_file(const TuneKey& k, const CopyParams& p, float ms) {
  const char* path = getenv("CVD_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s\t%u %u %u %u %u %u %u %u %u %u %u %u %u %u %u %u %.5f\n", k.gpu.c_str(), k.nguests, k.sel, k.nb,
          k.lreq, k.lseg, k.lstg, p.vec_bytes, p.unroll, p.chunk_bytes, p.blocks_per_sm, p.warps_per_block,
          p.small_bytes, p.engine, p.stages, p.stage_bytes, p.ring_bytes, ms);
  fclose(f);
}

}  // namespace

int cvd::fail_cuda(cudaError_t e) { return cuda_fail(e); }

namespace cvd {

bool prof_begin(ProfSpan* s, cudaStream_t st) {
  {
    std::lock_guard<std::mutex> pl(g_prof_mu);
    if (!g_prof_on) return false;
  }
  if (cudaEventCreate(&s->a) != cudaSuccess) { cudaGetLastError(); s->a = nullptr; return false; }
  if (cudaEventCreate(&s->b) != cudaSuccess || cudaEventRecord(s->a, st) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(s->a);
    if (s->b) cudaEventDestroy(s->b);
    s->a = s->b = nullptr;
    return false;
  }
  return true;
}

void prof_end(ProfSpan* s, ProfKind kind, cudaStream_t st) {
  if (!s->a) return;
  if (cudaEventRecord(s->b, st) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(s->a);
    cudaEventDestroy(s->b);
  } else {
    std::lock_guard<std::mutex> pl(g_prof_mu);
    g_prof.push_back(ProfRec{s->a, s->b, nullptr, (int)kind});
  }
  s->a = s->b = nullptr;
}

}  // namespace cvd

extern "C" {

int cvd_guest_create(const cvd_guest_desc* d, cvd_guest** out) {
  if (!d || !out || !d->d_host_pool) return CVD_EINVAL;
  if (d->second > CVD_SECOND_EPT || d->reserved1) return CVD_EINVAL;
  const bool ept = d->second == CVD_SECOND_EPT;
  if (ept) {   // the EPT alone backs guest memory; no PT pool (installs are refused)
    if (d->nslots || d->pt_pool_n || (d->ept_root & 4095) || d->host_pool_bytes < 4096 ||
        d->ept_root > d->host_pool_bytes - 4096)
      return CVD_EINVAL;
  } else if (!d->slots || d->nslots == 0 || d->nslots > CVD_MAX_SLOTS) {
    return CVD_EINVAL;
  }
  if (d->rsv_n && !d->d_p2m) return CVD_EINVAL;
  if (d->paging != CVD_PAGING_X86_64 && d->paging != CVD_PAGING_PAE) return CVD_EINVAL;
  if (d->paging == CVD_PAGING_PAE && ((d->cr3_gpa & 31) || d->cr3_gpa >= (1ull << 32))) return CVD_EINVAL;
  std::vector<cvd_memslot> s;
  if (d->nslots) s.assign(d->slots, d->slots + d->nslots);
  std::sort(s.begin(), s.end(), [](const cvd_memslot& x, const cvd_memslot& y) { return x.base_gfn < y.base_gfn; });
  uint64_t pool_frames = d->host_pool_bytes >> 12;
  for (size_t i = 0; i < s.size(); i++) {
    if (s[i].npages == 0 || (s[i].host_off & 4095)) return CVD_EINVAL;
    if (s[i].base_gfn + s[i].npages < s[i].base_gfn) return CVD_EINVAL;
    if ((s[i].host_off >> 12) > pool_frames || s[i].npages > pool_frames - (s[i].host_off >> 12)) return CVD_EINVAL;
    if (i && s[i - 1].base_gfn + s[i - 1].npages > s[i].base_gfn) return CVD_EINVAL;
    if (d->rsv_n && overlaps(d->rsv_gfn, d->rsv_gfn + d->rsv_n, s[i].base_gfn, s[i].base_gfn + s[i].npages))
      return CVD_EINVAL;
  }
  if (d->rsv_n && d->rsv_gfn + d->rsv_n < d->rsv_gfn) return CVD_EINVAL;
  // PT-pool frames must be backed by the slots (the frontend allocated them in guest RAM)
  for (uint64_t f = d->pt_pool_gfn, covered = 0; covered < d->pt_pool_n;) {
    bool hit = false;
    for (auto& sl : s)
      if (f >= sl.base_gfn && f < sl.base_gfn + sl.npages) {
        uint64_t take = std::min(sl.base_gfn + sl.npages - f, d->pt_pool_n - covered);
        covered += take;
        f += take;
        hit = true;
        break;
      }
    if (!hit) return CVD_EINVAL;
  }
  prepare_kernels();
  std::unique_ptr<cvd_guest> g(new cvd_guest());
  memset(&g->host, 0, sizeof(DevGuest));
  g->host.pool = reinterpret_cast<uint8_t*>(d->d_host_pool);
  g->host.pool_bytes = d->host_pool_bytes;
  g->host.cr3_gpa = d->cr3_gpa;
  g->host.paging = d->paging;
  g->host.rsv_gfn = d->rsv_gfn;
  g->host.rsv_n = d->rsv_n;
  g->host.p2m = d->d_p2m;
  g->host.pt_pool_gfn = d->pt_pool_gfn;
  g->host.pt_pool_n = d->pt_pool_n;
  g->host.nslots = d->nslots;
  g->host.ept = ept ? 1u : 0u;
  g->host.ept_root = ept ? d->ept_root : 0;
  // unit tables: every slot on 2 MiB guest-frame boundaries below kUnitSlots
  // units, with its host-frame delta inside the int32 range
  bool units = d->nslots > 0 && d->nslots < kNoUnit;
  uint64_t nunits = 0;
  for (uint32_t i = 0; i < d->nslots && units; i++) {
    const int64_t delta = (int64_t)(s[i].host_off >> 12) - (int64_t)s[i].base_gfn;
    units = (s[i].base_gfn % 512) == 0 && (s[i].npages % 512) == 0 &&
            s[i].base_gfn + s[i].npages <= (uint64_t)kUnitSlots * 512 && delta > (int64_t)INT32_MIN &&
            delta <= (int64_t)INT32_MAX;
    nunits = std::max<uint64_t>(nunits, (s[i].base_gfn + s[i].npages) / 512);
  }
  const size_t delta_bytes = 4 * ((nunits + 3) & ~3ull);   // 16-byte multiple: staged as 16-byte vectors
  std::vector<uint8_t> table;
  if (units) {
    table.assign(delta_bytes + nunits, 0);
    int32_t* dl = reinterpret_cast<int32_t*>(table.data());
    uint8_t* sl = table.data() + delta_bytes;
    for (uint64_t u = 0; u < delta_bytes / 4; u++) dl[u] = kNoUnitDelta;
    memset(sl, kNoUnit, nunits);
    for (uint32_t i = 0; i < d->nslots; i++)
      for (uint64_t u = s[i].base_gfn / 512; u < (s[i].base_gfn + s[i].npages) / 512; u++) {
        dl[u] = (int32_t)((int64_t)(s[i].host_off >> 12) - (int64_t)s[i].base_gfn);
        sl[u] = (uint8_t)i;
      }
  }
  g->host.nunits = 0;
  g->host.unit_delta = nullptr;
  g->host.unit_slot = nullptr;
  g->d_units = nullptr;
  for (uint32_t i = 0; i < d->nslots; i++) g->host.slots[i] = DevSlot{s[i].base_gfn, s[i].npages, s[i].host_off};
  cudaGetDevice(&g->device);
  g->dev = nullptr;
  g->d_alloc = nullptr;
  if (cudaMalloc(&g->dev, sizeof(DevGuest)) != cudaSuccess || cudaMalloc(&g->d_alloc, 16) != cudaSuccess) {
    cudaGetLastError();
    if (g->dev) cudaFree(g->dev);
    return CVD_ENOMEM;
  }
  auto fail = [&](cudaError_t e) {   // a failed copy: free what was allocated
    cudaFree(g->dev);
    cudaFree(g->d_alloc);
    if (g->d_units) cudaFree(g->d_units);
    return cuda_fail(e);
  };
  g->host.alloc = g->d_alloc;
  cudaError_t e = cudaMemset(g->d_alloc, 0, 16);
  if (e != cudaSuccess) return fail(e);
  if (units && cudaMalloc(&g->d_units, table.size()) == cudaSuccess) {   // without it, lookups search the slots
    e = cudaMemcpy(g->d_units, table.data(), table.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(e);
    g->host.unit_delta = reinterpret_cast<const int32_t*>(g->d_units);
    g->host.unit_slot = g->d_units + delta_bytes;
    g->host.nunits = (uint32_t)nunits;
  } else {
    cudaGetLastError();
    g->d_units = nullptr;
  }
  e = cudaMemcpy(g->dev, &g->host, sizeof(DevGuest), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(e);
  *out = g.release();
  return CVD_OK;
}

int cvd_guest_destroy(cvd_guest* g) {
  if (!g) return CVD_EINVAL;
  cudaDeviceSynchronize();
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& kv : g_ws) {   // cached graphs and guest arrays may name this guest
      std::lock_guard<std::mutex> l2(kv.second->mu);
      kv.second->drop_graphs();
      kv.second->guest_list.clear();
    }
    for (auto& kv : g_pipes)   // and the planned-ahead slots' guest arrays
      for (auto& w : kv.second->w) {
        std::lock_guard<std::mutex> l2(w.mu);
        w.guest_list.clear();
      }
  }
  cudaFree(g->dev);
  cudaFree(g->d_alloc);
  if (g->d_units) cudaFree(g->d_units);
  delete g;
  return CVD_OK;
}

int cvd_guest_alloc_state(cvd_guest* g, uint64_t* pt_used, uint64_t* rsv_used) {
  if (!g || !pt_used || !rsv_used) return CVD_EINVAL;
  uint64_t v[2];
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(v, g->d_alloc, 16, cudaMemcpyDeviceToHost));
  *pt_used = v[0];
  *rsv_used = v[1];
  return CVD_OK;
}

int cvd_guest_set_alloc_state(cvd_guest* g, uint64_t pt_used, uint64_t rsv_used) {
  if (!g || pt_used > g->host.pt_pool_n || rsv_used > g->host.rsv_n) return CVD_EINVAL;
  const uint64_t v[2] = {pt_used, rsv_used};
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(g->d_alloc, v, 16, cudaMemcpyHostToDevice));
  return CVD_OK;
}

int cvd_translate(cvd_guest* g, const uint64_t* d_gva, uint64_t n, uint32_t access, uint64_t* d_gpa,
                  uint64_t* d_hpa, uint32_t* d_fault, cvd_stream_t stream) {
  if (!g || access > 1) return CVD_EINVAL;
  if (n && (!d_gva || !d_gpa || !d_hpa || !d_fault)) return CVD_EINVAL;
  prepare_kernels();
  CK(launch_translate(g->dev, walk_selector(g->host), g->host.paging, g->host.nunits, d_gva, n, access == 1, d_gpa,
                      d_hpa, d_fault, (cudaStream_t)stream));
  return CVD_OK;
}

// Scratch of cvd_gather_chained, per device (one call at a time: a mutex).
struct ChainWs { DevBuf q1, s1, r1, len, pairs, offs, tmp, q2, s2, r2; };
static std::mutex g_chain_mu;
static std::map<int, ChainWs> g_chain_ws;

int cvd_gather_chained(cvd_guest* const* guests, uint32_t nguests, const cvd_chain_req* d_req, uint32_t nreq,
                       void* d_desc, uint64_t desc_bytes, void* d_payload, uint64_t payload_bytes,
                       cvd_chain_result* d_res, uint32_t flags, cvd_stream_t stream) {
  if (flags & ~(CVD_BATCH_HAZARD_FREE | CVD_BATCH_CHECK)) return CVD_EINVAL;
  if (nreq && (!d_req || !d_res)) return CVD_EINVAL;
  if (desc_bytes && (!d_desc || ((uintptr_t)d_desc & 15))) return CVD_EINVAL;
  if (desc_bytes >= (1ull << 36)) return CVD_EINVAL;   // entry places are u32
  if (payload_bytes && !d_payload) return CVD_EINVAL;
  // payload places are sums of at most nreq lengths clamped to payload_bytes + 1
  if (nreq && (payload_bytes >= (1ull << 52) || (payload_bytes + 1) > (1ull << 63) / nreq)) return CVD_EINVAL;
  if (nreq == 0) return CVD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  prepare_kernels();
  std::lock_guard<std::mutex> lk(g_chain_mu);
  int dev = 0;
  cudaGetDevice(&dev);
  ChainWs& W = g_chain_ws[dev];
  const size_t n = nreq, np = 2 * (n + 1);
  // the payload entry list holds as many entries as the descriptor buffer
  const uint64_t ecap = desc_bytes / 16;
  if (!W.q1.grow(n * sizeof(Req), nullptr) || !W.s1.grow(n * sizeof(Seg), nullptr) ||
      !W.r1.grow(n * sizeof(Result), nullptr) || !W.len.grow(n * 8, nullptr) || !W.pairs.grow(np * 8, nullptr) ||
      !W.offs.grow(np * 8, nullptr) || !W.tmp.grow(2 * scan_tmp_elems(n) * 8, nullptr) ||
      !W.q2.grow(n * sizeof(Req), nullptr) || !W.r2.grow(n * sizeof(Result), nullptr) ||
      !W.s2.grow(std::max<uint64_t>(ecap, 1) * sizeof(Seg), nullptr))
    return CVD_ENOMEM;
  const ChainReq* req = reinterpret_cast<const ChainReq*>(d_req);
  ChainRes* res = reinterpret_cast<ChainRes*>(d_res);
  const uint8_t* desc = reinterpret_cast<const uint8_t*>(d_desc);
  // level 1: the descriptor tables (a hazard-free call reads them in one
  // launch; otherwise as a batch of one copy_from request per table)
  CK(launch_chain_l1(req, nreq, nguests, W.q1.as<Req>(), W.s1.as<Seg>(), st));
  Call c1{guests, nguests, reinterpret_cast<const cvd_req*>(W.q1.p), nreq,
          reinterpret_cast<const cvd_seg*>(W.s1.p), nreq, d_desc, desc_bytes,
          reinterpret_cast<cvd_result*>(W.r1.p), flags, -1};
  int rc;
  if (flags == CVD_BATCH_HAZARD_FREE) {
    if ((rc = validate(c1))) return rc;
    Workspace& ws = workspace(st);
    std::lock_guard<std::mutex> wl(ws.mu);
    BatchArgs a;
    bool moved = false;
    if ((rc = prepare(ws, c1, &a, &moved, st))) return rc;
    CK(launch_chain_tables(a, req, nreq, W.r1.as<Result>(), st));
  } else if ((rc = run_batch(c1, st))) {
    return rc;
  }
  // lengths, payload places and entry places (device-side scan: no host round trip)
  CK(launch_chain_len(req, nreq, W.r1.as<Result>(), desc, payload_bytes, W.len.as<uint64_t>(),
                      W.pairs.as<uint64_t>(), st));
  CK(launch_scan_pairs(W.pairs.as<uint64_t>(), W.offs.as<uint64_t>(), n, W.tmp.as<uint64_t>(), st));
  CK(launch_chain_l2(req, nreq, W.r1.as<Result>(), W.len.as<uint64_t>(), W.offs.as<uint64_t>(), desc, payload_bytes,
                     ecap, W.q2.as<Req>(), W.s2.as<Seg>(), res, st));
  // level 2: the payload gathers over the entry list (its capacity bounds the segments)
  Call c2{guests, nguests, reinterpret_cast<const cvd_req*>(W.q2.p), nreq,
          reinterpret_cast<const cvd_seg*>(W.s2.p), ecap, d_payload, payload_bytes,
          reinterpret_cast<cvd_result*>(W.r2.p), CVD_BATCH_HAZARD_FREE, -1};
  rc = run_batch(c2, st);
  if (rc) return rc;
  CK(launch_chain_final(W.r2.as<Result>(), nreq, res, st));
  return CVD_OK;
}

int cvd_copy_batches(cvd_guest* const* guests, uint32_t nguests, const cvd_dev_batch* batches, uint32_t nbatches,
                     void* d_host_buf, uint64_t host_buf_bytes, uint32_t flags, cvd_stream_t stream) {
  if (flags != CVD_BATCH_HAZARD_FREE || (nbatches && !batches)) return CVD_EINVAL;
  return run_batches_dev(guests, nguests, batches, nbatches, d_host_buf, host_buf_bytes, (cudaStream_t)stream);
}

static std::mutex g_map_mu;   // the installer's and the placer's scratch is shared by all streams

int cvd_mmap_install(cvd_guest* g, const cvd_map_req* d_req, uint32_t nreq, const uint64_t* d_hf, uint64_t nhf,
                     int32_t* d_page_status, cvd_stream_t stream) {
  if (!g || (nreq && (!d_req || !d_page_status)) || (nhf && !d_hf)) return CVD_EINVAL;
  prepare_kernels();
  std::lock_guard<std::mutex> lk(g_map_mu);
  int rc = mmap_install(g->dev, g->host, reinterpret_cast<const MapReq*>(d_req), nreq, d_hf, nhf, d_page_status,
                        (cudaStream_t)stream);
  if (rc == -5) return cuda_fail(cudaGetLastError());
  return rc;
}

int cvd_mmap_place(cvd_guest* g, uint64_t va_lo, uint64_t va_hi, const cvd_map_place_req* d_req, uint32_t nreq,
                   const uint64_t* d_hf, uint64_t nhf, uint64_t* d_gva, int32_t* d_page_status, cvd_stream_t stream) {
  if (!g || (nreq && (!d_req || !d_gva || !d_page_status)) || (nhf && !d_hf)) return CVD_EINVAL;
  const uint64_t top = g->host.paging == kPagingPae ? kPaeTop : kUserTop;
  if ((va_lo & 4095) || (va_hi & 4095) || va_lo >= va_hi || va_hi > top) return CVD_EINVAL;
  prepare_kernels();
  std::lock_guard<std::mutex> lk(g_map_mu);
  int rc = mmap_place(g->dev, g->host, va_lo, va_hi, reinterpret_cast<const MapPlaceReq*>(d_req), nreq, d_hf, nhf,
                      d_gva, d_page_status, (cudaStream_t)stream);
  if (rc == -5) return cuda_fail(cudaGetLastError());
  return rc;
}

int cvd_copy_from_guest(cvd_guest* g, const cvd_req* d_req, uint32_t nreq, const cvd_seg* d_seg, uint64_t nseg,
                        void* d_host_buf, uint64_t host_buf_bytes, cvd_result* d_res, cvd_stream_t stream) {
  if (!g) return CVD_EINVAL;
  Call c{&g, 1, d_req, nreq, d_seg, nseg, d_host_buf, host_buf_bytes, d_res, 0, 0};
  return run_batch(c, (cudaStream_t)stream);
}

int cvd_copy_to_guest(cvd_guest* g, const cvd_req* d_req, uint32_t nreq, const cvd_seg* d_seg, uint64_t nseg,
                      const void* d_host_buf, uint64_t host_buf_bytes, cvd_result* d_res, cvd_stream_t stream) {
  if (!g) return CVD_EINVAL;
  Call c{&g, 1, d_req, nreq, d_seg, nseg, const_cast<void*>(d_host_buf), host_buf_bytes, d_res, 0, 1};
  return run_batch(c, (cudaStream_t)stream);
}

int cvd_copy_batch(cvd_guest* const* guests, uint32_t nguests, const cvd_req* d_req, uint32_t nreq,
                   const cvd_seg* d_seg, uint64_t nseg, void* d_host_buf, uint64_t host_buf_bytes,
                   cvd_result* d_res, uint32_t flags, cvd_stream_t stream) {
  if (flags & ~(CVD_BATCH_HAZARD_FREE | CVD_BATCH_GRAPH | CVD_BATCH_CHECK)) return CVD_EINVAL;
  Call c{guests, nguests, d_req, nreq, d_seg, nseg, d_host_buf, host_buf_bytes, d_res, flags, -1};
  return run_batch(c, (cudaStream_t)stream);
}

int cvd_copy_batch_host(cvd_guest* const* guests, uint32_t nguests, const cvd_req* h_req, uint32_t nreq,
                        const cvd_seg* h_seg, uint64_t nseg, void* h_host_buf, uint64_t host_buf_bytes,
                        cvd_result* h_res, uint32_t flags, cvd_stream_t stream) {
  cvd_host_batch b;
  b.h_req = h_req; b.nreq = nreq; b.pad = 0; b.h_seg = h_seg; b.nseg = nseg;
  b.h_host_buf = h_host_buf; b.host_buf_bytes = host_buf_bytes; b.h_res = h_res;
  return cvd_copy_batches_host(guests, nguests, &b, 1, flags, stream);
}

int cvd_copy_batches_host(cvd_guest* const* guests, uint32_t nguests, const cvd_host_batch* bt, uint32_t nb,
                          uint32_t flags, cvd_stream_t stream) {
  if (flags & ~(CVD_BATCH_HAZARD_FREE | CVD_BATCH_CHECK)) return CVD_EINVAL;
  if (nb && !bt) return CVD_EINVAL;
  for (uint32_t i = 0; i < nb; i++) {
    const cvd_host_batch& b = bt[i];
    if ((b.nreq && (!b.h_req || !b.h_res)) || (b.nseg && !b.h_seg) || (b.host_buf_bytes && !b.h_host_buf))
      return CVD_EINVAL;
  }
  if (nb == 0) return CVD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Workspace& ws = workspace(st);
  // Byte ranges of each host buffer the batch reads (copy-to sources) and may
  // write (copy-from destinations), from the host copies of the descriptors.
  // Requests whose range leaves the buffer are rejected on the device
  // (HOSTBUF) and transfer nothing.  Copy-to ranges less than 64 KiB apart
  // travel as one copy (the bytes between them are never written back unless
  // a written range spans them).
  struct Plan { Ranges in; std::vector<std::pair<uint64_t, uint64_t>> span; uint64_t wlo = ~0ull, whi = 0; };
  std::vector<Plan> pl(nb);
  size_t mreq = 1, mseg = 1, mstg = 16;
  for (uint32_t i = 0; i < nb; i++) {
    const cvd_host_batch& b = bt[i];
    Plan& P = pl[i];
    P.span.assign(b.nreq, {0, 0});
    for (uint32_t r = 0; r < b.nreq; r++) {
      uint64_t L = 0;
      const cvd_req& q = b.h_req[r];
      if (!host_req_len(q, b.h_seg, b.nseg, &L) || L == 0) continue;
      if (L > b.host_buf_bytes || q.host_off > b.host_buf_bytes - L) continue;
      P.span[r] = {q.host_off, q.host_off + L};
      if (q.dir == 1) P.in.push_back(P.span[r]);
      if (q.dir == 0) { P.wlo = std::min(P.wlo, q.host_off); P.whi = std::max(P.whi, q.host_off + L); }
    }
    P.in = merge_ranges(std::move(P.in), 64u << 10);
    mreq = std::max<size_t>(mreq, b.nreq);
    mseg = std::max<size_t>(mseg, b.nseg);
    mstg = std::max<size_t>(mstg, b.host_buf_bytes);
  }
  {
    std::lock_guard<std::mutex> lk(ws.mu);
    bool mv = false;
    for (auto& S : ws.hs) {
      if (!S.req.grow(mreq * sizeof(cvd_req), &mv) || !S.seg.grow(mseg * sizeof(cvd_seg), &mv) ||
          !S.stg.grow(mstg, &mv) || !S.res.grow(mreq * sizeof(cvd_result), &mv))
        return CVD_ENOMEM;
      for (cudaEvent_t* e : {&S.in, &S.res_done, &S.free})
        if (!*e) CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
    if (!ws.up) CK(cudaStreamCreateWithFlags(&ws.up, cudaStreamNonBlocking));
    if (!ws.down) CK(cudaStreamCreateWithFlags(&ws.down, cudaStreamNonBlocking));
    if (!ws.res) CK(cudaStreamCreateWithFlags(&ws.res, cudaStreamNonBlocking));
  }
  // Work of batch i runs on the caller's stream (batches in order); its inputs
  // go up on ws.up into slot i % 2 once the slot's previous outputs have left;
  // its results come back on ws.res and its written bytes on ws.down (which
  // thus holds only write-backs, in batch order: a wait for batch i's kernel
  // queued there would hold back batch i - 1's write-back behind batch i's
  // inputs).
  auto send = [&](uint32_t i) -> int {
    const cvd_host_batch& b = bt[i];
    Workspace::HostSlot& S = ws.hs[i & 1];
    if (i >= 2) CK(cudaStreamWaitEvent(ws.up, S.free, 0));
    if (b.nreq) CK(cudaMemcpyAsync(S.req.p, b.h_req, b.nreq * sizeof(cvd_req), cudaMemcpyHostToDevice, ws.up));
    if (b.nseg) CK(cudaMemcpyAsync(S.seg.p, b.h_seg, b.nseg * sizeof(cvd_seg), cudaMemcpyHostToDevice, ws.up));
    const uint8_t* hb = reinterpret_cast<const uint8_t*>(b.h_host_buf);
    for (auto& r : pl[i].in)
      CK(cudaMemcpyAsync(S.stg.as<uint8_t>() + r.first, hb + r.first, r.second - r.first, cudaMemcpyHostToDevice,
                         ws.up));
    CK(cudaEventRecord(S.in, ws.up));
    return CVD_OK;
  };
  auto run = [&](uint32_t i) -> int {
    const cvd_host_batch& b = bt[i];
    Workspace::HostSlot& S = ws.hs[i & 1];
    CK(cudaStreamWaitEvent(st, S.in, 0));
    int rc = cvd_copy_batch(guests, nguests, S.req.as<cvd_req>(), b.nreq, S.seg.as<cvd_seg>(), b.nseg, S.stg.p,
                            b.host_buf_bytes, S.res.as<cvd_result>(), flags, stream);
    if (rc) return rc;
    CK(cudaEventRecord(S.res_done, st));
    CK(cudaStreamWaitEvent(ws.res, S.res_done, 0));
    if (b.nreq) CK(cudaMemcpyAsync(b.h_res, S.res.p, b.nreq * sizeof(cvd_result), cudaMemcpyDeviceToHost, ws.res));
    CK(cudaEventRecord(S.res_done, ws.res));
    return CVD_OK;
  };
  // A copy-from request the device accepted wrote its whole range (copied
  // prefix, zero-filled tail); one it rejected (BADREQ, HOSTBUF) wrote
  // nothing.  Only written ranges come back; two of them travel as one copy
  // when the bytes between them went up unchanged.
  auto recv = [&](uint32_t i) -> int {
    const cvd_host_batch& b = bt[i];
    Workspace::HostSlot& S = ws.hs[i & 1];
    CK(cudaEventSynchronize(S.res_done));
    Ranges out;
    for (uint32_t r = 0; r < b.nreq; r++)
      if (b.h_req[r].dir == 0 && pl[i].span[r].second > pl[i].span[r].first && b.h_res[r].fault_code != kBadReq &&
          b.h_res[r].fault_code != kHostBuf)
        out.push_back(pl[i].span[r]);
    out = merge_ranges(std::move(out), 0);
    Ranges back;
    for (auto& r : out) {
      if (!back.empty() && covered(pl[i].in, back.back().second, r.first)) back.back().second = r.second;
      else back.push_back(r);
    }
    uint8_t* hb = reinterpret_cast<uint8_t*>(b.h_host_buf);
    for (auto& r : back)
      CK(cudaMemcpyAsync(hb + r.first, S.stg.as<uint8_t>() + r.first, r.second - r.first, cudaMemcpyDeviceToHost,
                         ws.down));
    CK(cudaEventRecord(S.free, ws.down));
    return CVD_OK;
  };
  // Batch i's inputs must not be read from host bytes that batch i - 1 may
  // still write back: then they go up only after those writes.
  auto depends = [&](uint32_t i) {
    const Plan& W = pl[i - 1];
    if (W.wlo >= W.whi || pl[i].in.empty()) return false;
    const uint64_t w0 = (uint64_t)(uintptr_t)bt[i - 1].h_host_buf + W.wlo;
    const uint64_t w1 = (uint64_t)(uintptr_t)bt[i - 1].h_host_buf + W.whi;
    const uint64_t base = (uint64_t)(uintptr_t)bt[i].h_host_buf;
    for (auto& r : pl[i].in)
      if (base + r.first < w1 && w0 < base + r.second) return true;
    return false;
  };
  auto body = [&]() -> int {
    int rc;
    if ((rc = send(0)) || (rc = run(0))) return rc;
    for (uint32_t i = 1; i < nb; i++) {
      if (depends(i)) {
        if ((rc = recv(i - 1))) return rc;
        CK(cudaStreamWaitEvent(ws.up, ws.hs[(i - 1) & 1].free, 0));
        if ((rc = send(i)) || (rc = run(i))) return rc;
      } else {
        if ((rc = send(i)) || (rc = run(i)) || (rc = recv(i - 1))) return rc;
      }
    }
    if ((rc = recv(nb - 1))) return rc;
    CK(cudaStreamSynchronize(ws.down));
    return CVD_OK;
  };
  int rc = body();
  if (rc) {   // leave no copy in flight on the caller's buffers
    cudaStreamSynchronize(ws.up);
    cudaStreamSynchronize(st);
    cudaStreamSynchronize(ws.res);
    cudaStreamSynchronize(ws.down);
    cudaGetLastError();
  }
  return rc;
}

int cvd_get_copy_params(cvd_copy_params* p) {
  if (!p) return CVD_EINVAL;
  *p = to_abi(current_params());
  return CVD_OK;
}

int cvd_set_copy_params(const cvd_copy_params* p) {
  if (!p || !params_ok(*p)) return CVD_EINVAL;
  set_current_params(from_abi(*p));
  return CVD_OK;
}

int cvd_tune(cvd_guest* const* guests, uint32_t nguests, const cvd_req* d_req, uint32_t nreq, const cvd_seg* d_seg,
             uint64_t nseg, void* d_host_buf, uint64_t host_buf_bytes, cvd_result* d_res, uint32_t reps,
             cvd_stream_t stream, cvd_copy_params* best, float* best_ms) {
  Call c{guests, nguests, d_req, nreq, d_seg, nseg, d_host_buf, host_buf_bytes, d_res, CVD_BATCH_HAZARD_FREE, -1};
  int v = validate(c);
  if (v) return v;
  if (reps == 0) reps = 1;
  cudaStream_t st = (cudaStream_t)stream;
  prepare_kernels();
  Workspace& ws = workspace(st);
  std::lock_guard<std::mutex> lk(ws.mu);
  BatchArgs a;
  bool moved = false;
  int rc = prepare(ws, c, &a, &moved, st);
  if (rc) return rc;
  CK(launch_plan(a, st));   // the copy engine never changes the plan's outputs
  const CopyParams base = current_params();
  const std::vector<CopyParams> cands = tune_candidates(base, false);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float bestt = 1e30f;
  CopyParams bp = base;
  for (const CopyParams& p : cands) {
      {
        CK(launch_copy(a, p, st));   // warm-up
        CK(cudaEventRecord(e0, st));
        for (uint32_t r = 0; r < reps; r++) CK(launch_copy(a, p, st));
        CK(cudaEventRecord(e1, st));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        ms /= reps;
        if (ms < bestt) { bestt = ms; bp = p; }
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  set_current_params(bp);
  if (best) *best = to_abi(bp);
  if (best_ms) *best_ms = bestt;
  return CVD_OK;
}

int cvd_tune_batches(cvd_guest* const* guests, uint32_t nguests, const cvd_dev_batch* batches, uint32_t nbatches,
                     void* d_host_buf, uint64_t host_buf_bytes, uint32_t reps, cvd_stream_t stream,
                     cvd_copy_params* best, float* best_ms, int* cached) {
  if (nbatches == 0 || !batches) return CVD_EINVAL;
  uint64_t nreq = 0, nseg = 0;
  for (uint32_t k = 0; k < nbatches; k++) {
    Call c{guests, nguests, batches[k].d_req, batches[k].nreq, batches[k].d_seg, batches[k].nseg, d_host_buf,
           host_buf_bytes, batches[k].d_res, CVD_BATCH_HAZARD_FREE, -1};
    int v = validate(c);
    if (v) return v;
    nreq += batches[k].nreq;
    nseg += batches[k].nseg;
  }
  if (reps == 0) reps = 1;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, dev));
  uint32_t sel = walk_selector(guests[0]->host);
  for (uint32_t i = 1; i < nguests; i++)
    if (walk_selector(guests[i]->host) != sel) sel = 0xFFu;
  TuneKey key{prop.name, nguests, sel, nbatches, log2_bucket(nreq), log2_bucket(nseg), log2_bucket(host_buf_bytes)};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_cache_read_file();
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      set_current_params(it->second.first);
      if (best) *best = to_abi(it->second.first);
      if (best_ms) *best_ms = it->second.second;
      if (cached) *cached = 1;
      return CVD_OK;
    }
  }
  const CopyParams base = current_params();
  const std::vector<CopyParams> cands = tune_candidates(base, true);
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float bestt = 1e30f;
  CopyParams bp = base;
  int rc = CVD_OK;
  for (const CopyParams& p : cands) {
    set_current_params(p);
    rc = run_batches_dev(guests, nguests, batches, nbatches, d_host_buf, host_buf_bytes, st);   // warm-up
    if (rc) break;
    CK(cudaEventRecord(e0, st));
    for (uint32_t r = 0; r < reps && rc == CVD_OK; r++)
      rc = run_batches_dev(guests, nguests, batches, nbatches, d_host_buf, host_buf_bytes, st);
    if (rc) break;
    CK(cudaEventRecord(e1, st));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    ms /= reps;
    if (ms < bestt) { bestt = ms; bp = p; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  set_current_params(rc ? base : bp);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = {bp, bestt};
    tune_cache_append_file(key, bp, bestt);
  }
  if (best) *best = to_abi(bp);
  if (best_ms) *best_ms = bestt;
  if (cached) *cached = 0;
  return CVD_OK;
}

int cvd_stream_check(cvd_stream_t stream, uint32_t* error_bits) {
  if (!error_bits) return CVD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Workspace& ws = workspace(st);
  std::lock_guard<std::mutex> lk(ws.mu);
  *error_bits = 0;
  CK(cudaStreamSynchronize(st));
  if (ws.err.p) {
    CK(cudaMemcpy(error_bits, ws.err.p, 4, cudaMemcpyDeviceToHost));
    CK(cudaMemset(ws.err.p, 0, 4));
  }
  // the no-allocation batch call keeps its own word in its fixed scratch
  unsigned int na = 0;
  CK(noalloc_take_errors(st, &na));
  *error_bits |= na;
  return CVD_OK;
}

int cvd_selftest_wait_timeout(cvd_stream_t stream, uint32_t tries, uint32_t* error_bits) {
  if (!error_bits || tries == 0 || tries > (1u << 22)) return CVD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Workspace& ws = workspace(st);
  {
    std::lock_guard<std::mutex> lk(ws.mu);
    if (!ws.err.p) {
      bool mv = false;
      if (!ws.err.grow(256, &mv)) return CVD_ENOMEM;
      CK(cudaMemsetAsync(ws.err.p, 0, 256, st));
    }
    CK(launch_wait_selftest(ws.err.as<unsigned int>(), tries, st));
  }
  return cvd_stream_check(stream, error_bits);
}

int cvd_last_levels(cvd_stream_t stream, uint32_t* levels) {
  if (!levels) return CVD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Workspace& ws = workspace(st);
  std::lock_guard<std::mutex> lk(ws.mu);
  if (ws.levels_on_device) {   // 1: one parallel pass; 2: conflicting requests also ran in order
    unsigned int marked = 0;
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpy(&marked, hz_flag_of(ws) + 1, 4, cudaMemcpyDeviceToHost));
    *levels = marked ? 2u : 1u;
    return CVD_OK;
  }
  *levels = ws.last_levels;
  return CVD_OK;
}

int cvd_level_runs(const cvd_run* runs, uint64_t n, int32_t* levels, uint64_t* marked) {
  static_assert(sizeof(cvd_run) == sizeof(Run), "cvd_run and the internal run record share one layout");
  if (!marked || (n && (!runs || !levels))) return CVD_EINVAL;
  for (uint64_t i = 0; i < n; i++)
    if (runs[i].dst + runs[i].len < runs[i].dst || runs[i].src + runs[i].len < runs[i].src) return CVD_EINVAL;
  try {
    LevelScratch S;
    std::vector<int> lev(n);
    const int maxl = level_runs(S, reinterpret_cast<const Run*>(runs), n, lev.data(), marked);
    for (uint64_t i = 0; i < n; i++) levels[i] = lev[i];
    return maxl;
  } catch (const std::bad_alloc&) {
    return CVD_ENOMEM;
  }
}

int cvd_profile_enable(int on) {
  std::lock_guard<std::mutex> pl(g_prof_mu);
  g_prof_on = on != 0;
  return CVD_OK;
}

int cvd_profile_read(cvd_profile* out) {
  if (!out) return CVD_EINVAL;
  std::vector<ProfRec> recs;
  {
    std::lock_guard<std::mutex> pl(g_prof_mu);
    recs.swap(g_prof);
  }
  memset(out, 0, sizeof(*out));
  int rc = CVD_OK;
  for (auto& r : recs) {
    float x = 0, y = 0;
    if (rc == CVD_OK && r.kind == 0) {
      cudaError_t e = cudaEventSynchronize(r.c);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&x, r.a, r.b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&y, r.b, r.c);
      if (e != cudaSuccess) rc = cuda_fail(e);
      out->plan_ms += x;
      out->copy_ms += y;
      out->plan_calls++;
      out->copy_calls++;
    } else if (rc == CVD_OK) {
      cudaError_t e = cudaEventSynchronize(r.b);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&x, r.a, r.b);
      if (e != cudaSuccess) rc = cuda_fail(e);
      if (r.kind == cvd::kProfMapProbe) { out->map_probe_ms += x; out->map_probe_calls++; }
      if (r.kind == cvd::kProfPlaceFit) { out->place_fit_ms += x; out->place_fit_calls++; }
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
    if (r.c) cudaEventDestroy(r.c);
  }
  return rc;
}

uint64_t cvd_launch_count(void) { return g_launches; }

int cvd_last_cuda_error(void) { return t_last_cuda; }

const char* cvd_strerror(int s) {
  switch (s) {
    case CVD_OK: return "ok";
    case CVD_EINVAL: return "invalid argument";
    case CVD_ENOMEM: return "out of memory";
    case CVD_ECUDA: return "CUDA error";
    case CVD_ETIMEDOUT: return "timed out";
    case CVD_EHAZARD: return "batch declared hazard-free has conflicting requests";
    case CVD_E2BIG: return "batch exceeds the fixed scratch of cvd_copy_batch_noalloc";
    default: return "unknown status";
  }
}

}  // extern "C"
