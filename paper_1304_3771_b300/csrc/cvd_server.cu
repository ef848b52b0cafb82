// cvd_server.cu -- serving request loop: continuous batching of forwarded
// memory operations from several guests (the batches of cvd_copy_batch fed
// from an arrival queue).
//
// Paper analogue: the dual thread (Sec. 5) lets forwarded operations proceed
// without blocking the guest and lets operations of different threads and
// devices overlap; here requests that arrive while others are on the GPU are
// admitted as staging memory and in-flight slots free up, and up to three
// waves are queued on the GPU at a time.
//
// Design:
//  * Requests carry a scheduled arrival time (ns since the server epoch), so
//    an open-loop arrival process is replayed exactly; a request is never
//    admitted before its arrival time.
//  * Admission is FIFO in arrival order: the head request is admitted when
//    fewer than max_inflight requests are admitted and its stream length fits
//    in the staging arena (best-fit allocator); later requests wait behind it.
//    The completion thread admits as waves free staging and slots, a
//    scheduler as arrival times pass.
//  * All waves go to one stream (with CVD_SERVER_TWO_STREAMS guest g uses
//    stream g % 2), so every guest's requests take effect in arrival order
//    (stream order) and different guests never conflict across streams.  One
//    stream is the default: the copy engine's persistent grid takes whole SMs,
//    so kernels of two streams wait for each other's SMs and each wave takes
//    several times longer than on one stream (measured on B300).  Each
//    scheduler thread launches one wave (up to max_batch of its stream's
//    admitted requests, in arrival order) as a levelled batch: the requests
//    whose guest frames conflict with another request of the wave are marked
//    on the device and copied in arrival order by one block after the
//    others, so sequential semantics hold inside the wave without a host
//    round trip.
//  * copy-to requests carry a device source; their bytes are gathered into
//    their staging range by a run-copy launch just before the wave.
//  * A completion thread polls the waves' events (a blocking-sync event wait
//    instead measured slower: its wake-up adds to every wave); completions
//    record arrival, admission, launch and completion times.  copy-from
//    results stay in the staging arena until cvd_server_release.  All waits
//    are bounded.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/cvd.h"
#include "cvd_internal.h"

using namespace cvd;

namespace {

using Clock = std::chrono::steady_clock;

struct Item {
  uint64_t ticket, tag;
  uint32_t guest, dir;
  std::vector<cvd_seg> segs;
  uint64_t len;
  uint64_t src;          // copy-to source (device)
  uint64_t arrival_ns;   // scheduled
  uint64_t admit_ns = 0, launch_ns = 0;
  uint64_t stg_off = 0;
};

// Descriptor/result buffers of one wave (reused).  A wave's requests, its
// segments and its gather runs lie back to back in one pinned, mapped block,
// which the wave's input kernel reads through its device address; results
// come back into pinned memory asynchronously.
struct WaveBuf {
  unsigned char* h_in = nullptr;   // requests | segments | runs (pinned, mapped)
  const unsigned char* h_in_dev = nullptr;   // its device address (the wave's input kernel reads it)
  void* d_in = nullptr;
  cvd_result* h_res = nullptr;
  void* d_res = nullptr;
  size_t cap_in = 0, cap_req = 0;
  cudaEvent_t start = nullptr, done = nullptr;   // the wave's first and last command (timed)
  bool busy = false;
  // The block for nreq requests, nseg segments and nruns runs: offsets of the
  // segments and the runs, and the block's size.
  static void layout(size_t nreq, size_t nseg, size_t nruns, size_t* off_seg, size_t* off_runs, size_t* bytes) {
    *off_seg = (nreq * sizeof(cvd_req) + 31) & ~(size_t)31;
    *off_runs = (*off_seg + nseg * sizeof(cvd_seg) + 31) & ~(size_t)31;
    *bytes = *off_runs + nruns * sizeof(Run);
  }
  bool reserve(size_t nreq, size_t nseg, size_t nruns) {
    size_t os, orr, in;
    layout(nreq, nseg, nruns, &os, &orr, &in);
    if (in <= cap_in && nreq <= cap_req) return true;
    release();
    cap_in = std::max(in, cap_in);
    cap_req = std::max(nreq, cap_req);
    void* hd = nullptr;
    bool ok = cudaHostAlloc((void**)&h_in, cap_in, cudaHostAllocMapped) == cudaSuccess &&
              cudaHostGetDevicePointer(&hd, h_in, 0) == cudaSuccess &&
              cudaHostAlloc((void**)&h_res, cap_req * sizeof(cvd_result), cudaHostAllocDefault) == cudaSuccess &&
              cudaMalloc(&d_in, cap_in) == cudaSuccess &&
              cudaMalloc(&d_res, cap_req * sizeof(cvd_result)) == cudaSuccess &&
              (start || cudaEventCreate(&start) == cudaSuccess) && (done || cudaEventCreate(&done) == cudaSuccess);
    h_in_dev = static_cast<const unsigned char*>(hd);
    if (!ok) cudaGetLastError();
    return ok;
  }
  void release() {
    if (h_in) cudaFreeHost(h_in);
    if (h_res) cudaFreeHost(h_res);
    if (d_in) cudaFree(d_in);
    if (d_res) cudaFree(d_res);
    h_in = nullptr; h_res = nullptr; h_in_dev = nullptr;
    d_in = d_res = nullptr;
    cap_in = cap_req = 0;
  }
};

struct Wave {
  std::vector<std::shared_ptr<Item>> items;
  int stream = 0, buf = 0;
};

// Best-fit allocator over [0, cap) with coalescing: free ranges indexed by
// offset (for merging with neighbours) and by size (O(log n) allocation; a
// linear first-fit scan slowed admission once completions out of order had
// split the arena into thousands of pieces).
class RangeAlloc {
 public:
  explicit RangeAlloc(uint64_t cap) { if (cap) put(0, cap); }
  bool alloc(uint64_t n, uint64_t* off) {
    if (n == 0) { *off = 0; return true; }
    const uint64_t need = (n + 15) & ~15ull;
    auto it = by_size_.lower_bound(need);
    if (it == by_size_.end()) return false;
    const uint64_t at = it->second, sz = it->first;
    by_size_.erase(it);
    by_off_.erase(at);
    if (sz > need) put(at + need, sz - need);
    *off = at;
    return true;
  }
  void release(uint64_t off, uint64_t n) {
    if (n == 0) return;
    uint64_t at = off, sz = (n + 15) & ~15ull;
    auto nx = by_off_.lower_bound(at);
    if (nx != by_off_.end() && at + sz == nx->first) {   // merge the following free range
      sz += nx->second;
      drop(nx);
    }
    auto pv = by_off_.lower_bound(at);
    if (pv != by_off_.begin()) {
      --pv;
      if (pv->first + pv->second == at) {                 // merge the preceding free range
        at = pv->first;
        sz += pv->second;
        drop(pv);
      }
    }
    put(at, sz);
  }

 private:
  std::map<uint64_t, uint64_t> by_off_;        // offset -> size
  std::multimap<uint64_t, uint64_t> by_size_;  // size -> offset
  void put(uint64_t at, uint64_t sz) {
    by_off_[at] = sz;
    by_size_.emplace(sz, at);
  }
  void drop(std::map<uint64_t, uint64_t>::iterator it) {
    auto r = by_size_.equal_range(it->second);
    for (auto k = r.first; k != r.second; ++k)
      if (k->second == it->first) { by_size_.erase(k); break; }
    by_off_.erase(it);
  }
};

}  // namespace

struct cvd_server {
  std::vector<cvd_guest*> guests;
  uint8_t* stg;
  uint64_t stg_bytes;
  uint32_t max_batch, max_inflight;
  bool auto_release = false;
  int device;
  int nstreams = 1;                                   // 1, or 2 with CVD_SERVER_TWO_STREAMS
  cudaStream_t streams[2] = {nullptr, nullptr};
  Clock::time_point epoch;

  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<std::shared_ptr<Item>> waiting;          // submitted, sorted by arrival
  std::deque<std::shared_ptr<Item>> ready[2];         // admitted, not launched
  std::deque<std::unique_ptr<Wave>> flying[2];        // launched, not complete
  static constexpr int kWaveBufs = 3;                 // waves in flight per stream
  WaveBuf bufs[2][kWaveBufs];
  std::deque<cvd_server_done> completed;
  std::map<uint64_t, std::pair<uint64_t, uint64_t>> held;   // ticket -> staging range (copy-from)
  RangeAlloc alloc{0};
  uint32_t admitted_inflight = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  int error = CVD_OK;
  std::thread sched[2], completer;
  std::vector<std::pair<uint64_t, uint64_t>> free_scratch;   // the completion thread's

  uint64_t now_ns() const {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - epoch).count();
  }

  void admit_one(uint64_t off, uint64_t now) {
    auto& it = waiting.front();
    it->stg_off = off;
    it->admit_ns = now;
    admitted_inflight++;
    ready[it->guest % nstreams].push_back(it);
    waiting.pop_front();
  }

  // Admit from the head of `waiting` while the rules allow (mu held).  The
  // due requests within the in-flight limit are taken in groups whose
  // staging is one range of the allocator, cut in arrival order (one
  // allocation per group instead of per request); a group that does not fit
  // is admitted request by request until one does not.
  static constexpr size_t kAdmitGroup = 256;
  void admit_locked() {
    const uint64_t now = now_ns();
    while (!waiting.empty()) {
      size_t k = 0;
      uint64_t total = 0;
      for (auto q = waiting.begin(); q != waiting.end() && k < kAdmitGroup; ++q, ++k) {
        if ((*q)->arrival_ns > now || admitted_inflight + k >= max_inflight) break;
        total += ((*q)->len + 15) & ~15ull;
      }
      if (k == 0) return;
      uint64_t base;
      if (k > 1 && total && alloc.alloc(total, &base)) {
        for (size_t j = 0; j < k; j++) {
          const uint64_t len = waiting.front()->len;
          admit_one(len ? base : 0, now);
          base += (len + 15) & ~15ull;
        }
        continue;
      }
      for (size_t j = 0; j < k; j++) {
        uint64_t off;
        if (!alloc.alloc(waiting.front()->len, &off)) return;
        admit_one(off, now);
      }
    }
  }

  void set_error(int e) {
    std::lock_guard<std::mutex> lk(mu);
    if (error == CVD_OK) error = e;
    stop = true;
    cv_sched.notify_all();
    cv_done.notify_all();
  }

  void scheduler(int s) {
    cudaSetDevice(device);
    for (;;) {
      std::vector<std::shared_ptr<Item>> batch;
      int bi = -1;
      {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
          if (stop) return;
          admit_locked();
          bi = -1;
          for (int k = 0; k < kWaveBufs && bi < 0; k++)
            if (!bufs[s][k].busy) bi = k;
          if (!ready[s].empty() && bi >= 0) break;
          // wake at the next arrival or when something changes (bounded)
          uint64_t wait_us = 200;
          if (!waiting.empty()) {
            uint64_t now = now_ns(), a = waiting.front()->arrival_ns;
            wait_us = a > now ? std::min<uint64_t>(wait_us, (a - now) / 1000 + 1) : 20;
          }
          cv_sched.wait_for(lk, std::chrono::microseconds(wait_us));
        }
        while (!ready[s].empty() && batch.size() < max_batch) {
          batch.push_back(ready[s].front());
          ready[s].pop_front();
        }
        bufs[s][bi].busy = true;
      }
      WaveBuf& B = bufs[s][bi];
      size_t nseg = 0, npieces = 0;
      for (size_t i = 0; i < batch.size(); i++) {   // the items were made by other threads: fetch ahead
        if (i + 8 < batch.size()) __builtin_prefetch(batch[i + 8].get());
        const Item& it = *batch[i];
        __builtin_prefetch(it.segs.data());
        nseg += it.segs.size();
        if (it.dir == 1) npieces += (it.len + kRunPiece - 1) / kRunPiece;
      }
      if (!B.reserve(std::max<size_t>(max_batch, batch.size()), std::max<size_t>(nseg, 64 * (size_t)max_batch),
                     std::max<size_t>(npieces, 4 * (size_t)max_batch))) {
        set_error(CVD_ENOMEM);
        return;
      }
      // every wave names all the server's guests in the same order, so the
      // library's device copy of the guest list never changes
      size_t off_seg, off_runs, in_bytes;
      WaveBuf::layout(batch.size(), nseg, npieces, &off_seg, &off_runs, &in_bytes);
      cvd_req* h_req = reinterpret_cast<cvd_req*>(B.h_in);
      cvd_seg* h_seg = reinterpret_cast<cvd_seg*>(B.h_in + off_seg);
      Run* h_runs = reinterpret_cast<Run*>(B.h_in + off_runs);
      size_t ns = 0, nruns = 0;
      bool no_long = true;   // no segment spans over kLongPages pages
      for (size_t i = 0; i < batch.size(); i++) {
        auto& it = batch[i];
        for (const cvd_seg& sg : it->segs)
          if (sg.len && (sg.gva + sg.len < sg.gva || ((sg.gva + sg.len - 1) >> 12) - (sg.gva >> 12) + 1 > kLongPages))
            no_long = false;
        cvd_req q;
        q.seg_begin = (uint32_t)ns;
        q.seg_count = (uint32_t)it->segs.size();
        q.dir = it->dir;
        q.guest = it->guest;
        q.host_off = it->stg_off;
        h_req[i] = q;
        memcpy(h_seg + ns, it->segs.data(), it->segs.size() * sizeof(cvd_seg));
        ns += it->segs.size();
        for (uint64_t o = 0; it->dir == 1 && o < it->len; o += kRunPiece) {   // gather, in warp-sized pieces
          Run r;
          r.dst = (uint64_t)(uintptr_t)(stg + it->stg_off + o);
          r.src = it->src + o;
          r.len = it->len - o < kRunPiece ? it->len - o : kRunPiece;
          r.pad = 0;
          h_runs[nruns++] = r;
        }
      }
      cudaStream_t st = streams[s];
      size_t nr = batch.size();
      unsigned char* d_in = static_cast<unsigned char*>(B.d_in);
      const cvd_req* d_req = reinterpret_cast<const cvd_req*>(d_in);
      const cvd_seg* d_seg = reinterpret_cast<const cvd_seg*>(d_in + off_seg);
      // one launch reads the requests and segments into d_in and gathers the
      // copy-to sources into staging, both straight from the pinned block
      const size_t up = ns ? off_seg + ns * sizeof(cvd_seg) : nr * sizeof(cvd_req);
      bool ok = cudaEventRecord(B.start, st) == cudaSuccess;
      ok = ok && launch_wave_in(B.h_in_dev, d_in, (up + 15) / 16, reinterpret_cast<const Run*>(B.h_in_dev + off_runs),
                               nruns, st) == cudaSuccess;
      uint64_t t_launch = now_ns();
      for (auto& it : batch) it->launch_ns = t_launch;
      // levelled (guest g's requests take effect in arrival order); the
      // staging allocator gives disjoint ranges, so only guest memory is
      // checked for conflicts
      int rc = ok ? copy_batch_staging_disjoint(guests.data(), (uint32_t)guests.size(), d_req, (uint32_t)nr,
                                                d_seg, ns, stg, stg_bytes, (cvd_result*)B.d_res, no_long, st)
                  : CVD_ECUDA;
      if (rc == CVD_OK &&
          cudaMemcpyAsync(B.h_res, B.d_res, nr * sizeof(cvd_result), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = CVD_ECUDA;
      if (rc == CVD_OK && cudaEventRecord(B.done, st) != cudaSuccess) rc = CVD_ECUDA;
      if (rc != CVD_OK) {
        set_error(rc);
        return;
      }
      std::unique_ptr<Wave> w(new Wave());
      w->stream = s;
      w->buf = bi;
      w->items = std::move(batch);
      {
        std::lock_guard<std::mutex> lk(mu);
        flying[s].push_back(std::move(w));
      }
      cv_done.notify_all();
    }
  }

  void completion_loop() {
    cudaSetDevice(device);
    for (;;) {
      Wave* w = nullptr;
      int s = -1;
      {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
          if (stop && flying[0].empty() && flying[1].empty()) return;
          // The oldest wave of each stream; only this thread removes waves,
          // so they stay valid while the lock is released for the queries
          // (an event query can wait inside the driver while a scheduler
          // synchronises its stream, and must not hold the schedulers off).
          Wave* front[2] = {nullptr, nullptr};
          cudaEvent_t ev[2] = {nullptr, nullptr};
          for (int k = 0; k < 2; k++)
            if (!flying[k].empty()) {
              front[k] = flying[k].front().get();
              ev[k] = bufs[k][front[k]->buf].done;
            }
          cudaError_t q[2] = {cudaErrorNotReady, cudaErrorNotReady};
          if (front[0] || front[1]) {
            lk.unlock();
            for (int k = 0; k < 2; k++)
              if (front[k]) q[k] = cudaEventQuery(ev[k]);
            lk.lock();
          }
          for (int k = 0; k < 2 && !w; k++) {
            if (!front[k]) continue;
            if (q[k] == cudaSuccess) { w = front[k]; s = k; }
            else if (q[k] != cudaErrorNotReady) {
              cudaGetLastError();
              if (error == CVD_OK) error = CVD_ECUDA;
              stop = true;
              flying[k].clear();   // abandon: the stream is broken
            }
          }
          if (w) break;
          cv_done.wait_for(lk, std::chrono::microseconds(10));
        }
      }
      uint64_t t_done = now_ns();
      uint64_t wave_ns = 0;
      {
        float ms = 0;   // both events have completed
        if (cudaEventElapsedTime(&ms, bufs[s][w->buf].start, bufs[s][w->buf].done) == cudaSuccess)
          wave_ns = (uint64_t)(ms * 1e6);
        else
          cudaGetLastError();
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        WaveBuf& B = bufs[s][w->buf];
        std::vector<std::pair<uint64_t, uint64_t>>& fr = free_scratch;   // staging ranges to give back
        fr.clear();
        for (size_t i = 0; i < w->items.size(); i++) {
          auto& it = w->items[i];
          cvd_server_done d;
          memset(&d, 0, sizeof(d));
          d.ticket = it->ticket;
          d.tag = it->tag;
          d.res = B.h_res[i];
          d.staging_off = it->stg_off;
          d.len = it->len;
          d.arrival_ns = it->arrival_ns;
          d.admit_ns = it->admit_ns;
          d.launch_ns = it->launch_ns;
          d.complete_ns = t_done;
          d.guest = it->guest;
          d.dir = it->dir;
          d.wave_device_ns = wave_ns;
          completed.push_back(d);
          admitted_inflight--;
          if (it->dir == 0 && it->len && !auto_release) held[it->ticket] = {it->stg_off, it->len};
          else if (it->len) fr.emplace_back(it->stg_off, (it->len + 15) & ~15ull);
        }
        // a wave's requests were mostly admitted together: give their ranges
        // back merged
        std::sort(fr.begin(), fr.end());
        for (size_t i = 0; i < fr.size();) {
          uint64_t off = fr[i].first, len = fr[i].second;
          for (i++; i < fr.size() && fr[i].first == off + len; i++) len += fr[i].second;
          alloc.release(off, len);
        }
        B.busy = false;
        flying[s].pop_front();
        admit_locked();   // the freed staging and slots go to waiting requests here, off the schedulers' path
      }
      cv_sched.notify_all();
      cv_done.notify_all();
    }
  }
};

extern "C" {

int cvd_server_create(cvd_guest* const* guests, uint32_t nguests, void* d_staging, uint64_t staging_bytes,
                      uint32_t max_batch, uint32_t max_inflight, uint32_t flags, cvd_server** out) {
  if (!guests || nguests == 0 || nguests > CVD_MAX_GUESTS_PER_BATCH || !d_staging || staging_bytes == 0 || !out ||
      max_batch == 0 || max_inflight == 0 || (flags & ~(CVD_SERVER_AUTO_RELEASE | CVD_SERVER_TWO_STREAMS)))
    return CVD_EINVAL;
  for (uint32_t i = 0; i < nguests; i++)
    if (!guests[i]) return CVD_EINVAL;
  std::unique_ptr<cvd_server> s(new cvd_server());
  s->guests.assign(guests, guests + nguests);
  s->stg = reinterpret_cast<uint8_t*>(d_staging);
  s->stg_bytes = staging_bytes;
  s->max_batch = max_batch;
  s->max_inflight = max_inflight;
  s->auto_release = (flags & CVD_SERVER_AUTO_RELEASE) != 0;
  s->nstreams = (flags & CVD_SERVER_TWO_STREAMS) ? 2 : 1;
  s->alloc = RangeAlloc(staging_bytes);
  cudaGetDevice(&s->device);
  prepare_kernels();
  auto undo = [&](int rc) {   // a failed create leaves nothing allocated
    for (int k = 0; k < 2; k++) {
      if (s->streams[k]) cudaStreamDestroy(s->streams[k]);
      for (int b = 0; b < cvd_server::kWaveBufs; b++) {
        s->bufs[k][b].release();
        if (s->bufs[k][b].done) cudaEventDestroy(s->bufs[k][b].done);
        if (s->bufs[k][b].start) cudaEventDestroy(s->bufs[k][b].start);
      }
    }
    return rc;
  };
  for (int k = 0; k < s->nstreams; k++)
    if (cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      s->streams[k] = nullptr;
      return undo(CVD_ECUDA);
    }
  // descriptor buffers are reserved up front so waves never allocate
  for (int k = 0; k < s->nstreams; k++)
    for (int b = 0; b < cvd_server::kWaveBufs; b++)
      if (!s->bufs[k][b].reserve(max_batch, 64 * (size_t)max_batch, 4 * (size_t)max_batch)) return undo(CVD_ENOMEM);
  s->epoch = Clock::now();
  cvd_server* raw = s.get();
  for (int k = 0; k < raw->nstreams; k++) raw->sched[k] = std::thread([raw, k] { raw->scheduler(k); });
  raw->completer = std::thread([raw] { raw->completion_loop(); });
  *out = s.release();
  return CVD_OK;
}

uint64_t cvd_server_now_ns(cvd_server* s) { return s ? s->now_ns() : 0; }

int cvd_server_submit(cvd_server* s, const cvd_server_req* reqs, uint32_t n, uint64_t* tickets) {
  if (!s || (n && !reqs)) return CVD_EINVAL;
  std::vector<std::shared_ptr<Item>> items;
  items.reserve(n);
  for (uint32_t i = 0; i < n; i++) {
    const cvd_server_req& r = reqs[i];
    if (r.guest >= s->guests.size() || r.dir > 1 || (r.nseg && !r.segs)) return CVD_EINVAL;
    auto it = std::make_shared<Item>();
    it->tag = r.tag;
    it->guest = r.guest;
    it->dir = r.dir;
    it->segs.assign(r.segs, r.segs + r.nseg);
    uint64_t L = 0;
    for (auto& sg : it->segs) {
      if (sg.len > s->stg_bytes || L + sg.len > s->stg_bytes) return CVD_EINVAL;   // could never be admitted
      L += sg.len;
    }
    if (r.dir == 1 && L && !r.d_src) return CVD_EINVAL;
    it->len = L;
    it->src = (uint64_t)(uintptr_t)r.d_src;
    it->arrival_ns = r.arrival_ns;
    items.push_back(it);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error) return s->error;
    for (uint32_t i = 0; i < n; i++) {
      items[i]->ticket = s->next_ticket++;
      if (tickets) tickets[i] = items[i]->ticket;
      // keep `waiting` sorted by arrival (stable for equal times)
      auto pos = std::upper_bound(s->waiting.begin(), s->waiting.end(), items[i],
                                  [](const std::shared_ptr<Item>& a, const std::shared_ptr<Item>& b) {
                                    return a->arrival_ns < b->arrival_ns;
                                  });
      s->waiting.insert(pos, items[i]);
    }
  }
  s->cv_sched.notify_all();
  return CVD_OK;
}

int cvd_server_poll(cvd_server* s, cvd_server_done* out, uint32_t max, uint32_t* n_out, uint32_t timeout_us) {
  if (!s || !n_out || (max && !out)) return CVD_EINVAL;
  *n_out = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  auto deadline = Clock::now() + std::chrono::microseconds(timeout_us);
  while (s->completed.empty()) {
    if (s->error) return s->error;
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && s->completed.empty())
      return timeout_us ? CVD_ETIMEDOUT : CVD_OK;
  }
  uint32_t k = 0;
  while (k < max && !s->completed.empty()) {
    out[k++] = s->completed.front();
    s->completed.pop_front();
  }
  *n_out = k;
  return CVD_OK;
}

int cvd_server_release(cvd_server* s, uint64_t ticket) {
  if (!s) return CVD_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->held.find(ticket);
  if (it == s->held.end()) return CVD_EINVAL;
  s->alloc.release(it->second.first, it->second.second);
  s->held.erase(it);
  s->cv_sched.notify_all();
  return CVD_OK;
}

int cvd_server_destroy(cvd_server* s) {
  if (!s) return CVD_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_all();
  s->cv_done.notify_all();
  for (int k = 0; k < 2; k++)
    if (s->sched[k].joinable()) s->sched[k].join();
  if (s->completer.joinable()) s->completer.join();
  for (int k = 0; k < 2; k++) {
    if (s->streams[k]) {
      cudaStreamSynchronize(s->streams[k]);
      cudaStreamDestroy(s->streams[k]);
    }
    for (int b = 0; b < cvd_server::kWaveBufs; b++) {
      s->bufs[k][b].release();
      if (s->bufs[k][b].done) cudaEventDestroy(s->bufs[k][b].done);
      if (s->bufs[k][b].start) cudaEventDestroy(s->bufs[k][b].start);
    }
  }
  int rc = s->error;
  delete s;
  return rc == CVD_ETIMEDOUT ? CVD_OK : rc;
}

}  // extern "C"
