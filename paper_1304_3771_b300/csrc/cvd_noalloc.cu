// cvd_noalloc.cu -- cvd_copy_batch_noalloc: the hazard-free single-guest
// batch (planner + persistent copy engine) with its scratch in a fixed
// device array that the library reserves when it is loaded, so the call
// itself allocates nothing.
//
// Who needs it: callers that must not allocate device memory on the request
// path.  cudaMalloc and cudaFree synchronise the whole device, which stalls
// every other stream of a latency-bound request loop; and a process whose
// device memory is already taken by another allocator (a framework's caching
// allocator, for instance) can see a late cudaMalloc fail.  The regular
// batch calls grow per-stream scratch with cudaMalloc on first use and
// whenever a larger batch arrives; this entry point never does.
#include <cstring>
#include <mutex>

#include "../../include/cvd.h"
#include "cvd_internal.h"

using namespace cvd;

namespace {

// 16 MiB, held by every GPU that loads the library until the process exits.
constexpr size_t kScratchBytes = (size_t)CVD_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  The array's
// name is only a host-side stand-in, so the address is looked up once per
// device, with that device current.
int scratch_for_current_device(void** out, int* err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { *err = (int)e; return CVD_ECUDA; }
  if (dev < 0 || dev >= kMaxDevices) return CVD_EINVAL;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) { cudaGetLastError(); *err = (int)e; return CVD_ECUDA; }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return CVD_OK;
}

size_t round_up(size_t n) { return (n + 255) & ~(size_t)255; }

// Long-segment list entries in the fixed scratch (more: walked inline).
constexpr uint64_t kNoallocLongItems = 4096;

// Bytes of scratch a call with nreq requests and nseg segments needs.
size_t scratch_need(uint64_t nreq, uint64_t nseg) {
  size_t pairs = round_up(16 * (nreq + 1));
  return 2 * pairs + round_up(16 * scan_tmp_elems(nreq)) + round_up(sizeof(ReqWork) * (nreq ? nreq : 1)) +
         round_up(sizeof(SegWork) * (nseg ? nseg : 1)) + round_up(8 * (nreq ? nreq : 1)) + round_up(4 * (nreq ? nreq : 1)) +
         round_up(sizeof(LongItem) * kNoallocLongItems) + round_up(16) + round_up(8) + round_up(8);
}

__global__ void k_store_ptr(const DevGuest** slot, const DevGuest* g) { *slot = g; }

}  // namespace

extern "C" int cvd_copy_batch_noalloc(cvd_guest* g, const cvd_req* d_req, uint32_t nreq, const cvd_seg* d_seg,
                                      uint64_t nseg, void* d_host_buf, uint64_t host_buf_bytes, cvd_result* d_res,
                                      cvd_stream_t stream) {
  if (!g) return CVD_EINVAL;
  if (nreq && (!d_req || !d_res)) return CVD_EINVAL;
  if (nseg && !d_seg) return CVD_EINVAL;
  if (host_buf_bytes && !d_host_buf) return CVD_EINVAL;
  if (host_buf_bytes >= (1ull << 52)) return CVD_EINVAL;   // fault keys hold request offsets in 52 bits
  if (nreq > CVD_NOALLOC_MAX_REQS || nseg > CVD_NOALLOC_MAX_SEGS) return CVD_E2BIG;
  if (scratch_need(nreq, nseg) > kScratchBytes) return CVD_E2BIG;
  int dev = 0;
  cudaGetDevice(&dev);
  if (g->device != dev) return CVD_EINVAL;
  uint64_t p0 = (uint64_t)(uintptr_t)g->host.pool, s0 = (uint64_t)(uintptr_t)d_host_buf;
  if (d_host_buf && host_buf_bytes && p0 < s0 + host_buf_bytes && s0 < p0 + g->host.pool_bytes) return CVD_EINVAL;
  if (nreq == 0) return CVD_OK;
  void* base = nullptr;
  int err = 0;
  int rc = scratch_for_current_device(&base, &err);
  if (rc) return rc;
  prepare_kernels();
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* b = reinterpret_cast<unsigned char*>(base);
  auto take = [&](size_t n) { unsigned char* r = b; b += round_up(n); return r; };
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.req = reinterpret_cast<const Req*>(d_req);
  a.nreq = nreq;
  a.seg = reinterpret_cast<const Seg*>(d_seg);
  a.nseg = nseg;
  a.pairs_in = reinterpret_cast<uint64_t*>(take(16 * ((size_t)nreq + 1)));
  a.pairs_out = reinterpret_cast<uint64_t*>(take(16 * ((size_t)nreq + 1)));
  a.scan_tmp = reinterpret_cast<uint64_t*>(take(16 * scan_tmp_elems(nreq)));
  a.rw = reinterpret_cast<ReqWork*>(take(sizeof(ReqWork) * nreq));
  a.fkey = reinterpret_cast<unsigned long long*>(take(8 * (size_t)nreq));
  a.lcount = reinterpret_cast<unsigned int*>(take(4 * (size_t)nreq));
  a.long_items = reinterpret_cast<LongItem*>(take(sizeof(LongItem) * kNoallocLongItems));
  a.long_cap = kNoallocLongItems;
  a.sw = reinterpret_cast<SegWork*>(take(sizeof(SegWork) * (nseg ? nseg : 1)));
  a.counter = reinterpret_cast<unsigned long long*>(take(32));  // [0] copy windows (zeroed by the copy launch), [1] planner requests, [2] long-segment list
  const DevGuest** slot = reinterpret_cast<const DevGuest**>(take(8));
  a.err = reinterpret_cast<unsigned int*>(take(8));                 // private error word
  a.guests = slot;
  a.nguests = 1;
  a.single = g->dev;
  a.single_paging = walk_selector(g->host);
  a.dir_override = -1;
  a.stg = reinterpret_cast<uint8_t*>(d_host_buf);
  a.stg_bytes = host_buf_bytes;
  a.res = reinterpret_cast<Result*>(d_res);
  k_store_ptr<<<1, 1, 0, st>>>(slot, g->dev);
  g_launches++;
  CopyParams p;   // the library's defaults; cvd_set_copy_params does not apply here
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_plan(a, st);
  if (e == cudaSuccess) e = launch_copy(a, p, st);
  if (e != cudaSuccess) { cudaGetLastError(); return CVD_ECUDA; }
  return CVD_OK;
}
