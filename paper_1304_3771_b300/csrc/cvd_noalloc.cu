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
//
// Layout of the fixed array: a 256-byte control block (the call's device
// error word at offset 0, the guest-pointer slot the planner reads at offset
// 8), then the work arrays of one call.  The error word is zeroed when the
// array is set up on a device and whenever cvd_stream_check takes it; in
// between the calls' bits accumulate, so a report is never lost to a later
// call.  Everything a call needs zeroed is zeroed by its own kernels.
#include <cstring>
#include <mutex>

#include "../../include/cvd.h"
#include "cvd_internal.h"

using namespace cvd;

namespace {

// 16 MiB, held by every GPU that loads the library until the process exits.
constexpr size_t kScratchBytes = (size_t)CVD_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr size_t kCtlBytes = 256;      // control block at the front of the array
constexpr size_t kCtlErr = 0;          // u32 device error word (kErr* bits)
constexpr size_t kCtlGuest = 8;        // const DevGuest* the planner and copy engine read

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  The array's
// name is only a host-side stand-in, so the address is looked up once per
// device, with that device current; the control block is zeroed then, in
// stream order on `st`.
cudaError_t scratch_for_current_device(cudaStream_t st, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    e = cudaMemsetAsync(p, 0, kCtlBytes, st);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

size_t round_up(size_t n) { return (n + 255) & ~(size_t)255; }

// Long-segment list entries in the fixed scratch (more: walked inline by the
// request's own planner warp, with the same results).
constexpr uint64_t kNoallocLongItems = 4096;

// Bytes of scratch a call with nreq requests and nseg segments needs, in the
// order the call carves them.
size_t scratch_need(uint64_t nreq, uint64_t nseg) {
  const uint64_t r = nreq ? nreq : 1, s = nseg ? nseg : 1;
  return kCtlBytes + 2 * round_up(16 * (nreq + 1)) + round_up(16 * scan_tmp_elems(nreq)) +
         round_up(sizeof(ReqWork) * r) + round_up(8 * r) + round_up(4 * r) +
         round_up(sizeof(LongItem) * kNoallocLongItems) + round_up(sizeof(SegWork) * s) + round_up(32);
}

__global__ void k_store_ptr(const DevGuest** slot, const DevGuest* g) { *slot = g; }

}  // namespace

cudaError_t cvd::noalloc_take_errors(cudaStream_t st, unsigned int* bits) {
  *bits = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaSuccess;
  void* p = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    p = g_scratch_ptr[dev];
  }
  if (!p) return cudaSuccess;   // the call never ran on this device
  unsigned char* w = reinterpret_cast<unsigned char*>(p) + kCtlErr;
  e = cudaMemcpyAsync(bits, w, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w, 0, 4, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

extern "C" int cvd_copy_batch_noalloc(cvd_guest* g, const cvd_req* d_req, uint32_t nreq, const cvd_seg* d_seg,
                                      uint64_t nseg, void* d_host_buf, uint64_t host_buf_bytes, cvd_result* d_res,
                                      cvd_stream_t stream) {
  if (!g) return CVD_EINVAL;
  cvd_guest* gl[1] = {g};
  int v = check_batch_args(gl, 1, d_req, nreq, d_seg, nseg, d_host_buf, host_buf_bytes, d_res);
  if (v) return v;
  if (nreq > CVD_NOALLOC_MAX_REQS || nseg > CVD_NOALLOC_MAX_SEGS) return CVD_E2BIG;
  if (scratch_need(nreq, nseg) > kScratchBytes) return CVD_E2BIG;
  if (nreq == 0) return CVD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  void* base = nullptr;
  cudaError_t e = scratch_for_current_device(st, &base);
  if (e != cudaSuccess) return fail_cuda(e);
  prepare_kernels();
  unsigned char* ctl = reinterpret_cast<unsigned char*>(base);
  unsigned char* b = ctl + kCtlBytes;
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
  // [0] copy windows (zeroed by the copy launch), [1] planner requests and
  // [2] long-segment list length (zeroed by the request-sizing kernel)
  a.counter = reinterpret_cast<unsigned long long*>(take(32));
  const DevGuest** slot = reinterpret_cast<const DevGuest**>(ctl + kCtlGuest);
  a.err = reinterpret_cast<unsigned int*>(ctl + kCtlErr);
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
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_plan(a, st);
  if (e == cudaSuccess) e = launch_copy(a, p, st);
  if (e != cudaSuccess) return fail_cuda(e);
  return CVD_OK;
}
