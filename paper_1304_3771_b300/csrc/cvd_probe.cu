// cvd_probe.cu -- dependent-load latency probe (pointer chase), translate
// launch shape, and the self-test of the bounded-wait failure path.
//
// Not a step of the paper's method: it measures the two latencies that bound
// the software page walk (Sec. 4.2) on this GPU -- an L2 hit and a DRAM access
// -- so that walk throughput can be stated against a latency roofline
// (resident lanes x walks in flight per lane / dependent latency of one walk).
//
// The buffer is cut into 128-byte slots; slot i holds the byte offset of slot
// (a*i + c) mod N (N a power of two, a = 1 mod 4, c odd: one cycle through all
// N slots by the Hull-Dobell theorem, with consecutive slots far apart).  One
// thread follows the chain with L1-bypassing loads, each address depending on
// the previous load, and the global timer brackets the timed steps.
#include <cstdint>

#include "../../include/cvd.h"
#include "cvd_internal.h"
#include "cvd_mbar.cuh"

namespace {

constexpr uint64_t kSlot = 128;                              // bytes per chain slot
constexpr uint64_t kMulA = 6364136223846793005ull;           // = 1 (mod 4)
constexpr uint64_t kAddC = 1442695040888963407ull;           // odd

__global__ void k_chain_init(uint64_t* buf, uint64_t nslots) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nslots; i += stride)
    buf[i * (kSlot / 8)] = ((kMulA * i + kAddC) & (nslots - 1)) * kSlot;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void k_chase(const uint64_t* buf, uint32_t warm, uint32_t steps, unsigned long long* out) {
  const uint8_t* b = reinterpret_cast<const uint8_t*>(buf);
  uint64_t off = 0;
  for (uint32_t s = 0; s < warm; s++) off = __ldcg(reinterpret_cast<const unsigned long long*>(b + off));
  const uint64_t t0 = global_ns();
  for (uint32_t s = 0; s < steps; s++) off = __ldcg(reinterpret_cast<const unsigned long long*>(b + off));
  const uint64_t t1 = global_ns();
  out[0] = t1 - t0;
  out[1] = off;   // keeps the chain live
}

}  // namespace

namespace cvd {

// Self-test of the wait-failure path: one warp waits on an mbarrier phase that
// needs two arrivals and gets one, gives up after `tries` attempts and reports
// through the device error word exactly as the copy engine does.  No copy is
// issued, so nothing is left in flight when the block exits.
__global__ void k_wait_selftest(unsigned int* err, uint32_t tries) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 2);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncwarp();
  if (threadIdx.x == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&bar)) : "memory");
  __syncwarp();
  const bool ok = mbar_wait_bounded(&bar, 0, tries);
  if (!ok && threadIdx.x == 0) atomicOr(err, kErrWaitTimeout);
}

cudaError_t launch_wait_selftest(unsigned int* err, uint32_t tries, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(err, tries);
  g_launches++;
  return cudaGetLastError();
}

}  // namespace cvd

extern "C" int cvd_probe_latency(void* d_buf, uint64_t bytes, uint32_t steps, cvd_stream_t stream,
                                 double* ns_per_load) {
  if (!d_buf || !ns_per_load || steps == 0 || ((uintptr_t)d_buf & 127)) return CVD_EINVAL;
  uint64_t nslots = bytes / kSlot;
  if (nslots < 2) return CVD_EINVAL;
  while (nslots & (nslots - 1)) nslots &= nslots - 1;   // largest power of two that fits
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long* d_out = nullptr;
  if (cudaMalloc(&d_out, 16) != cudaSuccess) {
    cudaGetLastError();
    return CVD_ENOMEM;
  }
  int rc = CVD_OK;
  const unsigned blocks = (unsigned)cvd::num_sms() * 4;
  k_chain_init<<<blocks, 256, 0, st>>>(reinterpret_cast<uint64_t*>(d_buf), nslots);
  // warm-up: one pass over up to 2^20 slots touches the chain (TLB, L2 for small buffers)
  const uint32_t warm = nslots < (1u << 20) ? (uint32_t)nslots : (1u << 20);
  k_chase<<<1, 1, 0, st>>>(reinterpret_cast<const uint64_t*>(d_buf), warm, steps, d_out);
  cvd::g_launches += 2;
  unsigned long long h[2] = {0, 0};
  if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(h, d_out, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    rc = CVD_ECUDA;
  } else {
    *ns_per_load = (double)h[0] / (double)steps;
  }
  cudaFree(d_out);
  return rc;
}

extern "C" int cvd_translate_shape(const cvd_guest* g, uint32_t* resident_threads_per_sm, uint32_t* walks_per_thread) {
  if (!resident_threads_per_sm || !walks_per_thread) return CVD_EINVAL;
  cvd::prepare_kernels();
  cvd::translate_shape(g ? cvd::walk_selector(g->host) : cvd::kPagingX86_64, g ? g->host.paging : cvd::kPagingX86_64,
                       g ? g->host.nunits : 0, resident_threads_per_sm, walks_per_thread);
  return *resident_threads_per_sm ? CVD_OK : CVD_ECUDA;
}
