// cvd_internal.h -- host-side declarations shared by the library's .cu files.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/cvd.h"
#include "cvd_device.cuh"

namespace cvd {

// One copy run of the levelled engine: dst <- src (src == 0: zero fill).
struct Run { uint64_t dst, src, len, pad; };
// Longest run one warp copies; longer runs are emitted as several.
constexpr uint64_t kRunPiece = 16384;

struct CopyParams {
  uint32_t vec_bytes = 16;
  uint32_t unroll = 4;
  uint32_t chunk_bytes = 256 << 10;
  uint32_t blocks_per_sm = 1;
  uint32_t warps_per_block = 16;
  uint32_t small_bytes = 256;
  uint32_t engine = 1;             // 0: register realign, 1: bulk-copy (TMA) staging ring
  uint32_t stages = 8;             // engine 1: pieces in flight per warp (descriptor slots, <= 32)
  uint32_t stage_bytes = 4096;     // engine 1: largest piece (destination bytes)
  uint32_t ring_bytes = 8320;      // engine 1: shared-memory byte ring per warp (two misaligned 4 KiB pieces)
};

// Work-balancing weight of one request in the scanned stream positions:
// request r occupies [R_r, R_r + kReqWeight + L_r), its bytes the last L_r of
// them.  A request costs a warp a few dependent loads whatever its size, so
// byte-balanced chunks would pile thousands of tiny requests onto one warp.
constexpr uint64_t kReqWeight = 4096;

// One block of pages of a long segment, walked by k_long_scan.
struct LongItem { uint32_t req, seg, page0, npages; };
constexpr uint32_t kLongBlock = 256;   // pages per LongItem
constexpr uint32_t kLongPages = 1024;  // segments spanning more pages are walked through the long-segment list

// Device error word bits (set by kernels, read by cvd_stream_check).
constexpr unsigned kErrWaitTimeout = 1u;   // a bounded mbarrier wait gave up

// Compiled walk of a launch: for one memslot guest kPagingX86_64 /
// kPagingPae (its format); kWalkEpt when a guest of the launch is behind an
// EPT (format and second dimension read per walk); 0 for several memslot
// guests (format read per walk).
constexpr uint32_t kWalkEpt = 2;
inline uint32_t walk_selector(const DevGuest& h) { return h.ept ? kWalkEpt : h.paging; }

// Arguments common to the planner and the copy engines.
struct BatchArgs {
  const Req* req;
  uint32_t nreq;
  const Seg* seg;
  uint64_t nseg;
  const DevGuest* const* guests;   // device array [nguests]
  uint32_t nguests;
  const DevGuest* single;          // == guests[0] when nguests == 1 (enables smem staging)
  uint32_t single_paging;          // walk selector of the launch (walk_selector; kWalkEpt for any EPT guest)
  int dir_override;                // -1: use req.dir and req.guest
  uint8_t* stg;                    // staging buffer (device)
  uint64_t stg_bytes;
  Result* res;
  // scratch
  uint64_t* pairs_in;              // [2*(nreq+1)]: (seg_count, L) per request
  uint64_t* pairs_out;             // exclusive scan of pairs_in, [nreq] = totals
  uint64_t* scan_tmp;              // block sums
  ReqWork* rw;                     // [nreq]
  SegWork* sw;                     // [nseg]
  unsigned long long* counter;     // [0] copy-engine window cursor, [1] fault-scan window cursor
  unsigned long long* fkey;        // [nreq] first fault per request: stream offset << 12 | code
  unsigned int* lcount;            // [nreq] blocks of the request on the long-segment list not yet walked
  LongItem* long_items;            // long-segment list, capacity long_cap (counter[2] = length)
  uint64_t long_cap;
  unsigned int* err;               // device error word (kErr* bits)
  uint32_t spare_sms;              // SMs the copy grid leaves free (for the next batch's planning)
  uint32_t no_long = 0;            // host only: no segment spans over kLongPages pages (the long-segment pass is skipped)
};

// SMs a planned-ahead copy leaves to the next batch's planning: the copy
// blocks take every register of their SM, so planning overlaps a copy only on
// SMs the copy grid leaves free.  On the 6-batch bench step (148 SMs): none
// 21.06 ms, 4 free 20.81, 8 free 20.64, 12 free 20.52, 16 free 20.63, 20 free
// 20.85 (the copy kernel 0.905 -> 0.897 of the measured peak at 12).
constexpr uint32_t kPlanAheadSms = 12;

extern unsigned long long g_launches;
int num_sms();

// Allow a kernel `bytes` of dynamic shared memory.
template <class K>
inline void allow_smem(K kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Resident blocks per SM of a kernel at its launch shape (queried once).
template <class K>
inline unsigned resident_blocks(K kernel, int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  return (unsigned)n;
}

// Sets the copy kernels' shared-memory attributes (cvd_copy.cu).
void prepare_copy_kernels();

// launchers (return the cudaError_t of the last launch)
cudaError_t launch_translate(const DevGuest* g, uint32_t sel, uint32_t paging, uint32_t nunits, const uint64_t* gva,
                             uint64_t n, bool write, uint64_t* gpa, uint64_t* hpa, uint32_t* code, cudaStream_t st);
// Resident threads per SM of the translate kernel and walks each keeps in flight.
// sel: the guest's walk selector; paging: its format; nunits: its unit-table length (0: none)
void translate_shape(uint32_t sel, uint32_t paging, uint32_t nunits, uint32_t* threads_per_sm,
                     uint32_t* walks_per_thread);
// Translation with every level above the leaf tables staged (cvd_translate.cu):
// memslot guests (4-level or PAE) with unit tables, and guests behind an EPT.
// paging: the guest's format (kPaging*).
bool translate_staged_ok(uint32_t sel, uint32_t paging, uint32_t nunits);
cudaError_t launch_translate_staged(const DevGuest* g, uint32_t sel, uint32_t paging, uint32_t nunits,
                                    const uint64_t* gva, uint64_t n, bool write, uint64_t* gpa, uint64_t* hpa,
                                    uint32_t* code, cudaStream_t st);
void translate_staged_shape(uint32_t sel, uint32_t paging, uint32_t nunits, uint32_t* threads_per_sm,
                            uint32_t* walks_per_thread);
void prepare_translate_staged();
cudaError_t launch_plan(const BatchArgs& a, cudaStream_t st);
// The plan in two parts: sizing (k_req_sizes and the pair scan) and the walk
// (k_plan, then the long-segment pass unless a.no_long); launch_plan is both.
cudaError_t launch_plan_sizes(const BatchArgs& a, cudaStream_t st);
cudaError_t launch_plan_walk(const BatchArgs& a, cudaStream_t st);
// One warp whose bounded mbarrier wait cannot complete: sets kErrWaitTimeout.
cudaError_t launch_wait_selftest(unsigned int* err, uint32_t tries, cudaStream_t st);
// counter_zeroed: a.counter[0], the work counter, was zeroed in stream order
// (the levelled calls' mark pass does it); otherwise a memset does.
cudaError_t launch_copy(const BatchArgs& a, const CopyParams& p, cudaStream_t st, bool counter_zeroed = false);
bool copy_params_supported(const CopyParams& p);
size_t copy_smem_bytes(const CopyParams& p, bool staged);
void prepare_kernels();
size_t scan_tmp_elems(uint64_t n);
cudaError_t launch_scan_pairs(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t* tmp, cudaStream_t st);
// levelled engine
// only (optional): list only the requests r with only[r] != 0.
cudaError_t launch_runs(const BatchArgs& a, bool emit, uint64_t* counts_pairs, const uint64_t* offs_pairs,
                        Run* runs, cudaStream_t st, const uint8_t* only = nullptr);
cudaError_t launch_run_copy(const Run* runs, uint64_t n, cudaStream_t st);
// A serving wave's inputs (k_wave_in): n16 16-byte words of the descriptor
// block copied from h_block (mapped pinned host memory, its device address)
// to d_block, and the nruns runs whose records h_runs (mapped, device
// address) holds.
cudaError_t launch_wave_in(const void* h_block, void* d_block, uint64_t n16, const Run* h_runs, uint64_t nruns,
                           cudaStream_t st);
// Levelled calls on the device.  Pass 1 (launch_hz_insert, after the plan's
// sizing, beside its walk) puts every guest page the requests may touch into
// the epoch-tagged hash table (keys, vals: cap slots, a power of two, zeroed
// when allocated; epoch >= 1 and < 2^24, new for every call) and marks pages
// touched with a conflict; unless the caller guarantees disjoint staging
// ranges their order is checked.  Pass 2 (launch_hz_mark, after the plan)
// sets mark[r] for every request touching a marked page (every request when
// *flag, zeroed by the sizing kernel, got bit 0 from the staging check or bit
// 1 from a full table), removes its work from the parallel launch and counts
// it in *nmarked (zeroed by the sizing kernel).
cudaError_t launch_hz_insert(const BatchArgs& a, unsigned long long* keys, unsigned long long* vals, uint64_t cap,
                             uint64_t epoch, bool staging_disjoint, unsigned int* flag, cudaStream_t st);
cudaError_t launch_hz_mark(const BatchArgs& a, const unsigned long long* keys, const unsigned long long* vals,
                           uint64_t cap, uint64_t epoch, const unsigned int* flag, uint8_t* mark, unsigned int* nmarked,
                           cudaStream_t st);
// The marked requests one after another in index order, by one block
// (cvd_copy.cu); nothing when *nmarked is 0.
cudaError_t launch_ordered_copy(const BatchArgs& a, const uint8_t* mark, const unsigned int* nmarked, cudaStream_t st);

// Library-side state of one cvd_guest handle.
}  // namespace cvd
struct cvd_guest {
  cvd::DevGuest host;   // host copy of the descriptor
  cvd::DevGuest* dev;   // device copy
  uint64_t* d_alloc;    // [pt_used, rsv_used]
  uint8_t* d_units;     // the unit tables (when host.nunits != 0): deltas, then slots
  int device;
};
namespace cvd {

// Argument checks every batch call makes before any CUDA work (cvd_capi.cu):
// guest count and device, staging buffer clear of every guest pool, pointers
// present for non-empty arrays, and the stream positions (sums of staging-
// bounded lengths plus kReqWeight per request) kept inside u64 with request
// offsets inside the fault key's 52 bits.  CVD_OK or CVD_EINVAL.
// cvd_copy_batch without flags for callers whose requests' staging ranges
// are pairwise disjoint (cvd_capi.cu; used by the serving loop).  no_long:
// the caller checked that no segment spans over kLongPages pages.
int copy_batch_staging_disjoint(cvd_guest* const* guests, uint32_t nguests, const cvd_req* d_req, uint32_t nreq,
                                const cvd_seg* d_seg, uint64_t nseg, void* d_host_buf, uint64_t host_buf_bytes,
                                cvd_result* d_res, bool no_long, cudaStream_t st);

// Record a failed CUDA call for cvd_last_cuda_error; returns CVD_ECUDA.
int fail_cuda(cudaError_t e);

int check_batch_args(cvd_guest* const* guests, uint32_t nguests, const void* req, uint32_t nreq, const void* seg,
                     uint64_t nseg, const void* stg, uint64_t stg_bytes, const void* res);

// Error bits the no-allocation batch call recorded on the current device
// since they were last taken (cvd_noalloc.cu), read and cleared in stream
// order on `st`; 0 when that call never ran on this device.
cudaError_t noalloc_take_errors(cudaStream_t st, unsigned int* bits);

// mmap install (cvd_mmap.cu)
struct MapReq { uint64_t gva; uint32_t npages, flags; uint64_t hf_begin; };
// With `place`, a record whose flags are exactly kMapNoSpace is a request the
// placer found no range for: its pages get ENOSPC and nothing is installed.
constexpr uint32_t kMapNoSpace = 1u << 30;
int mmap_install(const DevGuest* dg, const DevGuest& host_copy, const MapReq* req, uint32_t nreq,
                 const uint64_t* hf, uint64_t nhf, int32_t* status, cudaStream_t st, bool place = false);
// dependent second-level gathers (cvd_chain.cu): same layouts as
// cvd_chain_req / cvd_chain_result
struct ChainReq { uint64_t table_gva; uint32_t count, guest; uint64_t desc_off; };
struct ChainRes { uint64_t done, fault_gva; uint32_t fault_code, level; uint64_t payload_off, payload_len; };
constexpr uint32_t kChainMaxCount = 65536;
cudaError_t launch_chain_l1(const ChainReq* req, uint32_t nreq, uint32_t nguests, Req* q1, Seg* s1, cudaStream_t st);
// Level 1 of a hazard-free call in one launch (a.guests / nguests / stg /
// stg_bytes: the guests and the descriptor buffer); r1 as the batch gives.
cudaError_t launch_chain_tables(const BatchArgs& a, const ChainReq* req, uint32_t nreq, Result* r1, cudaStream_t st);
cudaError_t launch_chain_len(const ChainReq* req, uint32_t nreq, const Result* r1, const uint8_t* desc, uint64_t cap,
                             uint64_t* len, uint64_t* pairs, cudaStream_t st);
// ecap: entries the payload segment list s2 holds (desc_bytes / 16)
cudaError_t launch_chain_l2(const ChainReq* req, uint32_t nreq, const Result* r1, const uint64_t* len,
                            const uint64_t* offs, const uint8_t* desc, uint64_t cap, uint64_t ecap, Req* q2, Seg* s2,
                            ChainRes* res, cudaStream_t st);
cudaError_t launch_chain_final(const Result* r2, uint32_t nreq, ChainRes* res, cudaStream_t st);
// driver-initiated maps (cvd_place.cu): same layout as cvd_map_place_req
struct MapPlaceReq { uint32_t npages, flags; uint64_t hf_begin; };
int mmap_place(const DevGuest* dg, const DevGuest& host_copy, uint64_t va_lo, uint64_t va_hi, const MapPlaceReq* req,
               uint32_t nreq, const uint64_t* hf, uint64_t nhf, uint64_t* gva_out, int32_t* status, cudaStream_t st);
// Kernel timing of single launches (cvd_profile): prof_begin records an event
// on st when timing is on (false: off, or the event failed); prof_end records
// the closing one and queues the pair for cvd_profile_read under `kind`.
enum ProfKind { kProfMapProbe = 1, kProfPlaceFit = 2 };
struct ProfSpan { cudaEvent_t a = nullptr, b = nullptr; };
bool prof_begin(ProfSpan* s, cudaStream_t st);
void prof_end(ProfSpan* s, ProfKind kind, cudaStream_t st);
}  // namespace cvd
