// cvd_chain.cu -- dependent second-level gathers on the GPU, sm_103a.
//
// Paper: generic class drivers (DRM for GPUs) receive file operations and
// pass them on (Sec. 6.1); a command submission's argument structure holds
// further user pointers, so the host driver copies the structure in and then
// gathers the buffers it names -- every access through the software hybrid
// address space (copy_from_user, translated once per page, Sec. 4.2).
//
// A request names a descriptor table ({u64 gva, u64 len} entries) in its
// guest.  The call runs as two batch copies joined by three small kernels:
//   level 1  -- every table, one copy_from request each, into the caller's
//               descriptor buffer (hazard-free calls: k_chain_tables, one
//               warp per table; otherwise k_chain_l1 builds the records of
//               a levelled batch);
//   lengths  -- one warp per request sums its entries' lengths (saturating)
//               and emits (clamped length, entry count) for a pair scan;
//               the scan places the payloads back to back and the entries in
//               a list as large as the descriptor buffer (so its size is
//               known on the host and the call never waits for the device);
//   level 2  -- the fitting requests' entries copied into one segment list
//               (k_chain_l2), then one hazard-free copy_from batch gathers
//               them into the payload buffer (reads of guest memory into
//               disjoint payload ranges cannot conflict);
//   results  -- k_chain_final merges the level-2 results.
#include "cvd_internal.h"

namespace cvd {

namespace {

__global__ void k_chain_l1(const ChainReq* __restrict__ req, uint32_t nreq, uint32_t nguests, Req* __restrict__ q1,
                           Seg* __restrict__ s1) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nreq; r += (uint64_t)gridDim.x * blockDim.x) {
    const ChainReq c = req[r];
    const bool malformed = c.count > kChainMaxCount || (c.desc_off & 15) != 0;
    q1[r] = Req{(uint32_t)r, 1, 0, malformed ? nguests : c.guest, c.desc_off};   // guest out of range: BADREQ
    s1[r] = Seg{c.table_gva, 16ull * c.count};
  }
}

// Level 1 of a hazard-free call in one launch: one warp per request reads its
// table (one copy_from segment of 16 x count bytes at table_gva into
// d_desc[desc_off, ...)) by the rules of the batch calls: malformed (count
// over the maximum, desc_off not a multiple of 16, guest out of range) ->
// BADREQ; the range outside the descriptor buffer -> HOSTBUF; then the
// segment checks (non-canonical, outside the user range) at offset 0; the
// pages walked 32 at a time, the bytes before the first faulting byte copied
// page piece by page piece, the rest of the range zero-filled.  r1 gets the
// result the batch call would give.
__global__ void __launch_bounds__(256) k_chain_tables(BatchArgs a, const ChainReq* __restrict__ req, uint32_t nreq,
                                                      Result* __restrict__ r1) {
  const int lane = threadIdx.x & 31;
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = w0; r < nreq; r += nw) {
    const ChainReq c = req[r];
    Result o{0, 0, kOk, 0};
    const uint64_t L = 16ull * c.count;
    if (c.count > kChainMaxCount || (c.desc_off & 15) != 0 || c.guest >= a.nguests) {
      o.fault_code = kBadReq;
    } else if (L > a.stg_bytes || c.desc_off > a.stg_bytes - L) {
      o.fault_code = kHostBuf;
    } else if (L > 0) {
      const DevGuest& G = *a.guests[c.guest];
      uint8_t* dst = a.stg + c.desc_off;
      uint64_t done = L;
      if (!va_canonical(G, c.table_gva)) {
        o.fault_code = kNonCanonical; o.fault_gva = c.table_gva; done = 0;
      } else if (c.table_gva >= va_top(G) || L > va_top(G) - c.table_gva) {
        o.fault_code = kRange; o.fault_gva = c.table_gva; done = 0;
      } else {
        const uint64_t end = c.table_gva + L;
        for (uint64_t pos = c.table_gva; pos < end && done == L; pos = (pos & ~4095ull) + 32ull * 4096) {
          const uint64_t va = lane == 0 ? pos : (pos & ~4095ull) + (uint64_t)lane * 4096;
          const bool active = va < end;
          WalkOut w;
          w.code = kOk; w.hpa = 0;
          if (active) w = walk(G, nullptr, va, false);
          const unsigned bad = __ballot_sync(0xffffffffu, active && w.code != kOk);
          const int fl = bad ? __ffs(bad) - 1 : 32;
          if (bad) {
            const uint64_t fva = __shfl_sync(0xffffffffu, va, fl);
            o.fault_code = __shfl_sync(0xffffffffu, w.code, fl);
            o.fault_gva = fva;
            done = fva - c.table_gva;
          }
          // copy the pieces of the pages before the first faulting one
          for (int k = 0; k < fl; k++) {
            const uint64_t kva = __shfl_sync(0xffffffffu, va, k);
            const uint64_t kh = __shfl_sync(0xffffffffu, w.hpa, k);
            if (kva >= end) break;
            const uint64_t pe = (kva & ~4095ull) + 4096 < end ? (kva & ~4095ull) + 4096 : end;
            warp_copy<16, 2>(dst + (kva - c.table_gva), G.pool + kh, pe - kva, lane);
          }
        }
      }
      if (done < L) warp_zero<16>(dst + done, L - done, lane);
      o.done = done;
    }
    if (lane == 0) r1[r] = o;
  }
}

// One warp per request: L (saturating) and the scan pair (min(L, cap + 1),
// count) for requests whose table was read whole; (0, 0) otherwise.
__global__ void k_chain_len(const ChainReq* __restrict__ req, uint32_t nreq, const Result* __restrict__ r1,
                            const uint8_t* __restrict__ desc, uint64_t cap, uint64_t* __restrict__ len,
                            uint64_t* __restrict__ pairs) {
  const int lane = threadIdx.x & 31;
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = w0; r < nreq; r += nw) {
    const ChainReq c = req[r];
    const bool ok = r1[r].fault_code == kOk;
    uint64_t L = 0;
    if (ok) {
      const uint64_t* t = reinterpret_cast<const uint64_t*>(desc + c.desc_off);
      uint64_t part = 0;
      for (uint32_t k = lane; k < c.count; k += 32) {
        const uint64_t l = t[2 * k + 1];
        part = part + l < part ? ~0ull : part + l;
      }
      L = warp_sat_sum(part);
    }
    if (lane == 0) {
      len[r] = L;
      pairs[2 * r] = ok ? (L < cap + 1 ? L : cap + 1) : 0;
      pairs[2 * r + 1] = ok ? c.count : 0;
    }
  }
  if (w0 == 0 && lane == 0) { pairs[2 * (uint64_t)nreq] = 0; pairs[2 * (uint64_t)nreq + 1] = 0; }
}

// One warp per request: level-2 record, its entries into the segment list,
// and the result fields known before the payload copy.
__global__ void k_chain_l2(const ChainReq* __restrict__ req, uint32_t nreq, const Result* __restrict__ r1,
                           const uint64_t* __restrict__ len, const uint64_t* __restrict__ offs,
                           const uint8_t* __restrict__ desc, uint64_t cap, uint64_t ecap, Req* __restrict__ q2,
                           Seg* __restrict__ s2, ChainRes* __restrict__ res) {
  const int lane = threadIdx.x & 31;
  const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = w0; r < nreq; r += nw) {
    const ChainReq c = req[r];
    const Result a = r1[r];
    ChainRes o{0, 0, 0, 0, 0, 0};
    Req q{0, 0, 0, 0, 0};
    if (a.fault_code != kOk) {
      o.done = a.done; o.fault_gva = a.fault_gva; o.fault_code = a.fault_code; o.level = 1;
    } else {
      const uint64_t L = len[r], P = offs[2 * r], C = offs[2 * r + 1];
      const uint64_t Lc = L < cap + 1 ? L : cap + 1;
      o.payload_len = L;
      // no overflow: nreq x (cap + 1) < 2^63 is checked on the host; C + count
      // passes ecap only when tables overlap in the descriptor buffer
      if (P + Lc <= cap && C + c.count <= ecap) {
        o.payload_off = P;
        q = Req{(uint32_t)C, c.count, 0, c.guest, P};
        const Seg* t = reinterpret_cast<const Seg*>(desc + c.desc_off);
        for (uint32_t k = lane; k < c.count; k += 32) s2[C + k] = t[k];
      } else {
        o.fault_code = kHostBuf; o.level = 2;
      }
    }
    if (lane == 0) { q2[r] = q; res[r] = o; }
  }
}

__global__ void k_chain_final(const Result* __restrict__ r2, uint32_t nreq, ChainRes* __restrict__ res) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nreq; r += (uint64_t)gridDim.x * blockDim.x) {
    ChainRes o = res[r];
    if (o.level != 0) continue;
    const Result b = r2[r];
    o.done = b.done; o.fault_gva = b.fault_gva; o.fault_code = b.fault_code;
    if (b.fault_code != kOk) o.level = 2;
    res[r] = o;
  }
}

unsigned grid_for_n(uint64_t n, unsigned per_block) {
  uint64_t want = (n + per_block - 1) / per_block;
  uint64_t cap = (uint64_t)num_sms() * 8;
  if (want > cap) want = cap;
  return (unsigned)(want ? want : 1);
}

}  // namespace

cudaError_t launch_chain_l1(const ChainReq* req, uint32_t nreq, uint32_t nguests, Req* q1, Seg* s1, cudaStream_t st) {
  k_chain_l1<<<grid_for_n(nreq, 256), 256, 0, st>>>(req, nreq, nguests, q1, s1);
  g_launches++;
  return cudaGetLastError();
}

cudaError_t launch_chain_tables(const BatchArgs& a, const ChainReq* req, uint32_t nreq, Result* r1, cudaStream_t st) {
  k_chain_tables<<<grid_for_n(nreq, 8), 256, 0, st>>>(a, req, nreq, r1);
  g_launches++;
  return cudaGetLastError();
}

cudaError_t launch_chain_len(const ChainReq* req, uint32_t nreq, const Result* r1, const uint8_t* desc, uint64_t cap,
                             uint64_t* len, uint64_t* pairs, cudaStream_t st) {
  k_chain_len<<<grid_for_n(nreq, 8), 256, 0, st>>>(req, nreq, r1, desc, cap, len, pairs);
  g_launches++;
  return cudaGetLastError();
}

cudaError_t launch_chain_l2(const ChainReq* req, uint32_t nreq, const Result* r1, const uint64_t* len,
                            const uint64_t* offs, const uint8_t* desc, uint64_t cap, uint64_t ecap, Req* q2, Seg* s2,
                            ChainRes* res, cudaStream_t st) {
  k_chain_l2<<<grid_for_n(nreq, 8), 256, 0, st>>>(req, nreq, r1, len, offs, desc, cap, ecap, q2, s2, res);
  g_launches++;
  return cudaGetLastError();
}

cudaError_t launch_chain_final(const Result* r2, uint32_t nreq, ChainRes* res, cudaStream_t st) {
  k_chain_final<<<grid_for_n(nreq, 256), 256, 0, st>>>(r2, nreq, res);
  g_launches++;
  return cudaGetLastError();
}

}  // namespace cvd
