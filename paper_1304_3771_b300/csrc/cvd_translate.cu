// cvd_translate.cu -- cvd_translate for memslot guests with unit tables
// (sm_103a): the software page walk of Sec. 4.2 (gVA -> gPA through the
// guest's tables, gPA -> host through KVM's memslots) over a batch of
// addresses, with every level above the leaf tables staged in shared memory.
//
// A walk is a chain of dependent 8-byte loads; the paper keeps a 10-entry
// translation cache against that cost (Sec. 4.2).  Here each block copies the
// guest's top table, the first second-level tables, and as many third-level
// tables (page directories) as the guest's memory can need into shared
// memory, plus the per-2 MiB memslot deltas; then a mapped 4 KiB walk reads
// one entry from L2/HBM (the page-table entry itself) and everything else
// from shared memory.  Every thread keeps kTfWalks walks in flight, advanced
// in phases: staged levels for all of them, then all their leaf-table loads
// back to back, then the leaf checks.  A walk that meets anything unstaged
// above the leaf table (a second-level table not staged, a table or page not
// in a 2 MiB unit of a memslot: the reserved window, a missing slot) is
// finished by the generic walk out of line, so the common path stays short;
// a page directory that was not staged is read from the pool inline.
//
// Staging copies exactly the entries a walk would read (the tables do not
// change during a call), so results are those of the generic walk.
#include "cvd_internal.h"

namespace cvd {

namespace {

constexpr int kTfThreads = 512;
constexpr int kTfWalks = 2;            // walks in flight per thread
constexpr uint32_t kTfMaxL3 = 2;       // staged second-level tables (4-level guests)
constexpr uint8_t kTfNone = 0xFF;

// Most page directories a launch stages.
constexpr uint32_t kTfMaxL2 = 64;

// Shared-memory header; the tables follow it (see tf_layout).
struct TfHdr {
  uint32_t valid;                      // top table staged
  uint32_t n3, n2;                     // staged second- / third-level tables
  uint32_t nunits;                     // unit deltas staged
  uint64_t src3[kTfMaxL3];             // host offsets of the staged second-level tables
  uint64_t src2[kTfMaxL2];             // host offsets of the staged page directories
  uint8_t map4[512];                   // top index -> staged table slot (4-level: L3 slot; PAE: PD slot)
  uint8_t map3[kTfMaxL3][512];         // (L3 slot, index) -> staged PD slot (4-level)
};

struct TfLayout {
  size_t l4, l3, l2, units, bytes;
};

__host__ __device__ inline size_t tf_round(size_t x) { return (x + 127) & ~(size_t)127; }

// Offsets of the staged tables for a launch staging up to n2max page
// directories and nunits unit deltas.
__host__ __device__ inline TfLayout tf_layout(uint32_t n2max, uint32_t nunits) {
  TfLayout L;
  L.l4 = tf_round(sizeof(TfHdr));
  L.l3 = L.l4 + 4096;
  L.l2 = L.l3 + 4096 * (size_t)kTfMaxL3;
  L.units = L.l2 + 4096 * (size_t)n2max;
  L.bytes = L.units + tf_round(4 * (((size_t)nunits + 3) & ~(size_t)3));
  return L;
}

// gPA -> host offset through the staged unit deltas; false when the gPA lies
// in no 2 MiB unit of a memslot (the generic walk then decides).
__device__ __forceinline__ bool tf_unit(const int32_t* ud, uint32_t nunits, uint64_t gpa, uint64_t* h) {
  const uint64_t u = gpa >> 21;
  if (u >= nunits) return false;
  const int32_t d = ud[u];
  if (d == kNoUnitDelta) return false;
  *h = gpa + ((uint64_t)(int64_t)d << 12);
  return true;
}

// Pick, in index order, entries of a table that link a stageable table
// (present, a table link, the table in a unit of a memslot) until `want`
// slots are taken; slot numbers go to map[index], the linked tables' host
// offsets to src[slot].  One warp (all lanes) calls it.
__device__ inline void tf_pick(const uint64_t* t, uint32_t nent, const int32_t* ud, uint32_t nunits, uint8_t* map,
                               uint64_t* src, uint32_t* n, uint32_t want, bool pae_pdpt) {
  const int lane = threadIdx.x & 31;
  uint32_t base = *n;
  for (uint32_t c = 0; c < nent && base < want; c += 32) {
    const uint32_t i = c + lane;
    bool ok = false;
    uint64_t h = 0;
    if (i < nent) {
      const uint64_t e = t[i];
      const bool link = pae_pdpt ? !(e & kPaePdpteRsvd) : !(e & kPS);
      ok = (e & kP) && link && tf_unit(ud, nunits, e & kFrame4K, &h);
    }
    const uint32_t m = __ballot_sync(0xffffffffu, ok);
    const uint32_t rank = __popc(m & ((1u << lane) - 1));
    if (ok && base + rank < want) {
      map[i] = (uint8_t)(base + rank);
      src[base + rank] = h;
    }
    base += __popc(m);
    if (base > want) base = want;
  }
  __syncwarp();
  if (lane == 0) *n = base;
  __syncwarp();
}

// Copy `n` 4 KiB tables whose host offsets are src[0..n) to dst (all threads).
__device__ inline void tf_copy_tables(uint64_t* dst, const uint64_t* src, uint32_t n, const uint8_t* pool) {
  for (uint32_t w = threadIdx.x; w < n * 256; w += blockDim.x) {   // 16-byte words
    const uint32_t t = w >> 8, k = w & 255;
    reinterpret_cast<uint4*>(dst + 512ull * t)[k] = __ldg(reinterpret_cast<const uint4*>(pool + src[t]) + k);
  }
}

// Stage the tables (all threads of the block call it).
template <bool PAE>
__device__ inline void tf_stage(unsigned char* smem, const DevGuest& g, uint32_t n2max) {
  TfHdr* H = reinterpret_cast<TfHdr*>(smem);
  const TfLayout L = tf_layout(n2max, g.nunits);
  uint64_t* L4 = reinterpret_cast<uint64_t*>(smem + L.l4);
  uint64_t* L3 = reinterpret_cast<uint64_t*>(smem + L.l3);
  uint64_t* L2 = reinterpret_cast<uint64_t*>(smem + L.l2);
  int32_t* ud = reinterpret_cast<int32_t*>(smem + L.units);
  const uint32_t nunits = g.nunits;
  // unit deltas first: every backing check below goes through them
  const uint4* usrc = reinterpret_cast<const uint4*>(g.unit_delta);
  for (uint32_t i = threadIdx.x; i < (nunits + 3) / 4; i += blockDim.x) reinterpret_cast<uint4*>(ud)[i] = usrc[i];
  for (uint32_t i = threadIdx.x; i < 512; i += blockDim.x) H->map4[i] = kTfNone;
  for (uint32_t i = threadIdx.x; i < kTfMaxL3 * 512; i += blockDim.x) (&H->map3[0][0])[i] = kTfNone;
  if (threadIdx.x == 0) {
    H->n3 = 0;
    H->n2 = 0;
    H->nunits = nunits;
  }
  __syncthreads();
  const uint32_t ntop = PAE ? 4 : 512;
  uint64_t h = 0;
  const bool ok = tf_unit(ud, nunits, PAE ? (g.cr3_gpa & ~31ull) : (g.cr3_gpa & kFrame4K), &h);
  if (threadIdx.x == 0) H->valid = ok ? 1u : 0u;
  if (ok)
    for (uint32_t i = threadIdx.x; i < ntop; i += blockDim.x)
      L4[i] = __ldg(reinterpret_cast<const unsigned long long*>(g.pool + h) + i);
  __syncthreads();
  if (!ok) return;
  if (PAE) {   // page directories hang from the 4 PDPTEs
    if (threadIdx.x < 32) tf_pick(L4, 4, ud, nunits, H->map4, H->src2, &H->n2, n2max < 4 ? n2max : 4, true);
    __syncthreads();
  } else {
    if (threadIdx.x < 32) tf_pick(L4, 512, ud, nunits, H->map4, H->src3, &H->n3, kTfMaxL3, false);
    __syncthreads();
    tf_copy_tables(L3, H->src3, H->n3, g.pool);
    __syncthreads();
    if (threadIdx.x < 32)
      for (uint32_t s = 0; s < H->n3; s++) tf_pick(L3 + 512 * s, 512, ud, nunits, H->map3[s], H->src2, &H->n2, n2max, false);
    __syncthreads();
  }
  tf_copy_tables(L2, H->src2, H->n2, g.pool);
  __syncthreads();
}

// The generic walk (memslots searched, nothing staged) for the rare walks the
// staged path does not finish.
template <bool PAE>
__device__ __noinline__ WalkOut tf_generic(const DevGuest& g, uint64_t va, bool write) {
  return PAE ? walk_pae<kSdSlots>(g, nullptr, va, write) : walk4<kSdSlots>(g, nullptr, va, write);
}

// Walk states between the phases.
constexpr uint32_t kStDone = 0, kStLeafLoad = 1, kStLeaf = 2, kStGeneric = 3;

template <bool PAE>
__global__ void __launch_bounds__(kTfThreads) k_translate_staged(const DevGuest* __restrict__ gp,
                                                                  const uint64_t* __restrict__ gva, uint64_t n,
                                                                  int write, uint32_t n2max,
                                                                  uint64_t* __restrict__ gpa_out,
                                                                  uint64_t* __restrict__ hpa_out,
                                                                  uint32_t* __restrict__ code_out) {
  extern __shared__ __align__(128) unsigned char smem[];
  const DevGuest& G = *gp;
  tf_stage<PAE>(smem, G, n2max);
  const TfHdr* H = reinterpret_cast<const TfHdr*>(smem);
  const TfLayout L = tf_layout(n2max, G.nunits);
  const uint64_t* L4 = reinterpret_cast<const uint64_t*>(smem + L.l4);
  const uint64_t* L3 = reinterpret_cast<const uint64_t*>(smem + L.l3);
  const uint64_t* L2 = reinterpret_cast<const uint64_t*>(smem + L.l2);
  const int32_t* ud = reinterpret_cast<const int32_t*>(smem + L.units);
  const uint32_t nunits = H->nunits;
  const bool valid = H->valid != 0;
  const uint8_t* pool = G.pool;
  const bool wr = write != 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += kTfWalks * stride) {
    uint64_t va[kTfWalks], gpa[kTfWalks], hpa[kTfWalks], at[kTfWalks];
    uint32_t code[kTfWalks], st[kTfWalks], f[kTfWalks];
#pragma unroll
    for (int k = 0; k < kTfWalks; k++) {
      const uint64_t j = i + k * stride;
      va[k] = j < n ? __ldcs(gva + j) : (1ull << 63) | 1ull;   // past the end: non-canonical, no table read
    }
    // phase 1: the staged levels
#pragma unroll
    for (int k = 0; k < kTfWalks; k++) {
      const uint64_t v = va[k];
      const uint32_t hi = (uint32_t)(v >> 32), lo = (uint32_t)v;
      code[k] = kOk; st[k] = kStDone; f[k] = 0; gpa[k] = kAllOnes; at[k] = 0;
      uint64_t e2 = 0;
      bool have2 = false;
      if (PAE) {
        if (hi != 0) { code[k] = kRange; continue; }
        if (!valid) { st[k] = kStGeneric; continue; }
        const uint32_t i3 = lo >> 30;
        const uint64_t e3 = L4[i3];
        if (!(e3 & kP)) { code[k] = kNotPresent | (3u << 8); continue; }
        if (e3 & kPaePdpteRsvd) { code[k] = kRsvd; continue; }
        const uint32_t s2 = H->map4[i3];
        if (s2 == kTfNone) { st[k] = kStGeneric; continue; }
        e2 = L2[s2 * 512 + ((lo >> 21) & 511)];
        f[k] = 6;   // RW and US come from the PDE and the PTE only
        have2 = true;
      } else {
        const uint32_t top = hi >> 15;
        if (top != 0) { code[k] = top == 0x1FFFFu ? kRange : kNonCanonical; continue; }
        if (!valid) { st[k] = kStGeneric; continue; }
        const uint32_t i4 = (hi >> 7) & 511, i3 = ((hi << 2) | (lo >> 30)) & 511;
        const uint64_t e4 = L4[i4];
        if (!(e4 & kP)) { code[k] = kNotPresent | (4u << 8); continue; }
        if (e4 & kPS) { code[k] = kRsvd; continue; }
        const uint32_t s3 = H->map4[i4];
        if (s3 == kTfNone) { st[k] = kStGeneric; continue; }
        const uint64_t e3 = L3[s3 * 512 + i3];
        f[k] = (uint32_t)e4 & (uint32_t)e3;
        if (!(e3 & kP)) { code[k] = kNotPresent | (3u << 8); continue; }
        if (e3 & kPS) {
          gpa[k] = (e3 & kFrame1G) | (v & ((1ull << 30) - 1));
          st[k] = kStLeaf;
          continue;
        }
        const uint32_t s2 = H->map3[s3][i3];
        if (s2 != kTfNone) {
          e2 = L2[s2 * 512 + ((lo >> 21) & 511)];
        } else {   // a page directory beyond the staged ones: read it from the pool
          uint64_t h;
          if (!tf_unit(ud, nunits, (e3 & kFrame4K) + 8ull * ((lo >> 21) & 511), &h)) { st[k] = kStGeneric; continue; }
          e2 = __ldg(reinterpret_cast<const unsigned long long*>(pool + h));
        }
        have2 = true;
      }
      if (have2) {
        f[k] &= (uint32_t)e2;
        if (!(e2 & kP)) { code[k] = kNotPresent | (2u << 8); continue; }
        if (e2 & kPS) {
          gpa[k] = (e2 & kFrame2M) | (v & ((1ull << 21) - 1));
          st[k] = kStLeaf;
          continue;
        }
        uint64_t h;
        if (!tf_unit(ud, nunits, (e2 & kFrame4K) + 8ull * ((lo >> 12) & 511), &h)) { st[k] = kStGeneric; continue; }
        at[k] = h;
        st[k] = kStLeafLoad;
      }
    }
    // phase 2: the leaf-table entries, all loads in flight together
    uint64_t e1[kTfWalks];
#pragma unroll
    for (int k = 0; k < kTfWalks; k++)
      e1[k] = st[k] == kStLeafLoad ? __ldg(reinterpret_cast<const unsigned long long*>(pool + at[k])) : 0;
    // phase 3: leaf checks, in the generic walk's order
#pragma unroll
    for (int k = 0; k < kTfWalks; k++) {
      if (st[k] == kStLeafLoad) {
        f[k] &= (uint32_t)e1[k];
        if (!(e1[k] & kP)) {
          code[k] = kNotPresent | (1u << 8);
          st[k] = kStDone;
        } else {
          gpa[k] = (e1[k] & kFrame4K) | (va[k] & 4095);
          st[k] = kStLeaf;
        }
      }
      hpa[k] = kAllOnes;
      if (st[k] == kStLeaf) {
        if (!(f[k] & 4)) code[k] = kUser;
        else if (wr && !(f[k] & 2)) code[k] = kWriteProtect;
        else if (!tf_unit(ud, nunits, gpa[k], &hpa[k])) st[k] = kStGeneric;
      }
      if (st[k] == kStGeneric) {
        const WalkOut w = tf_generic<PAE>(G, va[k], wr);
        gpa[k] = w.gpa;
        hpa[k] = w.hpa;
        code[k] = w.code;
      } else if (code[k] != kOk) {
        gpa[k] = kAllOnes;
        hpa[k] = kAllOnes;
      }
      const uint64_t j = i + k * stride;
      if (j < n) {
        __stcs(gpa_out + j, gpa[k]);
        __stcs(hpa_out + j, hpa[k]);
        __stcs(code_out + j, code[k]);
      }
    }
  }
}

using TfFn = void (*)(const DevGuest*, const uint64_t*, uint64_t, int, uint32_t, uint64_t*, uint64_t*, uint32_t*);

// Page directories staged for a guest whose memslots end at unit nunits:
// enough for its memory's virtual span (a 1 GiB directory per 512 units, plus
// two for unaligned ends), within a shared-memory budget of a third of an
// SM's so that three blocks (1,536 threads) stay resident.
uint32_t tf_n2max(bool pae, uint32_t nunits) {
  if (pae) return 4;
  uint32_t want = (nunits + 511) / 512 + 2;
  if (want > kTfMaxL2) want = kTfMaxL2;
  const size_t budget = 74 * 1024;
  while (want > 1 && tf_layout(want, nunits).bytes > budget) want--;
  return want;
}

unsigned tf_blocks(TfFn fn, size_t smem) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kTfThreads, smem) != cudaSuccess || b < 1) {
    cudaGetLastError();
    b = 1;
  }
  return (unsigned)b;
}

}  // namespace

bool translate_staged_ok(uint32_t sel, uint32_t nunits) {
  return nunits > 0 && (sel == kPagingX86_64 || sel == kPagingPae) &&
         tf_layout(tf_n2max(sel == kPagingPae, nunits), nunits).bytes <= 227 * 1024;
}

void prepare_translate_staged() {
  cudaFuncSetAttribute(k_translate_staged<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  cudaFuncSetAttribute(k_translate_staged<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

void translate_staged_shape(uint32_t sel, uint32_t nunits, uint32_t* threads_per_sm, uint32_t* walks_per_thread) {
  const bool pae = sel == kPagingPae;
  const size_t sm = tf_layout(tf_n2max(pae, nunits), nunits).bytes;
  *threads_per_sm = tf_blocks(pae ? k_translate_staged<true> : k_translate_staged<false>, sm) * kTfThreads;
  *walks_per_thread = kTfWalks;
}

cudaError_t launch_translate_staged(const DevGuest* g, uint32_t sel, uint32_t nunits, const uint64_t* gva, uint64_t n,
                                    bool write, uint64_t* gpa, uint64_t* hpa, uint32_t* code, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const bool pae = sel == kPagingPae;
  const uint32_t n2max = tf_n2max(pae, nunits);
  const size_t sm = tf_layout(n2max, nunits).bytes;
  const TfFn fn = pae ? k_translate_staged<true> : k_translate_staged<false>;
  // one resident wave (a second, partial wave would run under-occupied)
  const uint64_t want = (n + kTfThreads - 1) / kTfThreads;
  const uint64_t cap = (uint64_t)num_sms() * tf_blocks(fn, sm);
  fn<<<(unsigned)(want < cap ? want : cap), kTfThreads, sm, st>>>(g, gva, n, write ? 1 : 0, n2max, gpa, hpa, code);
  g_launches++;
  return cudaGetLastError();
}

}  // namespace cvd
