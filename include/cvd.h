/*
 * cvd.h -- C ABI of libcvd.so: the memory operations of the Common Virtual
 * Driver (CVD) backend, i.e. the software hybrid address space, on one B300.
 *
 * The paper's boundary is the set of kernel memory routines a host driver
 * calls while servicing a file operation forwarded from a guest process:
 * copy_from_user / copy_to_user style access to a guest user buffer, and
 * insert_pfn style mapping of a page into the guest process (Sec. 4.2,
 * Sec. 6.2).  The backend services them against the guest process's memory:
 * it walks the guest page tables from the page-table root captured when the
 * guest process first called (Sec. 6.3), turns the guest-physical address into
 * a host address through KVM's memslots (Sec. 4.2), and translates once per
 * page because guest-virtual pages are not host-contiguous (Sec. 4.2).
 *
 * Conventions for every call:
 *  - Pointers named d_* are CUDA device pointers; h_* are host pointers.
 *    The caller owns every buffer it passes and keeps it alive until the
 *    stream has reached the call's work.  The library owns the guest handle,
 *    its device descriptor and the per-stream scratch it allocates.
 *  - Calls are stream ordered and return once the work is enqueued, except
 *    where a call says it synchronises.
 *  - Return value: CVD_OK or a negative API status (bad argument, out of
 *    memory, CUDA error).  Guest faults are NOT API errors: they are per
 *    request data (cvd_result) or per page status, like Linux copy_*_user
 *    returning the number of bytes not copied.
 *  - Guest-physical and host addresses are 64-bit byte offsets.  "hPA" is a
 *    byte offset into the guest's host pool (the device buffer that plays the
 *    host memory holding the guest's RAM).
 *  - Page-table format: x86-64 4-level paging, 512 little-endian u64 entries
 *    per 4 KiB table (Intel SDM Vol. 3 ch. 4).  The paper's implementation used
 *    32-bit PAE; the walk semantics are otherwise the paper's.
 *  - Buffers are read in whole aligned 16-byte blocks that contain at least
 *    one byte of the requested range, so up to 15 bytes just before and just
 *    after a range may be read (never written); writes are exact.  No
 *    buffer needs any alignment: an aligned 16-byte block lies inside one
 *    memory page, so a block holding one byte of a mapped buffer is mapped.
 *    A caller may pass a staging view at any byte offset of a larger
 *    allocation; the bytes around it are read at most, never changed.
 */
#ifndef CVD_H
#define CVD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *cvd_stream_t;    /* same type as cudaStream_t */
typedef struct cvd_guest cvd_guest;          /* opaque, library owned */

/* ---- API status ------------------------------------------------------- */
#define CVD_OK          0
#define CVD_EINVAL    (-22)   /* bad argument or descriptor */
#define CVD_ENOMEM    (-12)   /* device or host allocation failed */
#define CVD_ECUDA      (-5)   /* a CUDA call failed (cvd_last_cuda_error) */
#define CVD_ETIMEDOUT (-110)  /* a bounded wait ran out */
#define CVD_EHAZARD   (-11)   /* a batch declared hazard-free is not */
#define CVD_E2BIG      (-7)   /* batch larger than cvd_copy_batch_noalloc's fixed scratch */

/* ---- per-request fault codes (cvd_result.fault_code) ------------------- */
#define CVD_FAULT_NONE           0
#define CVD_FAULT_NOT_PRESENT    1   /* | level << 8 (4 = top level) */
#define CVD_FAULT_WRITE_PROTECT  2   /* copy to a page whose effective RW is 0 */
#define CVD_FAULT_NONCANONICAL   3   /* bits 63:47 of a segment start differ */
#define CVD_FAULT_RANGE          4   /* segment reaches outside [0, 2^47) */
#define CVD_FAULT_NOSLOT         5   /* gPA (or a table) backed by no memslot / no usable EPT mapping */
#define CVD_FAULT_RSVD           6   /* PS set in a level-4 entry */
#define CVD_FAULT_USER           7   /* effective US is 0 */
#define CVD_FAULT_HOSTBUF        8   /* staging range outside the staging buffer */
#define CVD_FAULT_BADREQ         9   /* malformed request descriptor */
#define CVD_FAULT_EPT_VIOLATION 10   /* copy to a page the guest's EPT maps without write permission */

/* ---- per-page mmap status ---------------------------------------------- */
#define CVD_MAP_OK       0
#define CVD_MAP_EBUSY  (-16)  /* a present leaf or a huge leaf is in the way */
#define CVD_MAP_ENOMEM (-12)  /* PT pool or reserved window exhausted (latches) */
#define CVD_MAP_EINVAL (-22)  /* malformed request or host frame outside the pool */
#define CVD_MAP_EFAULT (-14)  /* a present table is not backed by a memslot */
#define CVD_MAP_ENOSPC (-28)  /* cvd_mmap_place: no free range of that size in the window */

#define CVD_MAX_SLOTS 64
#define CVD_MAX_GUESTS_PER_BATCH 64

/* Guest paging formats (Intel SDM Vol. 3 ch. 4).  x86-64 4-level: gVA bits
 * 47:39/38:30/29:21/20:12, user range = the canonical lower half [0, 2^47),
 * 1 GiB and 2 MiB leaves.  32-bit PAE (the paper's implementation, Sec. 6.2):
 * a 4-entry page directory pointer table (gVA bits 31:30; a PDPTE carries P
 * and the frame, bits 1, 2 and 5..8 are reserved -> RSVD), then PD (29:21,
 * 2 MiB leaves) and PT (20:12); user range [0, 2^32), no non-canonical
 * addresses; fault levels 3, 2, 1. */
#define CVD_PAGING_X86_64 0u
#define CVD_PAGING_PAE    1u

/* Second dimension (guest-physical -> host).  Memslots: the KVM case of
 * Sec. 4.2.  EPT: the case of other hypervisors (Sec. 4.2), where the backend
 * finishes the translation by walking the EPT in software; format per the
 * Intel SDM Vol. 3 sec. 28.3.2: 4 levels indexed by gPA bits 47:39 / 38:30 /
 * 29:21 / 20:12 from the root at host-pool byte offset ept_root; entry bit 0
 * (read) makes an entry usable, bit 1 (write) is ANDed over the levels, bit 7
 * makes a 1 GiB / 2 MiB leaf at levels 3 / 2 and is reserved (entry unusable)
 * at level 4; addresses in bits 51:12 are host-pool byte offsets.  A page is
 * backed only when its whole 4 KiB host frame lies in the pool; guest table
 * reads need read permission only; a write through a mapping without write
 * permission faults with CVD_FAULT_EPT_VIOLATION; anything not backed is
 * CVD_FAULT_NOSLOT.  Reserved frames (rsv window) still go through the p2m
 * first.  The EPT must not change while a call that walks it is in flight. */
#define CVD_SECOND_MEMSLOTS 0u
#define CVD_SECOND_EPT      1u

/* Memslot: guest frames [base_gfn, base_gfn + npages) live at host pool
 * offset host_off (4 KiB aligned).  Sec. 4.2: in KVM a guest-physical address
 * maps directly to a host address of the VM process. */
typedef struct { uint64_t base_gfn, npages, host_off; } cvd_memslot;

typedef struct {
    void    *d_host_pool;       /* device buffer holding the guest's RAM */
    uint64_t host_pool_bytes;
    const cvd_memslot *slots;   /* host array, copied; non-overlapping (unused with an EPT) */
    uint32_t nslots;            /* 1..CVD_MAX_SLOTS; 0 with an EPT */
    uint32_t paging;            /* CVD_PAGING_X86_64 or CVD_PAGING_PAE */
    uint64_t cr3_gpa;           /* top-level table gPA, captured at first call (Sec. 6.3);
                                   PAE: the 32-byte aligned 4-entry PDPT, below 4 GiB */
    uint64_t pt_pool_gfn, pt_pool_n;  /* frames the frontend handed over for new
                                         page-table pages (Sec. 4.2); inside memslots */
    uint64_t rsv_gfn, rsv_n;    /* reserved guest frames for mapped pages (Sec. 4.2);
                                   outside every memslot */
    uint64_t *d_p2m;            /* device u64[rsv_n]: reserved frame -> host frame
                                   (~0 = unmapped); caller owned, caller initialised */
    uint32_t second;            /* CVD_SECOND_MEMSLOTS or CVD_SECOND_EPT */
    uint32_t reserved1;         /* must be 0 */
    uint64_t ept_root;          /* CVD_SECOND_EPT: host-pool byte offset of the EPT's
                                   top table, 4 KiB aligned, inside the pool; the EPT
                                   tables live in the pool and are caller owned */
} cvd_guest_desc;

/* One guest buffer segment (an iovec entry). */
typedef struct { uint64_t gva, len; } cvd_seg;

/* One forwarded read/write/ioctl buffer: segments [seg_begin, seg_begin +
 * seg_count) of the segment array, concatenated, tied to the staging range
 * [host_off, host_off + L) where L is the sum of the segment lengths.
 * dir 0 = copy from guest (copy_from_user), 1 = copy to guest (copy_to_user).
 * guest indexes the guest array of cvd_copy_batch. */
typedef struct { uint32_t seg_begin, seg_count, dir, guest; uint64_t host_off; } cvd_req;

/* done = bytes copied = offset of the first faulting byte (L if none);
 * fault_gva = address of that byte; fault_code = CVD_FAULT_*. */
typedef struct { uint64_t done, fault_gva; uint32_t fault_code, pad; } cvd_result;

/* One mmap install: npages pages from page-aligned gva, page k backed by host
 * frame hf[hf_begin + k]; flags = PTE bits RW|US|PWT|PCD|G (P optional) plus
 * CVD_MAP_NX for the NX bit. */
typedef struct { uint64_t gva; uint32_t npages, flags; uint64_t hf_begin; } cvd_map_req;
#define CVD_MAP_NX (1u << 31)

/* One driver-initiated map (cvd_mmap_place): like cvd_map_req without an
 * address; the library picks it. */
typedef struct { uint32_t npages, flags; uint64_t hf_begin; } cvd_map_place_req;

/* ---- guest lifetime ----------------------------------------------------- */

/* Validate the descriptor and create the library's device copy of it
 * (memslots sorted by base_gfn).  EINVAL: no pool, nslots out of range,
 * overlapping slots, a slot outside the pool or not 4 KiB aligned, the
 * reserved window overlapping a slot, PT-pool frames outside the slots,
 * rsv_n > 0 with no p2m, an unknown paging format, or (PAE) a cr3 that is not
 * 32-byte aligned or not below 4 GiB; an unknown second dimension or a
 * non-zero reserved1; with an EPT: slots given (nslots != 0), a PT pool
 * (pt_pool_n != 0; mmap installs into an EPT guest are refused with
 * CVD_MAP_EINVAL per page), or an ept_root that is not 4 KiB aligned or whose
 * table does not lie in the pool.  ENOMEM if the descriptor's device copy or
 * its counters cannot be allocated, ECUDA if a copy to the device fails
 * (nothing is left allocated either way).  The library owns its device allocations: the
 * descriptor copy, the allocation counters, and (when every memslot starts
 * and ends on a 2 MiB guest-frame boundary below 32 GiB) the per-2 MiB unit
 * tables cvd_translate looks memslots up in (5 bytes per 2 MiB unit up to
 * the last slot's end, at most 80 KiB; without them translation searches
 * the slots, with the same results).  Synchronises the current device. */
int cvd_guest_create(const cvd_guest_desc *desc, cvd_guest **out);

/* Free the handle.  The caller must have synchronised every stream that has
 * work for this guest.  Synchronises the current device. */
int cvd_guest_destroy(cvd_guest *g);

/* Frames taken so far from the PT pool and the reserved window by
 * cvd_mmap_install (device-resident counters).  Synchronises the device. */
int cvd_guest_alloc_state(cvd_guest *g, uint64_t *pt_used, uint64_t *rsv_used);

/* Set those counters: a guest re-created from saved state (a repro file of
 * its pool, descriptor and counters) continues installing where the saved
 * one stopped -- the next PT-pool frame and reserved frame each install
 * takes (Sec. 4.2, insert_pfn) come after the ones already used.  EINVAL
 * when a count passes its pool (pt_pool_n, rsv_n).  Synchronises the
 * device. */
int cvd_guest_set_alloc_state(cvd_guest *g, uint64_t pt_used, uint64_t rsv_used);

/* ---- a1/a2: translation (Sec. 4.2 walk + memslot step) ------------------ */

/* For each of n gVAs: software walk of the guest's 4-level tables, then
 * gPA -> hPA via the memslots (or the p2m for reserved frames).  access:
 * 0 = read, 1 = write (checks effective RW).  Outputs, per index: d_gpa,
 * d_hpa (all ones on a fault) and d_fault (CVD_FAULT_*).  The walk never
 * writes the tables.  n may be 0.  Fault order per level, top-down: not
 * present, PS at level 4; then US, then RW, then the memslot step. */
int cvd_translate(cvd_guest *g, const uint64_t *d_gva, uint64_t n, uint32_t access,
                  uint64_t *d_gpa, uint64_t *d_hpa, uint32_t *d_fault, cvd_stream_t stream);

/* ---- a3/a4: gather / scatter of forwarded buffers (Sec. 4.2) ------------ */

/* copy_from_user for nreq requests (their dir and guest fields are ignored):
 * the bytes before the first faulting byte go to d_host_buf + host_off, the
 * rest of the staging range is zero-filled.  copy_to_user likewise from the
 * staging buffer into the guest, needing writable pages; guest bytes at and
 * after the fault are left untouched.  Requests take effect in index order
 * (sequential semantics): the device marks every request that may conflict
 * with another -- one touching a guest page that another request (or its own
 * other segment, for copy_to) also touches with a write, pages counted up to
 * each segment's end even past a fault, or every request when the staging
 * ranges are not in increasing order without overlap -- and copies the
 * unmarked ones in one parallel launch; one stream synchronisation then
 * reads how many were marked: up to 32 run one after another in index order
 * on the device, more are levelled byte-exactly on the host (their run list
 * comes back; two more synchronisations) and copied level by level.  All
 * translations of one call see the page tables as they were when the call
 * started; a call whose copies write the frames holding those tables gets
 * unspecified bytes (but never touches memory outside the pools and the
 * staging buffer).
 * Malformed requests fault with BADREQ / HOSTBUF and copy nothing.  A request
 * uses seg_count entries of library scratch sized by nseg: if the running
 * sum of seg_count over well-formed requests passes nseg, the request is
 * BADREQ (only possible when requests share segment descriptors).  The
 * staging buffer must not overlap a guest's host pool, and guests of one call
 * whose pools overlap must start a multiple of 4 KiB apart (EINVAL). */
int cvd_copy_from_guest(cvd_guest *g, const cvd_req *d_req, uint32_t nreq,
                        const cvd_seg *d_seg, uint64_t nseg,
                        void *d_host_buf, uint64_t host_buf_bytes,
                        cvd_result *d_res, cvd_stream_t stream);
int cvd_copy_to_guest(cvd_guest *g, const cvd_req *d_req, uint32_t nreq,
                      const cvd_seg *d_seg, uint64_t nseg,
                      const void *d_host_buf, uint64_t host_buf_bytes,
                      cvd_result *d_res, cvd_stream_t stream);

/* ---- a5: mmap PTE install (insert_pfn, Sec. 6.2; Sec. 4.2) -------------- */

/* Install pages in request order, page order: walk (creating missing
 * tables, each the next PT-pool frame, zeroed, linked P|RW|US), take the next
 * reserved guest frame r, write leaf r<<12 | P | flags (NX -> bit 63), set
 * d_p2m[r - rsv_gfn] = hf.  d_page_status[sum of npages] gets, per page,
 * CVD_MAP_OK / EBUSY (present or huge leaf in the way) / ENOMEM (pool or
 * window exhausted; every later page also ENOMEM; nothing of the page is
 * written) / EINVAL (request misaligned, outside the user half, hf range
 * outside [0, nhf), bad flags; or host frame outside the pool) / EFAULT.
 * The allocation order is exactly the sequential one.  Must not run
 * concurrently with any other call on the same guest.  Synchronises the
 * stream twice: once to size its scratch, once before returning. */
int cvd_mmap_install(cvd_guest *g, const cvd_map_req *d_req, uint32_t nreq,
                     const uint64_t *d_hf, uint64_t nhf, int32_t *d_page_status,
                     cvd_stream_t stream);

/* ---- dependent second-level gathers ------------------------------------- */

/* A command submission through a generic class driver (DRM, Sec. 6.1)
 * passes a structure holding further user pointers: the host driver copies
 * the structure in, then gathers the buffers it names, each access through
 * the hybrid address space (Sec. 4.2).  A request names a descriptor table
 * of `count` entries {u64 gva, u64 len} (the cvd_seg layout) at table_gva in
 * guest `guest`. */
typedef struct { uint64_t table_gva; uint32_t count, guest; uint64_t desc_off; } cvd_chain_req;
/* done = payload bytes gathered (level 0/2) or table bytes read (level 1);
 * level 0 = no fault, 1 = fault reading the table, 2 = fault in the payload
 * (or HOSTBUF: the payload does not fit); payload_off / payload_len = where
 * the payload went in the payload buffer and its length (the saturating sum
 * of the entries' lengths; 0 after a level-1 fault; payload_off 0 when it
 * does not fit). */
typedef struct {
    uint64_t done, fault_gva;
    uint32_t fault_code, level;
    uint64_t payload_off, payload_len;
} cvd_chain_result;
#define CVD_CHAIN_MAX_COUNT 65536u

/* (1) Every request's table is read, as one copy_from request each (rules of
 * cvd_copy_batch, with `flags` = HAZARD_FREE / CHECK applying to this step),
 * into d_desc[desc_off, desc_off + 16 count); every table read sees guest
 * memory as it was when the call started (nothing here writes guest
 * memory).  count > CVD_CHAIN_MAX_COUNT or desc_off not a multiple of 16 ->
 * BADREQ.  A fault ends the request at level 1.  (2) For the requests whose
 * table was read whole, in index order: the payload goes at the sum of the
 * earlier such requests' lengths, and the entries take places after the
 * earlier such requests' entries in a list of desc_bytes / 16 entries (as
 * many as the descriptor buffer holds); the request fits when its payload
 * ends within payload_bytes and its entries within that list (the second
 * fails only when tables overlap in d_desc); else HOSTBUF at level 2,
 * nothing copied.  (3) The entries of each fitting request are gathered in
 * order into its payload range with the copy_from rules (prefix up to the
 * first faulting byte, rest zero-filled), as one hazard-free batch.  d_desc
 * must be 16-byte aligned; neither buffer may overlap a guest pool.  EINVAL
 * also for flag bits other than HAZARD_FREE / CHECK, desc_bytes >= 2^36,
 * payload_bytes >= 2^52, or nreq x (payload_bytes + 1) >= 2^63.  The steps
 * are chained on the device: with HAZARD_FREE the call does not synchronise
 * (without it, step 1 is levelled and synchronises like cvd_copy_batch).
 * Library scratch: about 3 x desc_bytes plus per-request records; one call
 * at a time shares it (a mutex). */
int cvd_gather_chained(cvd_guest *const *guests, uint32_t nguests,
                       const cvd_chain_req *d_req, uint32_t nreq,
                       void *d_desc, uint64_t desc_bytes,
                       void *d_payload, uint64_t payload_bytes,
                       cvd_chain_result *d_res, uint32_t flags, cvd_stream_t stream);

/* ---- driver-initiated maps (Sec. 6.6) ---------------------------------- */

/* A driver maps memory from inside an operation, so the guest has not chosen
 * a virtual range: the library picks one in [va_lo, va_hi) and installs
 * there.  Steps: (1) a page of the window is free when its walk, on the
 * tables as they are when the call starts, meets a non-present entry before
 * a leaf (a present leaf, a present PS entry, a PAE PDPTE with reserved bits
 * or a present table no memslot backs make it taken); (2) requests in index
 * order: a malformed one (npages 0, bad flags, hf range outside [0, nhf))
 * gets no range and EINVAL for its pages; otherwise its range is the lowest
 * page-aligned [a, a + 4096 npages) of free pages inside the window that no
 * earlier request of the call was given (first fit), or none, with ENOSPC
 * for its pages; (3) the placed requests are installed at their ranges by
 * the rules of cvd_mmap_install, in index order.  d_gva[r] = the range start,
 * or all ones; d_page_status as in cvd_mmap_install (requests' pages in
 * order; ENOSPC pages are never ENOMEM).  A guest behind an EPT gets no
 * ranges and EINVAL everywhere.  EINVAL for the call: window not 4 KiB
 * aligned, empty, or past the guest's user range (2^47; PAE 2^32).  Must
 * not run concurrently with any other call on the same guest; synchronises
 * the stream (once per table level while scanning the window, then as
 * cvd_mmap_install does). */
int cvd_mmap_place(cvd_guest *g, uint64_t va_lo, uint64_t va_hi,
                   const cvd_map_place_req *d_req, uint32_t nreq,
                   const uint64_t *d_hf, uint64_t nhf, uint64_t *d_gva,
                   int32_t *d_page_status, cvd_stream_t stream);

/* ---- a6-a8: batches ------------------------------------------------------ */

#define CVD_BATCH_HAZARD_FREE  (1u << 0)  /* caller guarantees no two requests touch a
                                             common byte (guest or staging) with one of
                                             them writing it: one persistent launch over
                                             a byte-balanced work list, no synchronisation */
#define CVD_BATCH_GRAPH        (1u << 1)  /* with HAZARD_FREE: capture the launches in a
                                             CUDA graph on first use, replay it on later
                                             calls with identical arguments */
#define CVD_BATCH_CHECK        (1u << 2)  /* with HAZARD_FREE: verify the claim first (one
                                             stream synchronisation); CVD_EHAZARD if false,
                                             nothing copied */

/* Mixed-direction batch over up to CVD_MAX_GUESTS_PER_BATCH guests (req.guest
 * indexes guests[]).  Without HAZARD_FREE it behaves like the two calls above
 * (sequential semantics; one synchronisation, three when more than 32
 * requests are marked).  All guests of a batch must have been created on the
 * current device; guests whose pools overlap must start a multiple of 4 KiB
 * apart (the same guest twice is fine), else EINVAL. */
int cvd_copy_batch(cvd_guest *const *guests, uint32_t nguests,
                   const cvd_req *d_req, uint32_t nreq, const cvd_seg *d_seg, uint64_t nseg,
                   void *d_host_buf, uint64_t host_buf_bytes, cvd_result *d_res,
                   uint32_t flags, cvd_stream_t stream);

/* Same batch with requests, segments, staging buffer and results in host
 * memory (h_*; pinned memory gives full PCIe speed).  Copies the requests and
 * segments to library device scratch, and of the staging buffer only the
 * ranges that copy-to requests read (ranges less than 64 KiB apart travel as
 * one copy); runs the batch; copies the results back, then only the ranges
 * that accepted copy-from requests wrote (two of them travel as one copy when
 * the bytes between them went in unchanged); synchronises the stream.  Bytes
 * of h_host_buf outside every copy-from range are never written.  One
 * transfer per maximal run of ranges: a buffer that keeps copy-to sources and
 * copy-from destinations in separate regions moves in one copy each way. */
int cvd_copy_batch_host(cvd_guest *const *guests, uint32_t nguests,
                        const cvd_req *h_req, uint32_t nreq, const cvd_seg *h_seg, uint64_t nseg,
                        void *h_host_buf, uint64_t host_buf_bytes, cvd_result *h_res,
                        uint32_t flags, cvd_stream_t stream);

/* One batch of cvd_copy_batches: the device arguments of cvd_copy_batch. */
typedef struct {
    const cvd_req *d_req;
    uint32_t nreq, pad;
    const cvd_seg *d_seg;
    uint64_t nseg;
    cvd_result *d_res;
} cvd_dev_batch;

/* Hazard-free batches in order over one staging buffer, planned ahead: the
 * planning of batch i + 1 (request checks, walks, fault search) runs on a
 * library stream while batch i copies on `stream` (two scratch slots; batch
 * i + 2's planning waits for batch i's copy).  Results, staging bytes and
 * guest memory are those of nb consecutive cvd_copy_batch calls with
 * CVD_BATCH_HAZARD_FREE, provided no batch's copies write a frame holding a
 * page table that a later batch walks (planning may read the tables before
 * earlier batches' copies are done; with such a write the later batch's
 * results are unspecified, never outside the pools and the staging buffer).
 * flags must be exactly CVD_BATCH_HAZARD_FREE.  Errors: as cvd_copy_batch,
 * checked for every batch before anything is launched.  Does not
 * synchronise; with cvd_profile_enable each batch records (plan start on the
 * library stream, copy start, copy end). */
int cvd_copy_batches(cvd_guest *const *guests, uint32_t nguests, const cvd_dev_batch *batches,
                     uint32_t nbatches, void *d_host_buf, uint64_t host_buf_bytes,
                     uint32_t flags, cvd_stream_t stream);

/* One batch of cvd_copy_batches_host: the arguments of cvd_copy_batch_host. */
typedef struct {
    const cvd_req *h_req;
    uint32_t nreq, pad;
    const cvd_seg *h_seg;
    uint64_t nseg;
    void *h_host_buf;
    uint64_t host_buf_bytes;
    cvd_result *h_res;
} cvd_host_batch;

/* The batches in order, with the results of nb consecutive
 * cvd_copy_batch_host calls, pipelined: batch i + 1's inputs go to the device
 * while batch i's outputs come back (two library device slots, two private
 * copy streams; the batches themselves run in order on `stream`).  When batch
 * i + 1 reads host bytes that batch i may write back (its copy-from ranges),
 * its inputs wait for those writes.  Returns when every result and written
 * byte is in host memory.  Errors: as cvd_copy_batch_host; on an error no
 * copy on the caller's buffers is left in flight. */
int cvd_copy_batches_host(cvd_guest *const *guests, uint32_t nguests, const cvd_host_batch *batches,
                          uint32_t nbatches, uint32_t flags, cvd_stream_t stream);

/* No-allocation batch (the paper has no counterpart; this is a service for
 * callers of this library).  Some callers cannot allocate device memory on
 * their request path: cudaMalloc/cudaFree synchronise the whole device, which
 * stalls every other stream of a latency-bound request loop, and a process
 * whose device memory is already held by another allocator (a framework's
 * caching allocator, say) can see a late cudaMalloc fail.  The other batch
 * calls grow per-stream scratch with cudaMalloc on first use and for larger
 * batches; this one never allocates.  It runs one guest's batch with the
 * results, staging bytes and guest memory of cvd_copy_batch with
 * CVD_BATCH_HAZARD_FREE (same planner and copy engine), using a fixed scratch
 * area of CVD_NOALLOC_SCRATCH_BYTES that every GPU loading the library
 * reserves until the process exits.  It differs from that call in three ways
 * that change speed or reporting, never results: it always uses the
 * library's default copy parameters (cvd_set_copy_params and cvd_tune do not
 * apply); its list of long segments (over 1,024 pages) walked across the
 * whole grid holds 4,096 blocks of 256 pages, and the planner walks the rest
 * inline; and its device error word (bit 1: a bounded wait inside the copy
 * engine gave up and a piece was skipped) lives in the fixed area, not in the
 * stream's scratch.  cvd_stream_check reports that word together with the
 * stream's own and clears it; it is zeroed when the area is set up on a
 * device and otherwise accumulates across calls until checked.  req.guest
 * must be 0.  Limits: nreq <= CVD_NOALLOC_MAX_REQS and nseg <=
 * CVD_NOALLOC_MAX_SEGS, else CVD_E2BIG and nothing runs; the other argument
 * checks are those of cvd_copy_batch (CVD_EINVAL).  The first call on a
 * device looks up the scratch area's device address and zeroes its control
 * block in stream order (no allocation); make that first call before any
 * stream capture.  All calls share the one scratch area: calls that can
 * overlap on the GPU (different streams without ordering between them) race
 * and give wrong results; order them, or use cvd_copy_batch.  Every work
 * array a call needs cleared is cleared by that call's own kernels, so a
 * call never depends on the previous call's leftovers.  Returns once the
 * work is enqueued. */
#define CVD_NOALLOC_SCRATCH_BYTES (16u << 20)
#define CVD_NOALLOC_MAX_REQS 65536u
#define CVD_NOALLOC_MAX_SEGS 262144u
int cvd_copy_batch_noalloc(cvd_guest *g, const cvd_req *d_req, uint32_t nreq,
                           const cvd_seg *d_seg, uint64_t nseg,
                           void *d_host_buf, uint64_t host_buf_bytes, cvd_result *d_res,
                           cvd_stream_t stream);

/* ---- a9: serving request loop (continuous batching) ---------------------
 * Forwarded operations from several guests arrive over time; the server
 * admits them in arrival order as staging memory (a best-fit arena of
 * d_staging) and in-flight slots free up, and launches waves of admitted
 * requests (up to max_batch, three in flight) as levelled batches while
 * earlier waves run: on one stream, or with CVD_SERVER_TWO_STREAMS on two
 * (guest g on stream g % 2).  Every guest's requests take effect in arrival
 * order.  A wave never waits for the host: its conflicting requests are
 * found and ordered on the device.  The paper's dual thread (Sec. 5) plays
 * the same role of letting operations proceed and overlap without blocking
 * the guest. */
typedef struct cvd_server cvd_server;

typedef struct {
    uint32_t guest;        /* index into the server's guest array */
    uint32_t dir;          /* 0 copy from guest, 1 copy to guest */
    uint32_t nseg, pad;
    const cvd_seg *segs;   /* host array, copied by cvd_server_submit */
    const void *d_src;     /* copy to guest: device source of the request's L bytes,
                              read when the request's wave launches */
    uint64_t arrival_ns;   /* scheduled arrival (ns since the server epoch); the request
                              is not admitted earlier; 0 = already arrived */
    uint64_t tag;          /* caller's cookie, returned in the completion */
} cvd_server_req;

typedef struct {
    uint64_t ticket, tag;
    cvd_result res;
    uint64_t staging_off;  /* copy from guest: result bytes at d_staging + staging_off ... */
    uint64_t len;          /* ... of this length, held until cvd_server_release */
    uint64_t arrival_ns, admit_ns, launch_ns, complete_ns;   /* server-epoch times */
    uint32_t guest, dir;
    uint64_t wave_device_ns;   /* GPU time of the request's wave: from its first command
                                  to its last on the device (CUDA events) */
} cvd_server_done;

/* Start a server over the guests (all on the current device) and a caller-
 * owned staging arena.  Threads: one scheduler per stream, one completion
 * poller.  max_inflight bounds admitted-but-incomplete requests.  flags:
 * CVD_SERVER_AUTO_RELEASE frees copy-from results at completion (for callers
 * that do not read them, e.g. load generators); CVD_SERVER_TWO_STREAMS
 * spreads the guests over two streams. */
#define CVD_SERVER_AUTO_RELEASE (1u << 0)
#define CVD_SERVER_TWO_STREAMS  (1u << 1)
int cvd_server_create(cvd_guest *const *guests, uint32_t nguests, void *d_staging, uint64_t staging_bytes,
                      uint32_t max_batch, uint32_t max_inflight, uint32_t flags, cvd_server **out);
/* Current server-epoch time in ns. */
uint64_t cvd_server_now_ns(cvd_server *s);
/* Queue requests (non-blocking); tickets[n] receives their ids.  EINVAL for a
 * bad guest/dir, a request longer than the arena, or copy-to without source. */
int cvd_server_submit(cvd_server *s, const cvd_server_req *reqs, uint32_t n, uint64_t *tickets);
/* Up to max completions; waits at most timeout_us for the first one
 * (CVD_ETIMEDOUT if none).  A CUDA failure inside the server is returned here. */
int cvd_server_poll(cvd_server *s, cvd_server_done *out, uint32_t max, uint32_t *n_out, uint32_t timeout_us);
/* Give back the staging range of a completed copy-from request. */
int cvd_server_release(cvd_server *s, uint64_t ticket);
/* Stop admitting, finish launched waves, join the threads, free the server. */
int cvd_server_destroy(cvd_server *s);

/* Copy-engine launch parameters (the autotuner's search space). */
typedef struct {
    uint32_t vec_bytes;       /* engine 0: 4, 8 or 16, width of the realigned vector moves */
    uint32_t unroll;          /* engine 0: vectors in flight per lane (see cvd_set_copy_params) */
    uint32_t chunk_bytes;     /* byte-balanced work unit (one warp), power of two
                                 4 KiB..1 MiB; smaller = more warps per segment */
    uint32_t blocks_per_sm;   /* persistent grid = blocks_per_sm x SM count, 1..16 */
    uint32_t warps_per_block; /* 4 or 8 (engine 0); 1..32 (engine 1) */
    uint32_t small_bytes;     /* segments up to this size are copied lane-locally (<= 4096) */
    uint32_t engine;          /* 0: register realignment; 1 (default): per-warp ring of
                                 shared-memory stages filled by bulk (TMA) copies */
    uint32_t stages;          /* engine 1: pieces in flight per warp, 1..32 */
    uint32_t stage_bytes;     /* engine 1: largest piece, multiple of 16, 512..32768 */
    uint32_t ring_bytes;      /* engine 1: per-warp shared-memory byte ring holding the
                                 pieces' source windows, multiple of 128, at least
                                 stage_bytes + 32 rounded up to 128; warps x ring must
                                 fit in shared memory */
} cvd_copy_params;

/* Current parameters (defaults until set or tuned). */
int cvd_get_copy_params(cvd_copy_params *p);
/* Set parameters; EINVAL if outside the search space.  (vec_bytes, unroll)
 * must be one of (16,1) (16,2) (16,4) (8,2) (8,4) (4,4). */
int cvd_set_copy_params(const cvd_copy_params *p);
/* Autotune: run the HAZARD_FREE batch `reps` times under every candidate in
 * the search space, keep the fastest (CUDA-event timed), set it, and return
 * it in *best (and its time in *best_ms).  The batch is executed repeatedly:
 * use a batch whose repetition is harmless.  Synchronises the stream. */
int cvd_tune(cvd_guest *const *guests, uint32_t nguests, const cvd_req *d_req, uint32_t nreq,
             const cvd_seg *d_seg, uint64_t nseg, void *d_host_buf, uint64_t host_buf_bytes,
             cvd_result *d_res, uint32_t reps, cvd_stream_t stream,
             cvd_copy_params *best, float *best_ms);

/* Autotune the planned-ahead step itself (no counterpart in the paper): time
 * whole cvd_copy_batches calls over `batches` (planning of batch i + 1
 * beside the copy of batch i, the copies leaving SMs to that planning),
 * `reps` times after one warm-up, under every candidate of the bulk-copy
 * engine's space -- ring shape, chunk size (how many warps share a long
 * segment) and the largest segment copied lane-locally instead of through
 * the bulk-copy ring -- and keep the fastest for the current device.  The
 * batches run 1 + reps times per candidate: use batches whose repetition is
 * harmless (hazard-free batches that only copy are).  Results are cached
 * by (GPU name, number of guests, paging / second dimension, number of
 * batches, log2 of total requests, total segments and staging bytes): a
 * repeated shape returns the cached choice without timing (*cached = 1).
 * With the environment variable CVD_TUNE_CACHE naming a file, the cache is
 * read from it at the first call and every new choice is appended to it.
 * Errors: as cvd_copy_batches (EINVAL for no batches).  Synchronises the
 * stream. */
int cvd_tune_batches(cvd_guest *const *guests, uint32_t nguests, const cvd_dev_batch *batches,
                     uint32_t nbatches, void *d_host_buf, uint64_t host_buf_bytes, uint32_t reps,
                     cvd_stream_t stream, cvd_copy_params *best, float *best_ms, int *cached);

/* Kernel timing.  While enabled, every hazard-free batch call that is not
 * replayed from a graph records CUDA events on its stream around its planner
 * launches (request sizing, scan, plan) and around its copy-engine launch;
 * every mmap install (cvd_mmap_install, and the install step of
 * cvd_mmap_place) around its probe launch (the walk of every page and the
 * ownership inserts), and every cvd_mmap_place with a shared-memory extent
 * tree around its first-fit launch. */
typedef struct {
    double plan_ms, copy_ms;        /* summed event-to-event device time */
    uint64_t plan_calls, copy_calls;
    double map_probe_ms, place_fit_ms;
    uint64_t map_probe_calls, place_fit_calls;
} cvd_profile;
int cvd_profile_enable(int on);
/* Waits for the recorded events, returns the sums since enabling or the
 * last read, and resets them. */
int cvd_profile_read(cvd_profile *out);

/* Kernels report internal failures (a bounded wait that gave up) in a
 * per-stream device error word instead of trapping.  Synchronises the stream,
 * returns the bits (1 = a wait timed out) and clears them.  The bits of
 * cvd_copy_batch_noalloc's own word on the current device (set by calls on
 * any stream since it was last taken) are ORed in and cleared too. */
int cvd_stream_check(cvd_stream_t stream, uint32_t *error_bits);

/* Self-test of that reporting path (no counterpart in the paper): launches
 * one warp on `stream` whose bounded mbarrier wait cannot complete (one of
 * two arrivals), so it gives up after `tries` attempts (1..2^22) and sets bit
 * 1 in the stream's error word; then returns like cvd_stream_check (*error_bits
 * = 1, word cleared).  Nothing faults or hangs and the context stays usable.
 * CVD_EINVAL on a null pointer or tries out of range. */
int cvd_selftest_wait_timeout(cvd_stream_t stream, uint32_t tries, uint32_t *error_bits);

/* Levels of the last levelled call on this stream (statistics): 1 when every
 * request ran in the one parallel launch; 2 when requests marked by the
 * conflict check then ran in order on the device; 1 + the byte-exact
 * levels of their runs when they were levelled on the host.  After a
 * HAZARD_FREE | CHECK call, the levels of the byte-exact leveller (more
 * than 1: CVD_EHAZARD).  May synchronise the stream. */
int cvd_last_levels(cvd_stream_t stream, uint32_t *levels);

/* The byte-exact leveller of the host path above, on its own (no CUDA call):
 * the runs are copies in stream order -- dst written, src read (0: a zero
 * fill, nothing read), len bytes each -- and levels[i] gets 1 + the highest
 * level of an earlier run that touches a common byte with run i, one of the
 * two writing it (0 when none), so running the levels in order gives the
 * sequential result.  *marked gets the number of runs with a range in a
 * cluster of overlapping ranges (sorted by address) that holds two or more
 * ranges, one written: the runs that can conflict at all.  Returns the
 * highest level (0 with nothing to order), CVD_EINVAL for null pointers
 * (n > 0) or a range that wraps past 2^64, CVD_ENOMEM when host scratch
 * cannot be had. */
typedef struct {
    uint64_t dst, src, len, pad;
} cvd_run;
int cvd_level_runs(const cvd_run *runs, uint64_t n, int32_t *levels, uint64_t *marked);

/* Kernel launches the library enqueued since load (all streams). */
uint64_t cvd_launch_count(void);

/* Dependent-load latency probe (no counterpart in the paper: it measures the
 * L2-hit and DRAM latencies that bound the software page walk of Sec. 4.2, so
 * walk throughput can be stated against a latency roofline).  Writes a chain
 * into the caller's device buffer d_buf (128-byte aligned; the largest
 * power-of-two number of 128-byte slots that fits in `bytes` is used, at
 * least 2): slot i points to slot (a*i + c) mod N, one cycle through all
 * slots.  One thread then follows the chain with L2-only loads, each address
 * taken from the previous load, for up to 2^20 warm-up steps and `steps`
 * timed steps (global timer).  *ns_per_load = timed ns / steps.  A buffer much
 * smaller than the L2 measures an L2 hit, one much larger a DRAM access.
 * Synchronises the stream; the buffer's contents are overwritten.  Errors:
 * CVD_EINVAL (null pointers, steps == 0, misaligned or too small buffer),
 * CVD_ENOMEM, CVD_ECUDA. */
int cvd_probe_latency(void *d_buf, uint64_t bytes, uint32_t steps, cvd_stream_t stream, double *ns_per_load);

/* Launch shape of cvd_translate for guest g (NULL: a guest whose memslots
 * are searched) on the current device: resident threads per SM and the walks
 * each thread keeps in flight (with the probe's latencies this gives the
 * translation's latency roofline).  A memslot guest (4-level or PAE) whose
 * memslots all lie on 2 MiB guest-frame boundaries below 32 GiB is
 * translated with per-2 MiB lookup tables in shared memory, whose size sets
 * the occupancy.  CVD_EINVAL
 * on null output pointers, CVD_ECUDA if the occupancy query fails. */
int cvd_translate_shape(const cvd_guest *g, uint32_t *resident_threads_per_sm, uint32_t *walks_per_thread);

const char *cvd_strerror(int status);
/* The CUDA error code behind the last CVD_ECUDA on this thread. */
int cvd_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CVD_H */
