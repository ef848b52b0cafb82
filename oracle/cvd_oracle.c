/*
 * CPU oracle for the CVD memory operations -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * this file.  It is a plain, slow, single-threaded restatement of what the
 * software hybrid address space computes (Sec. 4.2, Sec. 6.2), written for a
 * reader to check against the paper by eye.  It shares no code, header or
 * constant table with the CUDA library.
 *
 * Paper facts restated here:
 *  - A guest user buffer at a guest virtual address is reached by walking the
 *    guest page tables in software to a guest-physical address, which KVM's
 *    memslots turn into a host address (Sec. 4.2, "The CVD backend translates
 *    a guest virtual address ...").
 *  - Translation is done once per page, because pages that are contiguous in
 *    the guest virtual space need not be contiguous on the host (Sec. 4.2).
 *  - The page-table root is the location captured when the guest process
 *    first calls (Sec. 6.3); here it is the guest's cr3 guest-physical address.
 *  - Mapping a page into the guest (insert_pfn, Sec. 6.2) writes a guest PTE
 *    to a guest-physical frame the guest OS does not use (reserved through
 *    the hypervisor) and the second-dimension map from that frame to the host
 *    frame; new page-table pages come from a pool the frontend handed over at
 *    initialisation (Sec. 4.2, last paragraphs).
 *  - Without KVM the second dimension is finished by walking the EPT in
 *    software (Sec. 4.2, on other hypervisors); a guest may carry an EPT
 *    root instead of relying on memslots (Intel SDM Vol. 3 sec. 28.3.2).
 *
 * Readings of points the paper leaves open (x86-64 4-level format per the
 * Intel SDM Vol. 3 ch. 4; fault order; partial-copy semantics; allocation
 * order) are the ones listed in the design notes and are restated at each
 * function below.
 *
 * Parity: pinned by the CPU tests (identity and permutation maps, 2 MiB leaf
 * = 512 frames, hand-encoded tables with one fault per level, round trips,
 * per-byte = per-page, mmap closed forms and a hand-computed 2-page install;
 * for PAE guests hand-encoded tables and the generator's page record; for the
 * EPT hand-encoded guest + EPT tables, EPT mode = memslot mode on an EPT that
 * maps what the memslots map, and planted EPT faults against the record;
 * for driver-initiated maps closed forms on empty tables, hand-built holes,
 * and a brute-force first-fit checker over free pages taken from the walk;
 * for chained gathers identity-map closed forms, hand-placed faults at both
 * levels, and every payload byte re-derived through the walk).
 * The paper prints no worked example, so nothing pins it to printed values.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- records (little-endian, same byte layout as the generator's dtypes) */
typedef struct { uint64_t base_gfn, npages, host_off; } o_slot;
typedef struct { uint64_t gva, len; } o_seg;
typedef struct { uint32_t seg_begin, seg_count, dir, guest; uint64_t host_off; } o_req;
typedef struct { uint64_t done, fault_gva; uint32_t fault_code, pad; } o_res;
typedef struct { uint64_t gva; uint32_t npages, flags; uint64_t hf_begin; } o_map;
typedef struct { uint32_t npages, flags; uint64_t hf_begin; } o_place;

typedef struct {
    uint8_t *pool;            /* host memory that holds every memslot */
    uint64_t pool_bytes;
    const o_slot *slots;
    uint32_t nslots;
    uint32_t paging;          /* 0: x86-64 4-level, 1: 32-bit PAE (3 levels) */
    uint64_t cr3_gpa;         /* guest-physical address of the top table */
    uint64_t pt_pool_gfn, pt_pool_n, pt_used;   /* frontend's PT-page pool */
    uint64_t rsv_gfn, rsv_n, rsv_used;          /* reserved guest frames */
    uint64_t *p2m;            /* reserved frame -> host frame, ~0 = unmapped */
    uint32_t ept, pad2;       /* 1: the second dimension is a software EPT walk, not memslots */
    uint64_t ept_root;        /* host-pool byte offset of the EPT PML4 (4 KiB aligned) */
} o_guest;

/* fault codes */
enum { F_OK = 0, F_NOT_PRESENT = 1, F_WRITE_PROTECT = 2, F_NONCANONICAL = 3,
       F_RANGE = 4, F_NOSLOT = 5, F_RSVD = 6, F_USER = 7, F_HOSTBUF = 8, F_BADREQ = 9,
       F_EPT_VIOLATION = 10 };
/* per-page mmap status */
enum { S_OK = 0, S_EBUSY = -16, S_ENOMEM = -12, S_EINVAL = -22, S_EFAULT = -14 };

#define PAGE 4096ull
#define USER_TOP (1ull << 47)
#define NO_FRAME (~0ull)

static uint64_t load_u64(const uint8_t *p);

/*
 * Second dimension without KVM (Sec. 4.2: with other hypervisors a software
 * walk of the EPT finishes the translation; Sec. 2.2: two-dimensional paging
 * translates guest-physical to system-physical addresses).  Format per the
 * Intel SDM Vol. 3 sec. 28.3.2: a 4-level table in host memory indexed by gPA
 * bits 47:39 / 38:30 / 29:21 / 20:12; an entry is usable when its read bit
 * (bit 0) is set; bit 1 (write) is ANDed over the levels; bit 7 at level 3 /
 * 2 makes a 1 GiB / 2 MiB leaf and is reserved at level 4 (unusable);
 * addresses are bits 51:12 (51:30, 51:21 for leaves) and here they are host
 * pool byte offsets.  A page is backed only when its whole 4 KiB host frame
 * lies inside the pool (as memslots and p2m frames must).  Returns F_OK with
 * *host set, F_NOSLOT when no usable mapping reaches such a frame, or
 * F_EPT_VIOLATION for a write through a mapping without write permission.
 */
static uint32_t ept_to_host(const o_guest *g, uint64_t gpa, int write, uint64_t *host)
{
    if (gpa >> 48) return F_NOSLOT;
    uint64_t table = g->ept_root;
    int w = 1;
    for (int level = 4; level >= 1; level--) {
        unsigned idx = (unsigned)((gpa >> (12 + 9 * (level - 1))) & 511);
        if (table + 8ull * idx + 8 > g->pool_bytes) return F_NOSLOT;
        uint64_t e = load_u64(g->pool + table + 8ull * idx);
        if (!(e & 1)) return F_NOSLOT;
        w &= (e >> 1) & 1;
        uint64_t h = 0;
        int leaf = 0;
        if (level == 4 && (e & (1ull << 7))) return F_NOSLOT;
        if (level == 3 && (e & (1ull << 7))) { h = (e & 0x000FFFFFC0000000ull) | (gpa & ((1ull << 30) - 1)); leaf = 1; }
        if (level == 2 && (e & (1ull << 7))) { h = (e & 0x000FFFFFFFE00000ull) | (gpa & ((1ull << 21) - 1)); leaf = 1; }
        if (level == 1) { h = (e & 0x000FFFFFFFFFF000ull) | (gpa & 4095); leaf = 1; }
        if (leaf) {
            if ((h & ~(PAGE - 1)) + PAGE > g->pool_bytes) return F_NOSLOT;
            if (write && !w) return F_EPT_VIOLATION;
            *host = h;
            return F_OK;
        }
        table = e & 0x000FFFFFFFFFF000ull;
    }
    return F_NOSLOT;
}

/* ---- guest-physical -> host (Sec. 4.2: KVM turns a gPA into a host address) */
/* Returns 1 and sets *host if the guest frame is backed, else 0.  Reserved
 * frames (mapped by mmap installs) are looked up in the p2m array; every
 * other frame through the memslot whose frame range contains it. */
static uint32_t gpa_to_host_code(const o_guest *g, uint64_t gpa, int write, uint64_t *host)
{
    uint64_t gfn = gpa / PAGE, off = gpa % PAGE;
    if (gfn >= g->rsv_gfn && gfn - g->rsv_gfn < g->rsv_n) {
        uint64_t hf = g->p2m[gfn - g->rsv_gfn];
        if (hf == NO_FRAME || hf >= g->pool_bytes / PAGE) return F_NOSLOT;
        *host = hf * PAGE + off;
        return F_OK;
    }
    if (g->ept) return ept_to_host(g, gpa, write, host);
    for (uint32_t i = 0; i < g->nslots; i++) {
        const o_slot *s = &g->slots[i];
        if (gfn >= s->base_gfn && gfn - s->base_gfn < s->npages) {
            *host = s->host_off + (gpa - s->base_gfn * PAGE);
            return F_OK;
        }
    }
    return F_NOSLOT;
}

/* Read access of a table entry or a frame: 1 and *host if backed. */
static int gpa_to_host(const o_guest *g, uint64_t gpa, uint64_t *host)
{
    return gpa_to_host_code(g, gpa, 0, host) == F_OK;
}


static uint64_t load_u64(const uint8_t *p)
{
    uint64_t v = 0;
    for (int i = 7; i >= 0; i--) v = (v << 8) | p[i];
    return v;
}

static void store_u64(uint8_t *p, uint64_t v)
{
    for (int i = 0; i < 8; i++) { p[i] = (uint8_t)v; v >>= 8; }
}

/* Read entry `idx` of the page table at guest-physical `table_gpa`: page
 * tables live in guest memory, so they are reached through the memslots. */
static int read_entry(const o_guest *g, uint64_t table_gpa, unsigned idx, uint64_t *e)
{
    uint64_t h;
    if (!gpa_to_host(g, table_gpa + 8ull * idx, &h)) return 0;
    *e = load_u64(g->pool + h);
    return 1;
}

#define BIT_P  (1ull << 0)
#define BIT_RW (1ull << 1)
#define BIT_US (1ull << 2)
#define BIT_PS (1ull << 7)
#define FRAME_4K (0x000FFFFFFFFFF000ull)   /* bits 51:12 */
#define FRAME_2M (0x000FFFFFFFE00000ull)   /* bits 51:21 */
#define FRAME_1G (0x000FFFFFC0000000ull)   /* bits 51:30 */

static int canonical(uint64_t va)
{
    uint64_t top = va >> 47;             /* bits 63:47 must be all 0 or all 1 */
    return top == 0 || top == 0x1FFFF;
}

/* Address checks of a guest's virtual space: a 4-level guest's user buffers
 * lie in the canonical lower half [0, 2^47); a 32-bit PAE guest has no
 * non-canonical addresses and its whole space is [0, 2^32). */
static int va_canonical(const o_guest *g, uint64_t va) { return g->paging == 1 || canonical(va); }
static uint64_t va_top(const o_guest *g) { return g->paging == 1 ? (1ull << 32) : USER_TOP; }

/*
 * Software walk of a 32-bit PAE guest (the paging mode of the paper's own
 * implementation, Sec. 6.2; format per the Intel SDM Vol. 3 sec. 4.4).
 * cr3 holds the 32-byte aligned guest-physical address of the 4-entry page
 * directory pointer table; indexes are va bits 31:30, 29:21, 20:12.
 * Levels, top-down: PDPTE (3), PDE (2), PTE (1).  P=0 -> NOT_PRESENT with the
 * level in bits 8..11.  A PDPTE has no RW/US/PS bits: bits 1, 2 and 5..8 are
 * reserved there, and a present PDPTE with any of them set -> RSVD.  PS=1 in a
 * PDE -> 2 MiB leaf.  RW and US are ANDed over the PDE and PTE; then USER,
 * WRITE_PROTECT and the gPA backing as in the 4-level walk.  A va at or above
 * 2^32 -> RANGE.
 */
#define PAE_PDPTE_RSVD ((1ull << 1) | (1ull << 2) | (0xFull << 5))

static uint32_t oracle_walk_pae(const o_guest *g, uint64_t va, int write, uint64_t *gpa_out, uint64_t *hpa_out)
{
    if (va >= (1ull << 32)) return F_RANGE;
    unsigned i3 = (unsigned)((va >> 30) & 3), i2 = (unsigned)((va >> 21) & 511), i1 = (unsigned)((va >> 12) & 511);
    uint64_t e;
    /* PDPTE */
    if (!read_entry(g, g->cr3_gpa & ~31ull, i3, &e)) return F_NOSLOT;
    if (!(e & BIT_P)) return F_NOT_PRESENT | (3u << 8);
    if (e & PAE_PDPTE_RSVD) return F_RSVD;
    /* PDE */
    if (!read_entry(g, e & FRAME_4K, i2, &e)) return F_NOSLOT;
    if (!(e & BIT_P)) return F_NOT_PRESENT | (2u << 8);
    int rw = (e & BIT_RW) != 0, us = (e & BIT_US) != 0;
    uint64_t gpa;
    if (e & BIT_PS) {
        gpa = (e & FRAME_2M) | (va & ((1ull << 21) - 1));
    } else {
        /* PTE */
        if (!read_entry(g, e & FRAME_4K, i1, &e)) return F_NOSLOT;
        if (!(e & BIT_P)) return F_NOT_PRESENT | (1u << 8);
        rw &= (e & BIT_RW) != 0;
        us &= (e & BIT_US) != 0;
        gpa = (e & FRAME_4K) | (va & (PAGE - 1));
    }
    if (!us) return F_USER;
    if (write && !rw) return F_WRITE_PROTECT;
    uint64_t h;
    uint32_t c = gpa_to_host_code(g, gpa, write, &h);   /* the data page: read or write access */
    if (c != F_OK) return c;
    *gpa_out = gpa;
    *hpa_out = h;
    return F_OK;
}

/*
 * Software page walk of one guest virtual address (Sec. 4.2, Sec. 6.2-6.3).
 * x86-64 4-level reading: indexes are va bits 47:39, 38:30, 29:21, 20:12.
 * Per level, top-down: P=0 -> NOT_PRESENT with the level in bits 8..11;
 * PS=1 at level 4 -> RSVD; PS=1 at level 3 / 2 -> 1 GiB / 2 MiB leaf.
 * RW and US are ANDed over the visited levels; after the leaf, US=0 -> USER,
 * then (for a write) RW=0 -> WRITE_PROTECT; finally the gPA must be backed
 * (memslot or mapped reserved frame) -> else NOSLOT.  A table that is not in
 * a memslot also gives NOSLOT.  The walk never writes (no A/D updates).
 * On any fault *gpa and *hpa are set to all ones.
 */
uint32_t oracle_walk(const o_guest *g, uint64_t va, int write, uint64_t *gpa_out, uint64_t *hpa_out)
{
    *gpa_out = NO_FRAME;
    *hpa_out = NO_FRAME;
    if (g->paging == 1) return oracle_walk_pae(g, va, write, gpa_out, hpa_out);
    if (!canonical(va)) return F_NONCANONICAL;
    if (va >= USER_TOP) return F_RANGE;
    unsigned idx[5];
    idx[4] = (unsigned)((va >> 39) & 511);
    idx[3] = (unsigned)((va >> 30) & 511);
    idx[2] = (unsigned)((va >> 21) & 511);
    idx[1] = (unsigned)((va >> 12) & 511);
    uint64_t table = g->cr3_gpa & FRAME_4K;
    int rw = 1, us = 1;
    uint64_t gpa = 0;
    for (int level = 4; level >= 1; level--) {
        uint64_t e;
        if (!read_entry(g, table, idx[level], &e)) return F_NOSLOT;
        if (!(e & BIT_P)) return F_NOT_PRESENT | ((uint32_t)level << 8);
        rw &= (e & BIT_RW) != 0;
        us &= (e & BIT_US) != 0;
        if (level == 4 && (e & BIT_PS)) return F_RSVD;
        if (level == 3 && (e & BIT_PS)) { gpa = (e & FRAME_1G) | (va & ((1ull << 30) - 1)); break; }
        if (level == 2 && (e & BIT_PS)) { gpa = (e & FRAME_2M) | (va & ((1ull << 21) - 1)); break; }
        if (level == 1) { gpa = (e & FRAME_4K) | (va & (PAGE - 1)); break; }
        table = e & FRAME_4K;
    }
    if (!us) return F_USER;
    if (write && !rw) return F_WRITE_PROTECT;
    uint64_t h;
    uint32_t c = gpa_to_host_code(g, gpa, write, &h);   /* the data page: read or write access */
    if (c != F_OK) return c;
    *gpa_out = gpa;
    *hpa_out = h;
    return F_OK;
}

void oracle_translate(const o_guest *g, const uint64_t *va, uint64_t n, int write,
                      uint64_t *gpa, uint64_t *hpa, uint32_t *code)
{
    for (uint64_t i = 0; i < n; i++) code[i] = oracle_walk(g, va[i], write, &gpa[i], &hpa[i]);
}

/* ---- forwarded read/write buffers (Sec. 4.2, first category of routines) ---
 *
 * A request is a list of segments whose bytes, concatenated in order, form a
 * stream of L bytes tied to the staging range [host_off, host_off + L).
 * dir 0 (copy_from_user): guest -> staging; dir 1 (copy_to_user): staging ->
 * guest, which additionally needs writable pages.  The bytes before the first
 * faulting byte are copied; nothing after it.  copy-from zero-fills the rest
 * of its staging range; copy-to leaves the guest untouched after the fault.
 * done = offset of the first faulting byte (L if none).  Per segment, before
 * any of its bytes is walked: a non-canonical start -> NONCANONICAL, a range
 * reaching past the user half -> RANGE, both at the segment's first byte.
 * Zero-length segments are no-ops.
 *
 * Requests of one call run in index order (sequential semantics).  All
 * translations of a call see the page tables as they were when the call
 * started (translate first, then copy).
 *
 * Malformed requests: dir > 1, guest index out of range or a segment range
 * outside the segment array -> BADREQ; staging range outside the staging
 * buffer -> HOSTBUF; and, counting seg_count over the requests that passed
 * those two checks, a request whose running total exceeds the segment array
 * length -> BADREQ.  Such a request copies and zero-fills nothing, done = 0.
 */
typedef struct { uint64_t host; uint64_t len; } span;

typedef struct {
    span *v;
    size_t n, cap;
} spanvec;

static int push(spanvec *s, uint64_t host, uint64_t len)
{
    if (s->n && s->v[s->n - 1].host + s->v[s->n - 1].len == host) {
        s->v[s->n - 1].len += len;            /* merge host-contiguous bytes */
        return 1;
    }
    if (s->n == s->cap) {
        size_t c = s->cap ? 2 * s->cap : 64;
        span *nv = (span *)realloc(s->v, c * sizeof(span));
        if (!nv) return 0;
        s->v = nv;
        s->cap = c;
    }
    s->v[s->n].host = host;
    s->v[s->n].len = len;
    s->n++;
    return 1;
}

static uint64_t sat_add(uint64_t a, uint64_t b) { return a + b < a ? ~0ull : a + b; }

/* Returns 0 on success, -12 if host memory for the span lists ran out. */
int oracle_copy_batch(o_guest *const *guests, uint32_t nguests, const o_req *reqs, uint32_t nreq,
                      const o_seg *segs, uint64_t nseg, uint8_t *stg, uint64_t stg_bytes,
                      o_res *res, int per_byte)
{
    spanvec *tr = (spanvec *)calloc(nreq ? nreq : 1, sizeof(spanvec));
    uint8_t *ok = (uint8_t *)calloc(nreq ? nreq : 1, 1);
    uint64_t *L = (uint64_t *)calloc(nreq ? nreq : 1, sizeof(uint64_t));
    if (!tr || !ok || !L) { free(tr); free(ok); free(L); return -12; }
    int rc = 0;
    uint64_t seg_total = 0;

    /* validation, in request order */
    for (uint32_t r = 0; r < nreq; r++) {
        const o_req *q = &reqs[r];
        o_res *o = &res[r];
        o->done = 0; o->fault_gva = 0; o->fault_code = F_OK; o->pad = 0;
        if (q->dir > 1 || q->guest >= nguests ||
            (uint64_t)q->seg_begin + q->seg_count > nseg) { o->fault_code = F_BADREQ; continue; }
        uint64_t len = 0;
        for (uint32_t k = 0; k < q->seg_count; k++) len = sat_add(len, segs[q->seg_begin + k].len);
        if (len > stg_bytes || q->host_off > stg_bytes - len) { o->fault_code = F_HOSTBUF; continue; }
        seg_total += q->seg_count;
        if (seg_total > nseg) { o->fault_code = F_BADREQ; continue; }
        L[r] = len;
        ok[r] = 1;
    }

    /* phase 1: translate every request against the tables as they are now */
    for (uint32_t r = 0; r < nreq && rc == 0; r++) {
        if (!ok[r]) continue;
        const o_req *q = &reqs[r];
        const o_guest *g = guests[q->guest];
        o_res *o = &res[r];
        int write = q->dir == 1;
        uint64_t soff = 0;
        int faulted = 0;
        for (uint32_t k = 0; k < q->seg_count && !faulted; k++) {
            const o_seg *s = &segs[q->seg_begin + k];
            if (s->len == 0) continue;
            if (!va_canonical(g, s->gva)) { o->fault_code = F_NONCANONICAL; o->fault_gva = s->gva; o->done = soff; faulted = 1; break; }
            if (s->gva >= va_top(g) || s->len > va_top(g) - s->gva) { o->fault_code = F_RANGE; o->fault_gva = s->gva; o->done = soff; faulted = 1; break; }
            uint64_t j = 0;
            while (j < s->len) {
                uint64_t va = s->gva + j;
                /* once per page (Sec. 4.2); per byte in the brute-force mode */
                uint64_t chunk = per_byte ? 1 : PAGE - (va % PAGE);
                if (chunk > s->len - j) chunk = s->len - j;
                uint64_t gpa, hpa;
                uint32_t c = oracle_walk(g, va, write, &gpa, &hpa);
                if (c != F_OK) { o->fault_code = c; o->fault_gva = va; o->done = soff + j; faulted = 1; break; }
                if (!push(&tr[r], hpa, chunk)) { rc = -12; break; }
                j += chunk;
            }
            if (rc) break;
            soff += s->len;
        }
        if (!faulted) o->done = L[r];
    }

    /* phase 2: copy, requests in index order, bytes in stream order */
    for (uint32_t r = 0; r < nreq && rc == 0; r++) {
        if (!ok[r]) continue;
        const o_req *q = &reqs[r];
        uint8_t *pool = guests[q->guest]->pool;
        uint8_t *st = stg + q->host_off;
        uint64_t pos = 0;
        for (size_t i = 0; i < tr[r].n; i++) {
            span sp = tr[r].v[i];
            for (uint64_t b = 0; b < sp.len; b++) {
                if (q->dir == 0) st[pos + b] = pool[sp.host + b];
                else pool[sp.host + b] = st[pos + b];
            }
            pos += sp.len;
        }
        if (q->dir == 0)
            for (uint64_t b = res[r].done; b < L[r]; b++) st[b] = 0;
    }

    for (uint32_t r = 0; r < nreq; r++) free(tr[r].v);
    free(tr); free(ok); free(L);
    return rc;
}

/* ---- mmap install (Sec. 4.2 second category; insert_pfn, Sec. 6.2) -------
 *
 * Requests in index order, pages in order.  For page k of a request (va =
 * gva + 4096 k, host frame hf[hf_begin + k]):
 *   1. request malformed (va not page aligned, range outside the user half,
 *      hf range outside the hf array, or flag bits outside P|RW|US|PWT|PCD|G
 *      plus bit 31 = NX) -> EINVAL; a host frame outside the pool -> EINVAL.
 *   2. once any page ran out of memory, every later page -> ENOMEM.
 *   3. probe the path read-only: a present PS entry (level 4, 3 or 2) or a
 *      present leaf is in the way -> EBUSY; a present entry whose table is not
 *      in a memslot -> EFAULT.  Count the missing tables below the first
 *      non-present entry (3, 2, 1 or 0).
 *   4. if the PT pool lacks that many frames or the reserved window is used
 *      up -> ENOMEM (and latch 2); nothing of this page is written.
 *   5. otherwise create the missing tables top-down, each the next PT-pool
 *      frame, zeroed, linked as frame|P|RW|US; take the next reserved guest
 *      frame r; write the leaf r<<12 | P | (flags & RW|US|PWT|PCD|G) | NX<<63;
 *      set p2m[r - rsv_gfn] = hf.
 * A guest whose second dimension is an EPT gets EINVAL for every page.
 * A PAE guest walks 3 levels from its 4-entry PDPT and its user range is
 * [0, 2^32); a present PDPTE with reserved bits set is in the way (EBUSY);
 * a new page directory is linked from its PDPTE as frame|P (a PDPTE has no
 * RW/US bits).
 */
#define MAP_NX (1u << 31)
#define MAP_ALLOWED (0x1u | 0x2u | 0x4u | 0x8u | 0x10u | 0x100u | MAP_NX)

static int zero_frame(o_guest *g, uint64_t gfn)
{
    uint64_t h;
    if (!gpa_to_host(g, gfn * PAGE, &h)) return 0;
    memset(g->pool + h, 0, PAGE);
    return 1;
}

static int write_entry(o_guest *g, uint64_t table_gpa, unsigned idx, uint64_t e)
{
    uint64_t h;
    if (!gpa_to_host(g, table_gpa + 8ull * idx, &h)) return 0;
    store_u64(g->pool + h, e);
    return 1;
}

int oracle_mmap_install(o_guest *g, const o_map *reqs, uint32_t nreq, const uint64_t *hf,
                        uint64_t nhf, int32_t *status)
{
    int latch = 0;
    uint64_t out = 0;
    if (g->ept) {   /* installs into a guest behind an EPT are not supported: EINVAL */
        for (uint32_t r = 0; r < nreq; r++)
            for (uint32_t k = 0; k < reqs[r].npages; k++) status[out++] = S_EINVAL;
        return 0;
    }
    for (uint32_t r = 0; r < nreq; r++) {
        const o_map *q = &reqs[r];
        const uint64_t vtop = va_top(g);
        const int top = g->paging == 1 ? 3 : 4;
        int bad = (q->gva % PAGE) != 0 || q->gva >= vtop ||
                  (uint64_t)q->npages * PAGE > vtop - q->gva ||
                  q->hf_begin > nhf || q->npages > nhf - q->hf_begin ||
                  (q->flags & ~MAP_ALLOWED) != 0;
        for (uint32_t k = 0; k < q->npages; k++, out++) {
            uint64_t va = q->gva + (uint64_t)k * PAGE;
            if (bad) { status[out] = S_EINVAL; continue; }
            uint64_t frame = hf[q->hf_begin + k];
            if (frame >= g->pool_bytes / PAGE) { status[out] = S_EINVAL; continue; }
            if (latch) { status[out] = S_ENOMEM; continue; }
            unsigned idx[5];
            idx[4] = (unsigned)((va >> 39) & 511);
            idx[3] = (unsigned)((va >> 30) & 511);
            idx[2] = (unsigned)((va >> 21) & 511);
            idx[1] = (unsigned)((va >> 12) & 511);
            /* step 3: read-only probe */
            uint64_t table[5];
            table[top] = g->paging == 1 ? (g->cr3_gpa & ~31ull) : (g->cr3_gpa & FRAME_4K);
            int first_missing = 0;     /* level whose entry is non-present */
            int st = S_OK;
            for (int level = top; level >= 1; level--) {
                uint64_t e;
                if (!read_entry(g, table[level], idx[level], &e)) { st = S_EFAULT; break; }
                if (!(e & BIT_P)) { first_missing = level; break; }
                if (level == 1 || (e & BIT_PS)) { st = S_EBUSY; break; }
                if (g->paging == 1 && level == 3 && (e & PAE_PDPTE_RSVD)) { st = S_EBUSY; break; }
                table[level - 1] = e & FRAME_4K;
            }
            if (st != S_OK) { status[out] = st; continue; }
            uint64_t need = (uint64_t)(first_missing - 1);    /* tables below it */
            if (g->pt_used + need > g->pt_pool_n || g->rsv_used + 1 > g->rsv_n) {
                latch = 1;
                status[out] = S_ENOMEM;
                continue;
            }
            /* step 5: create tables top-down, then the leaf */
            for (int level = first_missing; level >= 2; level--) {
                uint64_t gfn = g->pt_pool_gfn + g->pt_used++;
                if (!zero_frame(g, gfn)) return -14;
                uint64_t link = (gfn * PAGE) | ((g->paging == 1 && level == 3) ? BIT_P : 0x7);
                if (!write_entry(g, table[level], idx[level], link)) return -14;
                table[level - 1] = gfn * PAGE;
            }
            uint64_t rg = g->rsv_gfn + g->rsv_used++;
            uint64_t leaf = (rg * PAGE) | BIT_P | (q->flags & (0x2u | 0x4u | 0x8u | 0x10u | 0x100u));
            if (q->flags & MAP_NX) leaf |= 1ull << 63;
            if (!write_entry(g, table[1], idx[1], leaf)) return -14;
            g->p2m[rg - g->rsv_gfn] = frame;
            status[out] = S_OK;
        }
    }
    return 0;
}

/* ---- driver-initiated mmap (Sec. 6.6) -------------------------------------
 *
 * A driver maps memory from inside an operation, so no guest virtual range
 * was chosen for it: the backend records the request, picks a range in the
 * guest and installs the map there.  Here one call takes requests
 * (npages, flags, hf_begin) without an address and a window [va_lo, va_hi):
 *   0. window not page aligned, empty, or past the guest's user range ->
 *      the call fails (EINVAL); a guest behind an EPT cannot take installs:
 *      every request gets no range and every page EINVAL.
 *   1. a page of the window is free when its walk, on the tables as they
 *      were at call start, meets a non-present entry (at any level) before
 *      a leaf; a present leaf, a present PS entry, a PAE PDPTE with reserved
 *      bits or a present entry whose table no memslot backs make it taken.
 *   2. requests in index order: a malformed one (npages 0, flag bits outside
 *      P|RW|US|PWT|PCD|G plus bit 31 = NX, or hf range outside the hf array)
 *      gets no range and EINVAL for its pages; otherwise its range is the
 *      lowest page-aligned address a with [a, a + 4096 npages) inside the
 *      window, every page free and in no range given to an earlier request
 *      of the call (first fit); with none, it gets no range and ENOSPC for
 *      its pages.
 *   3. the requests given a range are installed there, in index order, with
 *      the install's rules (oracle_mmap_install); their statuses take their
 *      places in the per-page status array (requests' pages in order).
 * gva_out[r] = the range's start, or all ones for no range.
 */
#define S_ENOSPC (-28)

static int page_free(const o_guest *g, uint64_t va)
{
    const int top = g->paging == 1 ? 3 : 4;
    uint64_t table = g->paging == 1 ? (g->cr3_gpa & ~31ull) : (g->cr3_gpa & FRAME_4K);
    for (int level = top; level >= 1; level--) {
        unsigned idx = (unsigned)((va >> (12 + 9 * (level - 1))) & 511);
        uint64_t e;
        if (!read_entry(g, table, idx, &e)) return 0;
        if (!(e & BIT_P)) return 1;
        if (level == 1 || (e & BIT_PS)) return 0;
        if (g->paging == 1 && level == 3 && (e & PAE_PDPTE_RSVD)) return 0;
        table = e & FRAME_4K;
    }
    return 0;
}

int oracle_mmap_place(o_guest *g, uint64_t va_lo, uint64_t va_hi, const o_place *reqs, uint32_t nreq,
                      const uint64_t *hf, uint64_t nhf, uint64_t *gva_out, int32_t *status)
{
    if ((va_lo % PAGE) || (va_hi % PAGE) || va_lo >= va_hi || va_hi > va_top(g)) return S_EINVAL;
    uint64_t npg = 0;
    for (uint32_t r = 0; r < nreq; r++) npg += reqs[r].npages;
    if (g->ept) {
        for (uint32_t r = 0; r < nreq; r++) gva_out[r] = NO_FRAME;
        for (uint64_t p = 0; p < npg; p++) status[p] = S_EINVAL;
        return 0;
    }
    const uint64_t W = (va_hi - va_lo) / PAGE;
    uint8_t *avail = (uint8_t *)malloc(W ? W : 1);
    o_map *maps = (o_map *)calloc(nreq ? nreq : 1, sizeof(o_map));
    int32_t *st = (int32_t *)malloc(sizeof(int32_t) * (npg ? npg : 1));
    if (!avail || !maps || !st) { free(avail); free(maps); free(st); return S_ENOMEM; }
    for (uint64_t p = 0; p < W; p++) avail[p] = (uint8_t)page_free(g, va_lo + p * PAGE);   /* step 1 */
    uint32_t nmap = 0;
    for (uint32_t r = 0; r < nreq; r++) {                                                 /* step 2 */
        const o_place *q = &reqs[r];
        gva_out[r] = NO_FRAME;
        if (q->npages == 0 || (q->flags & ~MAP_ALLOWED) || q->hf_begin > nhf || q->npages > nhf - q->hf_begin)
            continue;
        uint64_t run = 0;
        for (uint64_t p = 0; p < W; p++) {
            run = avail[p] ? run + 1 : 0;
            if (run == q->npages) {
                uint64_t first = p + 1 - run;
                for (uint64_t k = first; k <= p; k++) avail[k] = 0;
                gva_out[r] = va_lo + first * PAGE;
                break;
            }
        }
        if (gva_out[r] != NO_FRAME) {
            maps[nmap].gva = gva_out[r];
            maps[nmap].npages = q->npages;
            maps[nmap].flags = q->flags;
            maps[nmap].hf_begin = q->hf_begin;
            nmap++;
        }
    }
    int rc = oracle_mmap_install(g, maps, nmap, hf, nhf, st);                             /* step 3 */
    uint64_t out = 0, in = 0;
    for (uint32_t r = 0; r < nreq && rc == 0; r++) {
        const o_place *q = &reqs[r];
        int malformed = q->npages == 0 || (q->flags & ~MAP_ALLOWED) || q->hf_begin > nhf ||
                        q->npages > nhf - q->hf_begin;
        for (uint32_t k = 0; k < q->npages; k++, out++)
            status[out] = gva_out[r] != NO_FRAME ? st[in++] : (malformed ? S_EINVAL : S_ENOSPC);
    }
    free(avail); free(maps); free(st);
    return rc;
}

/* ---- dependent second-level gathers (Sec. 6.1-6.2, generic class drivers) --
 *
 * A DRM-style command submission passes a structure that holds further
 * guest pointers: the host driver copies the structure in, then gathers the
 * buffers it names.  Here a request names a descriptor table -- `count`
 * entries of {u64 gva, u64 len} at table_gva in its guest -- and the call:
 *   1. reads every request's table (copy_from, the rules of
 *      oracle_copy_batch) into desc[desc_off, desc_off + 16 count), all
 *      against guest memory as it was when the call started; a request with
 *      count above 65,536 or desc_off not a multiple of 16 is BADREQ; a
 *      fault here ends the request at level 1 (done = table bytes read);
 *   2. for the requests whose table was read whole, in index order: L =
 *      the saturating sum of the entries' len; the payload of request r
 *      goes at P_r = the (saturating) sum of the L of the earlier such
 *      requests, and its entries take places E_r = the sum of the counts of
 *      the earlier such requests in a list that holds desc_bytes / 16
 *      entries (the capacity of the descriptor buffer itself); it fits when
 *      P_r + L_r <= payload_bytes and E_r + count <= desc_bytes / 16 (the
 *      second can fail only when tables overlap in the descriptor buffer); a
 *      request that does not fit gets HOSTBUF at level 2 (payload_off 0,
 *      nothing copied);
 *   3. gathers each fitting request's entries, in order, as the segments of
 *      one copy_from request into payload[P_r, P_r + L_r) (first faulting
 *      byte ends it, the rest is zero-filled).
 * Result per request: done (payload bytes copied, or table bytes at level
 * 1), fault_gva, fault_code, level (0 = no fault, 1 = table, 2 = payload),
 * payload_off, payload_len (L; 0 when level 1 faulted).
 */
typedef struct { uint64_t table_gva; uint32_t count, guest; uint64_t desc_off; } o_chain_req;
typedef struct { uint64_t done, fault_gva; uint32_t fault_code, level; uint64_t payload_off, payload_len; } o_chain_res;
#define CHAIN_MAX_COUNT 65536u

int oracle_gather_chained(o_guest *const *guests, uint32_t nguests, const o_chain_req *reqs, uint32_t nreq,
                          uint8_t *desc, uint64_t desc_bytes, uint8_t *payload, uint64_t payload_bytes,
                          o_chain_res *res)
{
    uint32_t n = nreq ? nreq : 1;
    o_req *q1 = (o_req *)calloc(n, sizeof(o_req));
    o_seg *s1 = (o_seg *)calloc(n, sizeof(o_seg));
    o_res *r1 = (o_res *)calloc(n, sizeof(o_res));
    o_req *q2 = (o_req *)calloc(n, sizeof(o_req));
    o_res *r2 = (o_res *)calloc(n, sizeof(o_res));
    uint64_t total = 0;
    for (uint32_t r = 0; r < nreq; r++) total += reqs[r].count <= CHAIN_MAX_COUNT ? reqs[r].count : 0;
    o_seg *s2 = (o_seg *)calloc(total ? total : 1, sizeof(o_seg));
    if (!q1 || !s1 || !r1 || !q2 || !r2 || !s2) {
        free(q1); free(s1); free(r1); free(q2); free(r2); free(s2);
        return -12;
    }
    /* step 1: every table, as one copy_from request each */
    for (uint32_t r = 0; r < nreq; r++) {
        const int malformed = reqs[r].count > CHAIN_MAX_COUNT || (reqs[r].desc_off % 16) != 0;
        q1[r].seg_begin = r; q1[r].seg_count = 1; q1[r].dir = 0;
        q1[r].guest = malformed ? nguests : reqs[r].guest;      /* guest out of range: BADREQ */
        q1[r].host_off = reqs[r].desc_off;
        s1[r].gva = reqs[r].table_gva; s1[r].len = 16ull * reqs[r].count;
    }
    int rc = oracle_copy_batch(guests, nguests, q1, nreq, s1, nreq, desc, desc_bytes, r1, 0);
    /* step 2: payload lengths and places; the fitting tables become the
     * segment list of step 3, in request order */
    uint64_t cursor = 0, nseg = 0, epos = 0;
    const uint64_t ecap = desc_bytes / 16;
    for (uint32_t r = 0; r < nreq && rc == 0; r++) {
        o_chain_res *o = &res[r];
        memset(o, 0, sizeof(*o));
        q2[r].seg_begin = (uint32_t)nseg; q2[r].seg_count = 0; q2[r].dir = 0; q2[r].guest = reqs[r].guest;
        q2[r].host_off = 0;
        if (r1[r].fault_code != F_OK) {
            o->done = r1[r].done; o->fault_gva = r1[r].fault_gva; o->fault_code = r1[r].fault_code; o->level = 1;
            continue;
        }
        const uint8_t *t = desc + reqs[r].desc_off;
        uint64_t L = 0;
        for (uint32_t k = 0; k < reqs[r].count; k++) L = sat_add(L, load_u64(t + 16ull * k + 8));
        o->payload_len = L;
        const uint64_t end = sat_add(cursor, L);
        const uint64_t e0 = epos;
        epos += reqs[r].count;
        if (end > payload_bytes || e0 + reqs[r].count > ecap) {
            o->fault_code = F_HOSTBUF; o->level = 2; cursor = end; continue;
        }
        o->payload_off = cursor;
        cursor = end;
        for (uint32_t k = 0; k < reqs[r].count; k++) {
            s2[nseg + k].gva = load_u64(t + 16ull * k);
            s2[nseg + k].len = load_u64(t + 16ull * k + 8);
        }
        q2[r].seg_count = reqs[r].count;
        q2[r].host_off = o->payload_off;
        nseg += reqs[r].count;
    }
    /* step 3: the payload gathers */
    if (rc == 0) rc = oracle_copy_batch(guests, nguests, q2, nreq, s2, nseg, payload, payload_bytes, r2, 0);
    for (uint32_t r = 0; r < nreq && rc == 0; r++) {
        o_chain_res *o = &res[r];
        if (o->level != 0) continue;
        o->done = r2[r].done; o->fault_gva = r2[r].fault_gva; o->fault_code = r2[r].fault_code;
        if (o->fault_code != F_OK) o->level = 2;
    }
    free(q1); free(s1); free(r1); free(q2); free(r2); free(s2);
    return rc;
}
