"""Mutation check of the oracle's pins -- TEST INFRASTRUCTURE ONLY.

Each mutant plants one plausible mistake in a copy of ``cvd_oracle.c`` (a
dropped term, a wrong bound, a swapped check, a missing step), builds it with
the oracle's own flags, and runs the oracle's CPU pins against it through
``CVD_ORACLE_LIB``.  A mutant the pins do not fail "survived": a gap in the
pins.  Nothing here touches the CUDA library or a GPU.

Not listed: mistakes equivalent to the oracle on every input the pins can
build, such as masking a 1 GiB leaf's frame with the 2 MiB mask (they differ
only in bits 29:21, which a 1 GiB leaf keeps clear), or testing only an EPT
entry's first byte against the pool's end (the two differ only for a pool
that ends inside an entry).

    python -m oracle.mutants            # every mutant (~15 min on one core); exit 1 if one survives
    python -m oracle.mutants -k ept     # the mutants whose name contains "ept"
"""
from __future__ import annotations

import argparse
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "cvd_oracle.c")
PINS = sorted(os.path.join("tests", f) for f in os.listdir(os.path.join(ROOT, "tests"))
              if f.startswith("test_oracle_") and f.endswith(".py"))

# (name, text to find -- exactly once in the source, replacement, the pin files that should fail it)
MUTANTS = [
    # 4-level walk (Sec. 4.2 software walk; SDM Vol. 3 ch. 4)
    ("walk_rw_not_anded",
     "rw &= (e & BIT_RW) != 0;\n        us &= (e & BIT_US) != 0;\n        if (level == 4",
     "rw = (e & BIT_RW) != 0;\n        us &= (e & BIT_US) != 0;\n        if (level == 4", ["walk"]),
    ("walk_us_not_anded",
     "rw &= (e & BIT_RW) != 0;\n        us &= (e & BIT_US) != 0;\n        if (level == 4",
     "rw &= (e & BIT_RW) != 0;\n        us = (e & BIT_US) != 0;\n        if (level == 4", ["walk"]),
    ("walk_write_protect_before_user",
     "    if (!us) return F_USER;\n    if (write && !rw) return F_WRITE_PROTECT;\n    uint64_t h;\n"
     "    uint32_t c = gpa_to_host_code(g, gpa, write, &h);   /* the data page: read or write access */\n"
     "    if (c != F_OK) return c;\n    *gpa_out = gpa;\n    *hpa_out = h;\n    return F_OK;\n}\n\nvoid",
     "    if (write && !rw) return F_WRITE_PROTECT;\n    if (!us) return F_USER;\n    uint64_t h;\n"
     "    uint32_t c = gpa_to_host_code(g, gpa, write, &h);   /* the data page: read or write access */\n"
     "    if (c != F_OK) return c;\n    *gpa_out = gpa;\n    *hpa_out = h;\n    return F_OK;\n}\n\nvoid", ["walk"]),
    ("walk_ps_allowed_at_level_4", "if (level == 4 && (e & BIT_PS)) return F_RSVD;", "", ["walk"]),
    ("walk_2m_offset_mask", "gpa = (e & FRAME_2M) | (va & ((1ull << 21) - 1)); break;",
     "gpa = (e & FRAME_2M) | (va & ((1ull << 12) - 1)); break;", ["walk"]),
    ("walk_1g_offset_mask", "gpa = (e & FRAME_1G) | (va & ((1ull << 30) - 1)); break;",
     "gpa = (e & FRAME_1G) | (va & ((1ull << 21) - 1)); break;", ["walk"]),
    ("walk_fault_level_dropped", "return F_NOT_PRESENT | ((uint32_t)level << 8);", "return F_NOT_PRESENT;",
     ["walk"]),
    ("walk_noncanonical_not_checked", "if (!canonical(va)) return F_NONCANONICAL;\n", "", ["walk"]),
    ("memslot_end_inclusive", "gfn - s->base_gfn < s->npages", "gfn - s->base_gfn <= s->npages", ["walk"]),
    ("p2m_frame_outside_pool_accepted", "if (hf == NO_FRAME || hf >= g->pool_bytes / PAGE) return F_NOSLOT;",
     "if (hf == NO_FRAME) return F_NOSLOT;", ["mmap", "walk"]),
    # PAE (Sec. 6.2: the paper's own 32-bit paging; SDM Vol. 3 sec. 4.4)
    ("pae_pdpte_reserved_ignored", "if (e & PAE_PDPTE_RSVD) return F_RSVD;", "", ["pae"]),
    ("pae_rw_not_anded",
     "rw &= (e & BIT_RW) != 0;\n        us &= (e & BIT_US) != 0;\n        gpa = (e & FRAME_4K)",
     "rw = (e & BIT_RW) != 0;\n        us &= (e & BIT_US) != 0;\n        gpa = (e & FRAME_4K)", ["pae"]),
    ("pae_2m_offset_mask", "gpa = (e & FRAME_2M) | (va & ((1ull << 21) - 1));\n    } else {",
     "gpa = (e & FRAME_2M) | (va & ((1ull << 12) - 1));\n    } else {", ["pae"]),
    # software EPT (Sec. 4.2 other hypervisors; SDM Vol. 3 sec. 28.3.2)
    ("ept_write_not_anded", "w &= (e >> 1) & 1;", "w = (e >> 1) & 1;", ["ept"]),
    ("ept_bit7_allowed_at_level_4", "if (level == 4 && (e & (1ull << 7))) return F_NOSLOT;", "", ["ept"]),
    ("ept_byte_rule_instead_of_frame_rule", "if ((h & ~(PAGE - 1)) + PAGE > g->pool_bytes) return F_NOSLOT;",
     "if (h + 1 > g->pool_bytes) return F_NOSLOT;", ["ept"]),
    ("ept_violation_not_checked", "if (write && !w) return F_EPT_VIOLATION;", "", ["ept"]),
    # copies (Sec. 4.2 first category: copy_from_user / copy_to_user per page)
    ("copy_fault_offset_off_by_one", "o->done = soff + j; faulted = 1; break; }",
     "o->done = soff + j + 1; faulted = 1; break; }", ["copy"]),
    ("copy_from_no_zero_fill", "for (uint64_t b = res[r].done; b < L[r]; b++) st[b] = 0;", ";", ["copy"]),
    ("copy_hostbuf_bound", "q->host_off > stg_bytes - len", "q->host_off >= stg_bytes - len", ["copy"]),
    ("copy_range_end_not_checked", "if (s->gva >= va_top(g) || s->len > va_top(g) - s->gva)",
     "if (s->gva >= va_top(g))", ["copy"]),
    ("copy_to_ignores_write_protect", "int write = q->dir == 1;", "int write = 0;", ["copy"]),
    ("copy_segment_offsets_not_summed", "soff += s->len;", "soff += 0;", ["copy"]),
    # mmap install (Sec. 4.2 second category; insert_pfn, Sec. 6.2)
    ("mmap_no_enomem_latch", "if (latch) { status[out] = S_ENOMEM; continue; }", "", ["mmap"]),
    ("mmap_link_flags", "? BIT_P : 0x7)", "? BIT_P : 0x3)", ["mmap"]),
    ("mmap_nx_dropped", "if (q->flags & MAP_NX) leaf |= 1ull << 63;", "", ["mmap"]),
    ("mmap_ps_not_busy", "if (level == 1 || (e & BIT_PS)) { st = S_EBUSY; break; }",
     "if (level == 1) { st = S_EBUSY; break; }", ["mmap"]),
    ("mmap_new_tables_not_zeroed", "if (!zero_frame(g, gfn)) return -14;", "", ["mmap"]),
    ("mmap_tables_needed_off_by_one", "uint64_t need = (uint64_t)(first_missing - 1);",
     "uint64_t need = (uint64_t)(first_missing - 2);", ["mmap"]),
    ("mmap_p2m_not_written", "g->p2m[rg - g->rsv_gfn] = frame;", "", ["mmap"]),
    # driver-initiated maps (Sec. 6.6)
    ("place_ranges_not_marked_taken", "for (uint64_t k = first; k <= p; k++) avail[k] = 0;", "", ["place"]),
    ("place_enospc_as_einval", "(malformed ? S_EINVAL : S_ENOSPC)", "S_EINVAL", ["place"]),
    ("place_free_only_at_leaf_level", "if (!(e & BIT_P)) return 1;", "if (!(e & BIT_P)) return level == 1;",
     ["place"]),
    # chained gathers (Sec. 6.1 generic class drivers)
    ("chain_payload_places_not_summed", "o->payload_off = cursor;\n        cursor = end;",
     "o->payload_off = cursor;\n        cursor = cursor + 0;", ["chain"]),
    ("chain_alignment_rule", "(reqs[r].desc_off % 16) != 0", "(reqs[r].desc_off % 8) != 0", ["chain"]),
    # further bounds and masks
    ("pae_range_bound", "if (va >= (1ull << 32)) return F_RANGE;", "if (va > (1ull << 32)) return F_RANGE;",
     ["pae"]),
    ("pae_pdpt_index_bits", "(unsigned)((va >> 30) & 3)", "(unsigned)((va >> 30) & 1)", ["pae"]),
    ("ept_2m_leaf_offset", "(e & 0x000FFFFFFFE00000ull) | (gpa & ((1ull << 21) - 1))",
     "(e & 0x000FFFFFFFE00000ull) | (gpa & ((1ull << 12) - 1))", ["ept"]),
    ("ept_1g_leaf_offset", "(e & 0x000FFFFFC0000000ull) | (gpa & ((1ull << 30) - 1))",
     "(e & 0x000FFFFFC0000000ull) | (gpa & ((1ull << 21) - 1))", ["ept"]),
    ("p2m_window_end_inclusive", "gfn - g->rsv_gfn < g->rsv_n", "gfn - g->rsv_gfn <= g->rsv_n", ["walk", "mmap"]),
    ("copy_whole_page_chunks", "uint64_t chunk = per_byte ? 1 : PAGE - (va % PAGE);",
     "uint64_t chunk = per_byte ? 1 : PAGE;", ["copy"]),
    ("copy_shared_segments_bound", "if (seg_total > nseg)", "if (seg_total > nseg + 1)", ["copy"]),
    ("copy_zero_fill_start", "for (uint64_t b = res[r].done; b < L[r]; b++) st[b] = 0;",
     "for (uint64_t b = res[r].done + 1; b < L[r]; b++) st[b] = 0;", ["copy"]),
    ("copy_length_not_saturating", "return a + b < a ? ~0ull : a + b;", "return a + b;", ["copy", "chain"]),
    ("mmap_unaligned_va_accepted", "int bad = (q->gva % PAGE) != 0 || q->gva >= vtop ||",
     "int bad = q->gva >= vtop ||", ["mmap"]),
    ("mmap_host_frame_bound", "if (frame >= g->pool_bytes / PAGE) { status[out] = S_EINVAL; continue; }",
     "if (frame > g->pool_bytes / PAGE) { status[out] = S_EINVAL; continue; }", ["mmap"]),
    ("mmap_reserved_window_bound", "g->rsv_used + 1 > g->rsv_n", "g->rsv_used > g->rsv_n", ["mmap"]),
    ("chain_count_limit", "reqs[r].count > CHAIN_MAX_COUNT ||", "reqs[r].count > CHAIN_MAX_COUNT + 1 ||",
     ["chain"]),
    ("chain_entry_capacity", "e0 + reqs[r].count > ecap", "e0 + reqs[r].count > ecap + 1", ["chain"]),
    ("ept_48bit_gpa_not_checked", "if (gpa >> 48) return F_NOSLOT;", "", ["ept"]),
    ("ept_before_reserved_window", "if (gfn >= g->rsv_gfn && gfn - g->rsv_gfn < g->rsv_n) {",
     "if (!g->ept && gfn >= g->rsv_gfn && gfn - g->rsv_gfn < g->rsv_n) {", ["ept"]),
    ("pae_pde_ps_ignored", "    if (e & BIT_PS) {\n        gpa = (e & FRAME_2M)", "    if (0) {\n        gpa = (e & FRAME_2M)",
     ["pae"]),
    ("walk_pdpt_index_shift", "    idx[3] = (unsigned)((va >> 30) & 511);\n    idx[2] = (unsigned)((va >> 21) & 511);\n"
     "    idx[1] = (unsigned)((va >> 12) & 511);\n    uint64_t table = g->cr3_gpa & FRAME_4K;",
     "    idx[3] = (unsigned)((va >> 31) & 511);\n    idx[2] = (unsigned)((va >> 21) & 511);\n"
     "    idx[1] = (unsigned)((va >> 12) & 511);\n    uint64_t table = g->cr3_gpa & FRAME_4K;", ["walk"]),
    ("copy_zero_length_segments_checked", "if (s->len == 0) continue;", ";", ["copy"]),
    ("copy_pae_canonical_as_4level", "if (!va_canonical(g, s->gva)) { o->fault_code = F_NONCANONICAL;",
     "if (!canonical(s->gva)) { o->fault_code = F_NONCANONICAL;", ["copy", "pae"]),
    ("copy_guest_index_bound", "q->guest >= nguests ||", "q->guest > nguests ||", ["copy", "chain"]),
    ("mmap_global_bit_dropped", "(q->flags & (0x2u | 0x4u | 0x8u | 0x10u | 0x100u))",
     "(q->flags & (0x2u | 0x4u | 0x8u | 0x10u))", ["mmap"]),
    ("place_window_end_bound", "va_lo >= va_hi || va_hi > va_top(g)) return S_EINVAL;",
     "va_lo >= va_hi || va_hi > va_top(g) + PAGE) return S_EINVAL;", ["place"]),
    ("chain_payload_end_not_saturating", "const uint64_t end = sat_add(cursor, L);",
     "const uint64_t end = cursor + L;", ["chain"]),
    ("memslot_base_not_subtracted", "*host = s->host_off + (gpa - s->base_gfn * PAGE);",
     "*host = s->host_off + gpa;", ["walk", "copy"]),
    ("walk_unbacked_table_not_present", "if (!read_entry(g, table, idx[level], &e)) return F_NOSLOT;",
     "if (!read_entry(g, table, idx[level], &e)) return F_NOT_PRESENT | ((uint32_t)level << 8);", ["walk"]),
    ("mmap_range_end_bound", "(uint64_t)q->npages * PAGE > vtop - q->gva ||",
     "(uint64_t)q->npages * PAGE > vtop - q->gva + PAGE ||", ["mmap", "pae"]),
    ("mmap_hf_range_bound", "q->hf_begin > nhf || q->npages > nhf - q->hf_begin ||\n",
     "q->hf_begin > nhf || q->npages > nhf - q->hf_begin + 1 ||\n", ["mmap"]),
    ("mmap_present_leaf_not_busy", "if (level == 1 || (e & BIT_PS)) { st = S_EBUSY; break; }",
     "if (level == 1 && 0) { st = S_EBUSY; break; }", ["mmap"]),
    ("place_empty_request_placed", "if (q->npages == 0 || (q->flags & ~MAP_ALLOWED) || q->hf_begin > nhf",
     "if ((q->flags & ~MAP_ALLOWED) || q->hf_begin > nhf", ["place"]),
    ("chain_table_fault_done_dropped", "o->done = r1[r].done; o->fault_gva = r1[r].fault_gva;",
     "o->done = 0; o->fault_gva = r1[r].fault_gva;", ["chain"]),
    # orders the sequential semantics fix
    ("copy_requests_in_reverse_order",
     "    for (uint32_t r = 0; r < nreq && rc == 0; r++) {\n        if (!ok[r]) continue;\n"
     "        const o_req *q = &reqs[r];\n        uint8_t *pool",
     "    for (uint32_t r0 = 0; r0 < nreq && rc == 0; r0++) {\n        uint32_t r = nreq - 1 - r0;\n"
     "        if (!ok[r]) continue;\n        const o_req *q = &reqs[r];\n        uint8_t *pool", ["copy"]),
    ("mmap_pt_pool_from_the_top", "uint64_t gfn = g->pt_pool_gfn + g->pt_used++;",
     "uint64_t gfn = g->pt_pool_gfn + g->pt_pool_n - 1 - g->pt_used++;", ["mmap"]),
    ("mmap_reserved_frames_from_the_top", "uint64_t rg = g->rsv_gfn + g->rsv_used++;",
     "uint64_t rg = g->rsv_gfn + g->rsv_n - 1 - g->rsv_used++;", ["mmap"]),
    ("upper_half_called_noncanonical", "return top == 0 || top == 0x1FFFF;", "return top == 0;", ["walk", "copy"]),
    ("pae_pdpt_page_aligned", "if (!read_entry(g, g->cr3_gpa & ~31ull, i3, &e)) return F_NOSLOT;",
     "if (!read_entry(g, g->cr3_gpa & FRAME_4K, i3, &e)) return F_NOSLOT;", ["pae"]),
    ("mmap_pae_pdpte_linked_rw_us", "((g->paging == 1 && level == 3) ? BIT_P : 0x7)", "(0x7)", ["pae", "mmap"]),
]


def build_mutant(text: str, out_dir: str) -> str:
    src = os.path.join(out_dir, "cvd_oracle.c")
    lib = os.path.join(out_dir, "libcvd_oracle.so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", lib, src],
                          stderr=subprocess.DEVNULL)
    return lib


def mutate(source: str, find: str, replace: str) -> str:
    if source.count(find) != 1:
        raise ValueError(f"mutation site found {source.count(find)} times, expected once: {find[:60]!r}")
    return source.replace(find, replace)


def pins_fail(lib: str, pins: list[str]) -> bool:
    """Whether the pin files fail with the oracle replaced by `lib`."""
    env = dict(os.environ, CVD_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *pins],
                       cwd=ROOT, env=env, stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
    return r.returncode != 0


def run(names=None, all_pins=False) -> dict:
    source = open(SRC).read()
    out = {}
    with tempfile.TemporaryDirectory() as tmp:
        for name, find, replace, areas in MUTANTS:
            if names is not None and name not in names:
                continue
            d = os.path.join(tmp, name)
            os.makedirs(d)
            lib = build_mutant(mutate(source, find, replace), d)
            pins = PINS if all_pins else [p for p in PINS if any(f"test_oracle_{a}" in p for a in areas)]
            out[name] = "killed" if pins_fail(lib, pins) else "survived"
    return out


def main() -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("-k", default="", help="run the mutants whose name contains this")
    ap.add_argument("--all-pins", action="store_true", help="run every oracle pin file against each mutant")
    args = ap.parse_args()
    names = [m[0] for m in MUTANTS if args.k in m[0]]
    res = run(names, args.all_pins)
    for name, verdict in res.items():
        print(f"{verdict:9s} {name}")
    survived = [n for n, v in res.items() if v == "survived"]
    print(f"{len(res) - len(survived)} of {len(res)} mutants killed")
    return 1 if survived else 0


if __name__ == "__main__":
    sys.exit(main())
