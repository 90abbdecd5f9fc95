// Device side of the nested-parallelism engine (sm_103a).
//
// One "level" runs the children of a set of parents. Parents are processed in
// tiles taken from an atomic ticket, so tile order = parent order and a tile
// only ever waits (in a look-back) on tiles that running threads already own:
// warp-sized tiles for the forms without device launches (parent_warp), tiles
// of `parent_block` parents per CTA for the device-launch forms, whose block
// granularity needs CTA tiles (parent_kernel). For every parent the child
// count N is computed (Section III-D: the number of child threads, not
// gDim * bDim), then:
//
//   NODP        the parent loops over its N children (no launch code at all);
//   N < T       the parent loops over its children (thresholding, Section III-A);
//   N >= T      the children go to a child grid of ceil(ceil(N/bDim)/CF)
//               coarsened blocks (coarsening, Section IV-B), launched
//               per parent (GRAN_NONE) or aggregated (Sections II-B, V-A).
//
// Aggregation scans the coarsened block counts of the launching parents of a
// scope (warp shuffles, a block scan, a decoupled look-back across the tiles
// of a group of blocks or of the whole grid, or the paper's packed 64-bit
// atomic), stores one record {parent, row start, N} per launching parent and
// the scanned block offset, and one thread launches Sum(cg) blocks. Each
// aggregated child block finds its parent by a 32-ary warp search over the
// offsets, then runs CF original blocks of that parent (disaggregation outside
// the coarsening loop, Section VI).
//
// Level bookkeeping is slot based so that no kernel has to finish a level:
// level L = base + k, where base only changes between graph bodies and k is
// the kernel's position in the body; per-level counters live in slot L % 4,
// and the parent grid of level L clears the slot and frontier count that
// level L + 2 will use.
#pragma once

#include "np_loop.cuh"   // and, through it, every part in order:
// np_state, np_sinks, np_bodies, np_child, np_parent, np_loop
