// Byte layout of one cell block's table packet (host and device share it).
//   part A: ids int32[nu] | d uint16[nu] | (scatter) incoff uint16[nu + 1]
//   part B: loc uint16[m] | (scatter) pos uint16[m]                          (m = ne * nloc)
// H1 blocks sum their copies in fixed-point accumulators indexed by loc; blocks of streamed
// cell matrices (H(curl), H(div)) scatter their products to the dof-sorted order (pos) and sum
// each dof's run [incoff[u], incoff[u + 1]) -- the "scatter" sections.
// Every section starts on a 16-byte boundary so that each part is one bulk copy.
//   ids[u]   global dof of block-local dof u (interior dofs first, by ascending id, then the
//            shared ones grouped by their set of blocks)
//   d[u]     its multiplicity (D = P^T P)
//   loc[s]   block-local dof of copy s = a * ne + e (cell e, local index a); bit 15 = sign -1
//   pos[s]   position of copy s in the dof-sorted order (dof u's copies are one contiguous run,
//            by ascending s: the fixed summation order)
//   incoff   dof u's copies occupy positions [incoff[u], incoff[u + 1]) of that order
#pragma once
#include <stddef.h>
#include <stdint.h>

#ifdef __CUDACC__
#define BRAS_HD __host__ __device__
#else
#define BRAS_HD
#endif

namespace bras {
BRAS_HD inline uint32_t pad16(uint32_t b) { return (b + 15u) & ~15u; }
BRAS_HD inline uint32_t pkt_off_d(uint32_t nu) { return pad16(4u * nu); }
BRAS_HD inline uint32_t pkt_off_incoff(uint32_t nu) { return pkt_off_d(nu) + pad16(2u * nu); }
BRAS_HD inline uint32_t pkt_size_a(uint32_t nu, bool scatter) {
    return pkt_off_incoff(nu) + (scatter ? pad16(2u * nu + 2u) : 0u);
}
BRAS_HD inline uint32_t pkt_off_pos(uint32_t m) { return pad16(2u * m); }
BRAS_HD inline uint32_t pkt_size_b(uint32_t m, bool scatter) { return (scatter ? 2u : 1u) * pad16(2u * m); }

// Per-cell packed symmetric matrices (lower triangle by rows, entry idx = a (a + 1) / 2 + q,
// npk entries a cell) are stored in tiles of 32 consecutive cells: groups of G consecutive
// entries of one cell are contiguous (16 bytes: G = 4 floats, 8 bfloat16, 2 doubles), group g
// of the tile's 32 cells forms one 512-byte row, and the tile's rows follow in g order.  Each
// thread of a warp loads 16 bytes of its own cell, the warp reads whole rows, and a warp of
// 32 consecutive cells streams its tile front to back.  Cell counts are padded to a multiple
// of 32.
BRAS_HD inline int pk_groups(int npk, int G) { return (npk + G - 1) / G; }
BRAS_HD inline size_t pk_index(int idx, int64_t e, int npk, int G) {
    const size_t ng = (size_t)pk_groups(npk, G);
    return (((((size_t)(e >> 5) * ng) + (size_t)(idx / G)) << 5) + (size_t)(e & 31)) * (size_t)G + (size_t)(idx % G);
}
}  // namespace bras
