// Byte layout of one cell block's table packet (host and device share it).
//   part A: ids int32[nu] | d uint16[nu] | incoff uint16[nu + 1]
//   part B: loc uint16[ne * nloc] | pos uint16[ne * nloc]
// Every section starts on a 16-byte boundary so that each part is one bulk copy.
#pragma once
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
BRAS_HD inline uint32_t pkt_size_a(uint32_t nu) { return pkt_off_incoff(nu) + pad16(2u * nu + 2u); }
BRAS_HD inline uint32_t pkt_size_b(uint32_t m) { return 2u * pad16(2u * m); }
}  // namespace bras
