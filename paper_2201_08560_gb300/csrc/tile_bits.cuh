// Bit access shared by the kernels that read B2SR tiles and k-bit segments of
// bitsets (Sec. III layout): row r of a tile held as 32-bit words is byte r
// (k <= 8; the low nibble at k = 4), half-word r (k = 16) or word r (k = 32);
// segment J of a bitset holds the bits of vertices kJ .. kJ+k-1.
#pragma once

#include <cstdint>

namespace b2sr {

template <int K>
__device__ __forceinline__ uint32_t tile_row(const uint32_t* w, int r) {
    if (K == 32) return w[r];
    if (K == 16) return (w[r >> 1] >> (16 * (r & 1))) & 0xFFFFu;
    return (w[r >> 2] >> (8 * (r & 3))) & 0xFFu;
}

template <int K>
__device__ __forceinline__ uint32_t seg_bits(const uint32_t* bits, int32_t J) {
    if (K == 32) return bits[J];
    if (K == 16) return reinterpret_cast<const uint16_t*>(bits)[J];
    if (K == 8) return reinterpret_cast<const uint8_t*>(bits)[J];
    return (reinterpret_cast<const uint8_t*>(bits)[J >> 1] >> ((J & 1) * 4)) & 0xFu;
}

template <int K>
__device__ __forceinline__ void clear_seg(uint32_t* bits, int32_t J) {
    if (K == 32) bits[J] = 0u;
    else if (K == 16) reinterpret_cast<uint16_t*>(bits)[J] = 0;
    else if (K == 8) reinterpret_cast<uint8_t*>(bits)[J] = 0;
    else atomicAnd(bits + (J >> 3), ~(0xFu << ((J & 7) * 4)));  // two segments share a byte
}

}  // namespace b2sr
