// Z-order (Morton) curve helpers shared by the device filter and the compact sets.
#pragma once

#include <cstdint>

namespace capt {

// Spread the low 21 bits of v so that bit b moves to bit 3b.
__device__ __forceinline__ uint64_t spread21(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Quantised coordinate: min(2^21 - 1, floor((p - lo) / (hi - lo) * 2^21)) in FP64, 0 on
// an axis of zero extent.
__device__ __forceinline__ uint32_t morton_q(float p, double lo, double hi) {
    const double ext = __dsub_rn(hi, lo);
    if (!(ext > 0.0)) return 0u;
    const double f = floor(__dmul_rn(__ddiv_rn(__dsub_rn((double)p, lo), ext), 2097152.0));
    return f >= 2097151.0 ? 2097151u : (uint32_t)f;
}

}  // namespace capt
