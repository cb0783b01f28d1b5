// Check-flag bitmaps (one bit per output position, uint32 words per group)
// assembled from a warp's per-lane results without atomics on the words.
#pragma once

#include "ne_common.cuh"

namespace ne {

// A warp owns 32*VEC consecutive positions of one group starting at word
// boundary seg*VEC; lane L holds the VEC flag bits of positions L*VEC ..
// L*VEC+VEC-1 in f.  Writes the warp's VEC words of flags_row (words at or
// beyond wpr are dropped) and adds their population to *nflag.
template <int VEC>
__device__ __forceinline__ void emit_flags(uint32_t f, int lane, int64_t seg, int64_t wpr,
                                           uint32_t* flags_row, unsigned long long* nflag) {
    if constexpr (VEC == 2) {
        uint32_t v = halfwarp_or(f << (2 * (lane & 15)));
        if ((lane & 15) == 0) {
            int64_t w = 2 * seg + (lane >> 4);
            if (w < wpr) {
                if (flags_row) flags_row[w] = v;
                if (nflag && v) atomicAdd(nflag, (unsigned long long)__popc(v));
            }
        }
    } else {
        uint32_t v = __ballot_sync(0xffffffffu, f != 0);
        if (lane == 0 && seg < wpr) {
            if (flags_row) flags_row[seg] = v;
            if (nflag && v) atomicAdd(nflag, (unsigned long long)__popc(v));
        }
    }
}

}  // namespace ne
