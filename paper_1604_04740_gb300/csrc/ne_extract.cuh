// Per-position disentanglement and check (Eq. 17-20, Eq. 24), shared by the
// stand-alone extraction kernels and the fused epilogues of the tensor-path
// operations, so both produce identical bits.
#pragma once

#include "ne_common.cuh"

namespace ne {

//
// rot[j] holds delta_{(r+j) mod M}; rot[0] (= delta_r) is only read when the
// check is requested.  Outputs out[j] = low 64 bits of d_{(r+j) mod M}.
// NARROW takes the 128-bit shifts from 64-bit halves (valid because l and
// (M-1) l lie in [1, 63] under Eq. 13); the results are the same bits either
// way, only the instruction mix differs (measured per kernel).
template <int MT, bool NARROW = true>
__device__ __forceinline__ bool extract_rot(const int64_t* rot, int M, int l, bool check, int64_t* out) {
    const auto shl = [](i128 x, int s) { return NARROW ? shl128_63(x, s) : shl128(x, s); };
    const auto sar = [](i128 x, int s) { return NARROW ? sar128_63(x, s) : sar128(x, s); };
    const int Mv = MT ? MT : M;
    // Eq. 17 by Horner's rule, times (-1)^M
    i128 acc = 0;
#pragma unroll
    for (int m = 0; m < (MT ? MT - 1 : 31); m++) {
        if (!MT && m >= Mv - 1) break;
        i128 v = (i128)rot[1 + m];
        acc = shl(acc, l) + ((m & 1) ? -v : v);
    }
    const i128 T = (Mv & 1) ? -acc : acc;
    const int L = (Mv - 1) * l;
    // Eq. 18: d_{r-1} = low L bits of T, sign-extended
    const int64_t d_last = sext_low((uint64_t)T, L);
    // Eq. 19: d_r = floor((-1)^M (T - d_{r-1}) / 2^L)
    i128 diff = T - (i128)d_last;
    if (Mv & 1) diff = -diff;
    const i128 d_r = sar(diff, L);
    out[0] = (int64_t)(uint64_t)d_r;
    out[Mv - 1] = d_last;
    // Eq. 20: d_{r+m} = delta_{r+m} - 2^l d_{r+m-1}.  Only the low 64 bits are
    // kept, and the low 64 bits of a difference/product depend only on the low
    // 64 bits of its operands, so wrapping 64-bit arithmetic is exact here.
    uint64_t prev = (uint64_t)d_r;
#pragma unroll
    for (int j = 1; j < (MT ? MT - 1 : 31); j++) {
        if (!MT && j >= Mv - 1) break;
        uint64_t cur = (uint64_t)rot[j] - (prev << l);
        out[j] = (int64_t)cur;
        prev = cur;
    }
    // Eq. 24 on the exact values: delta_r versus d_r + 2^l d_{r-1}
    bool flag = false;
    if (check) flag = ((i128)rot[0] != d_r + shl((i128)d_last, l));
    return flag;
}


}  // namespace ne
