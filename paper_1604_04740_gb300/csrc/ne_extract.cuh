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

// M = 3 with l = LT (8 or 16) in 64-bit arithmetic, the same bits as
// extract_rot<3>.  With A1 = a_hi 2^l + a_lo and A2 = b_hi 2^(2l) + b_lo
// (a_lo, b_lo the unsigned low parts), Eq. 19's exact quotient is
//     d_r = a_hi - b_hi + (a_lo 2^l - b_lo + d_{r-1}) / 2^(2l),
// every term of which fits 64 bits for l <= 30 (the last quotient is one of
// -2..2), and Eq. 24's d_r + 2^l d_{r-1} fits 64 bits for l <= 20, so the
// check compares exact values.
template <int LT>
__device__ __forceinline__ bool extract_rot3(const int64_t* rot, bool check, int64_t* out) {
    static_assert(LT >= 1 && LT <= 20, "64-bit bounds hold for l <= 20");
    constexpr int L = 2 * LT;
    const int64_t A1 = rot[1], A2 = rot[2];
    // Eq. 17-18: T = A2 - 2^l A1 (M = 3), d_{r-1} its low L bits sign-extended
    const int64_t d_last = (int64_t)(((uint64_t)A2 - ((uint64_t)A1 << LT)) << (64 - L)) >> (64 - L);
    const int64_t a_hi = A1 >> LT, a_lo = (int64_t)((uint64_t)A1 & ((1ull << LT) - 1));
    const int64_t b_hi = A2 >> L, b_lo = (int64_t)((uint64_t)A2 & ((1ull << L) - 1));
    const int64_t d_r = a_hi - b_hi + (((a_lo << LT) - b_lo + d_last) >> L);   // Eq. 19
    out[0] = d_r;
    out[2] = d_last;
    out[1] = (int64_t)((uint64_t)A1 - ((uint64_t)d_r << LT));                // Eq. 20
    return check && rot[0] != d_r + (int64_t)((uint64_t)d_last << LT);        // Eq. 24
}

}  // namespace ne
