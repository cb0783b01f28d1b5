// Entanglement into digit planes, eight positions at a time (Eq. 16 followed
// by the balanced base-256 split of every entangled word); shared by the
// stand-alone kernel (ne_entangle_digits) and the ragged batch runner.
#pragma once

#include "ne_common.cuh"

namespace ne {

// eps_m = c_m + 2^l c_{m-1} (mod M); the product is formed in unsigned
// arithmetic so that it is the exact two's-complement value (|c| < 2^31 and
// l <= 31 under Eq. 13 keep it far from 2^63).
__device__ __forceinline__ int64_t entangle_word(int32_t cm, int32_t cprev, int l) {
    return (int64_t)((uint64_t)(int64_t)cm + ((uint64_t)(int64_t)cprev << l));
}

// Digit planes when the plan knows the stream-value range [lo, hi] it was
// derived for and its top digit is at most 3.  Every input is checked to lie
// in [lo, hi]; then every entangled word fits 32 bits, so it is formed in
// 32-bit arithmetic, and its balanced digits are the bytes of y = x + OFF
// with OFF = 0x80 in every digit position (digit t = byte t of y minus 128,
// i.e. the byte XOR 0x80 read as int8).  Digits the plan does not store must
// be exactly 0x80 in y, and y must stay below 256^(top+1).
struct FastPlan {
    uint32_t off;        // 0x80 in digits 0..top
    uint32_t ns_mask;    // bytes of digits <= top that are not stored
    uint32_t ns_want;    // 0x80 in those bytes
    uint32_t lim;        // 256^(top+1), 0 when top = 3 (no limit in 32 bits)
    int S;
    int lo, hi;          // the stream-value range the plan covers
    int byte_of[4];      // stored plane s -> digit index
    uint32_t pmask;      // all ones: entangle with the predecessor; 0: digits of the raw stream
};

// false when the plan has no input range, does not match l, or needs a
// digit above 3 (then the generic per-word kernels apply)
inline bool make_fast_plan(const ne_digits& dg, int l, FastPlan* F) {
    if (!(dg.lo <= dg.hi) || dg.l != l || dg.S < 1 || dg.S > 4) return false;
    const int top = dg.shift[dg.S - 1] / 8;
    if (top > 3) return false;
    uint32_t stored = 0;
    for (int s = 0; s < dg.S; s++) stored |= 1u << (dg.shift[s] / 8);
    F->off = 0;
    F->ns_mask = 0;
    F->ns_want = 0;
    for (int t = 0; t <= top; t++) {
        F->off |= 0x80u << (8 * t);
        if (!(stored & (1u << t))) {
            F->ns_mask |= 0xffu << (8 * t);
            F->ns_want |= 0x80u << (8 * t);
        }
    }
    F->lim = top < 3 ? (1u << (8 * (top + 1))) : 0u;
    F->S = dg.S;
    F->lo = dg.lo;
    F->hi = dg.hi;
    for (int s = 0; s < 4; s++) F->byte_of[s] = s < dg.S ? dg.shift[s] / 8 : 0;
    F->pmask = 0xffffffffu;
    return true;
}

// Eight consecutive positions of the MT streams starting at cb (stream
// stride n): 2 x 16-byte loads per stream, issued before any arithmetic, and
// one 8-byte store per stored digit plane and stream (plane stride n, planes
// of stream m at pb + m * S * n).  PLAIN: digits of the raw streams (no
// predecessor term).  Returns the largest (value - lo) seen, as unsigned:
// the inputs were in range iff it is <= hi - lo.  In-range inputs need no
// further check: the plan enumerated the digits of every word they form.
template <int MT, bool PLAIN = false>
__device__ __forceinline__ uint32_t entangle_chunk8(const int32_t* __restrict__ cb, int8_t* __restrict__ pb,
                                                    int64_t n, int l, const FastPlan& F) {
    uint32_t worst = 0;
    int32_t v[MT][8];
#pragma unroll
    for (int m = 0; m < MT; m++) {
        const int4* src = reinterpret_cast<const int4*>(cb + (int64_t)m * n);
        const int4 a = __ldcs(src), bb = __ldcs(src + 1);
        v[m][0] = a.x; v[m][1] = a.y; v[m][2] = a.z; v[m][3] = a.w;
        v[m][4] = bb.x; v[m][5] = bb.y; v[m][6] = bb.z; v[m][7] = bb.w;
#pragma unroll
        for (int e = 0; e < 8; e++) worst = max(worst, (uint32_t)v[m][e] - (uint32_t)F.lo);
    }
#pragma unroll
    for (int m = 0; m < MT; m++) {
        const int pm = (m + MT - 1) % MT;
        uint32_t y[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            if constexpr (PLAIN) y[e] = (uint32_t)v[m][e] + F.off;
            else y[e] = (uint32_t)v[m][e] + ((uint32_t)v[pm][e] << l) + F.off;
        }
#pragma unroll
        for (int s = 0; s < 4; s++) {
            if (s >= F.S) break;
            const uint32_t t = (uint32_t)F.byte_of[s];
            const uint32_t sel = t | ((t + 4) << 4);
            const uint32_t w0 = __byte_perm(__byte_perm(y[0], y[1], sel), __byte_perm(y[2], y[3], sel), 0x5410);
            const uint32_t w1 = __byte_perm(__byte_perm(y[4], y[5], sel), __byte_perm(y[6], y[7], sel), 0x5410);
            __stcs(reinterpret_cast<uint2*>(pb + ((int64_t)m * F.S + s) * n),
                   make_uint2(w0 ^ 0x80808080u, w1 ^ 0x80808080u));
        }
    }
    return worst;
}

}  // namespace ne
