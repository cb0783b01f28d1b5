// Shared device/host helpers of the numerical-entanglement library (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ne.h"

namespace ne {

// ---- host-side error reporting (ne_host.cu) --------------------------------
ne_status fail(ne_status st, const char* fmt, ...);
ne_status check_launch(const char* what);
int sm_count();                      // SMs of the current device (cached per device)
ne_status validate_params(const ne_params& p);
ne_status validate_digits(const ne_digits& dg);
ne_status validate_faults(const ne_faults& f, const char* who);

// internal launches shared by the entry points (ne_ops_i64.cu, ne_extract.cu)
ne_status gemm_i64_launch(int32_t P, const int64_t* x, const int8_t* G, int64_t* out, int32_t rows, int32_t cols,
                          int32_t k, uint32_t skip_mask, cudaStream_t s);
ne_status cconv_i64_launch(int32_t P, const int64_t* x, const int8_t* g, int64_t* out, int64_t batch, int64_t N,
                           uint32_t skip_mask, cudaStream_t s);
ne_status faults_launch(int64_t* delta, int M, int64_t batch, int64_t n, const ne_faults& F, uint32_t skip_mask,
                        cudaStream_t s);
// the tensor-path operations on the entangled words, split into the digits of
// dg in the tiles' loaders (ne_gemm_digits.cu, ne_cconv_digits.cu)
ne_status gemm_s8slice(ne_params p, ne_digits dg, const int64_t* words, const int8_t* G, int64_t* out,
                       uint32_t* flags, uint64_t* nflag, int32_t rows, int32_t cols, int32_t k, int32_t fuse,
                       int32_t r, const ne_faults& faults, int32_t* status, cudaStream_t s);
ne_status cconv_s8slice(ne_params p, ne_digits dg, const int64_t* words, const int8_t* g, int64_t* out,
                        uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t N, int32_t fuse, int32_t r,
                        const ne_faults& faults, int32_t* status, cudaStream_t s);
ne_status extract_launch(const ne_params& p, const int64_t* delta, int64_t* d_hat, int64_t batch, int64_t n, int r,
                         bool check, uint32_t* flags, unsigned long long* nflag, cudaStream_t s);

// grid of roughly `waves` full waves of `threads`-thread blocks on this GPU
inline int wave_blocks(int threads, int waves = 4) {
    int per_sm = 2048 / threads;
    if (per_sm < 1) per_sm = 1;
    return sm_count() * per_sm * waves;
}

inline bool aligned(const void* p, int bytes) {
    return (reinterpret_cast<uintptr_t>(p) % bytes) == 0;
}

// ---- 128-bit helpers (Remark 1: the 2w-bit temporaries) ---------------------
typedef __int128 i128;
typedef unsigned __int128 u128;

__device__ __forceinline__ i128 shl128(i128 x, int s) { return (i128)((u128)x << s); }
// arithmetic (floor) shift; nvcc implements >> on signed 128-bit as arithmetic
__device__ __forceinline__ i128 sar128(i128 x, int s) { return x >> s; }

// the same two shifts for 1 <= s <= 63, from 64-bit halves: the shifts of
// the extraction are l and (M-1) l, both in that range under Eq. 13 with
// w = 64, and a general 128-bit shift costs several times as many
// instructions when s is not a compile-time constant
__device__ __forceinline__ i128 shl128_63(i128 x, int s) {
    const uint64_t lo = (uint64_t)x, hi = (uint64_t)((u128)x >> 64);
    const uint64_t h = (hi << s) | (lo >> (64 - s));
    return (i128)(((u128)h << 64) | (u128)(lo << s));
}
__device__ __forceinline__ i128 sar128_63(i128 x, int s) {
    const uint64_t lo = (uint64_t)x;
    const int64_t hi = (int64_t)(x >> 64);
    const uint64_t h = (uint64_t)(hi >> s);
    return (i128)(((u128)h << 64) | (u128)((lo >> s) | ((uint64_t)hi << (64 - s))));
}

// sign extension of the low L bits of a word, 1 <= L <= 63 (Eq. 18)
__device__ __forceinline__ int64_t sext_low(uint64_t lo, int L) {
    return (int64_t)(lo << (64 - L)) >> (64 - L);
}

// ---- flag bitmaps -----------------------------------------------------------
// The extraction kernels give each lane two consecutive positions; lanes 0-15
// cover bits 0..31 of one bitmap word and lanes 16-31 the next.  OR-reduce the
// 2-bit contributions over each half-warp.
__device__ __forceinline__ uint32_t halfwarp_or(uint32_t v) {
    v |= __shfl_xor_sync(0xffffffffu, v, 1);
    v |= __shfl_xor_sync(0xffffffffu, v, 2);
    v |= __shfl_xor_sync(0xffffffffu, v, 4);
    v |= __shfl_xor_sync(0xffffffffu, v, 8);
    return v;
}

}  // namespace ne
