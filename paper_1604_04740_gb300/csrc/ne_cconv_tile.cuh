// One output tile of the batched circular convolution on the int8 tensor
// path, shared by the stand-alone kernel (ne_cconv_digits) and the ragged
// batch kernel (ne_batch_run).
//
// Every entangled word is held as balanced base-256 digit planes sigma_s, so
//     delta_m[i] = sum_s 2^shift_s  sum_j sigma_{m,s}[j] g[(i - j) mod N]
// and each inner sum is an exact int8 x int8 -> int32 contraction (|sum| <=
// N 2^14 < 2^31 for N <= 65536).
//
// Block-Toeplitz form.  With i = T p + q and j = T p' + t (T = 64),
//     sum_j sigma[j] g[(i - j) mod N] = sum_u sum_t G_u[q][t] sigma[T (p - u) + t],
//     G_u[q][t] = g[(T u + q - t) mod N],
// so for each shift u the block G_u (T x T, Toeplitz) multiplies a matrix
// whose columns are the input blocks p - u of every digit plane.  A tile owns
// up to NPB = 16 output blocks (1024 outputs) of one group and all planes:
//   D[q][(p, plane)] += sum_t G_u[q][t] B_u[t][(p, plane)],
// a dense T x (npb * planes) x T product per u, on mma.sync.m16n8k32.
// G_u is read from four byte-shifted copies of a reversed window of g in
// shared memory (every lane reads aligned words); the digit planes of the
// input blocks a u-chunk needs sit in shared memory, block-major, 80-byte
// rows, so the ldmatrix rows of any 8 consecutive columns hit distinct banks.
// The epilogue recombines the digits in int64, optionally flips injected
// fault bits into delta, then extracts/checks per position with the shared
// device code of the stand-alone extraction kernel.
// The digit rows come either from digit planes in memory (cp.async) or, for
// the fused form, straight from the raw int32 streams: Eq. 16 and the digit
// split are computed while the window is loaded, so the entangled words never
// reach memory.
#pragma once

#include "ne_common.cuh"
#include "ne_extract.cuh"
#include "ne_faults.cuh"
#include "ne_mma.cuh"

namespace ne {
namespace cconv {

constexpr int T = 64;                  // Toeplitz block
constexpr int NPB = 16;                // output blocks per tile (at most)
constexpr int UCH = 16;                // shifts u per chunk
constexpr int ROWB = 80;               // bytes per (block, plane) row in shared memory
constexpr int PADB = 16;               // margin of each g copy
constexpr int GW = 1184;               // bytes per g copy (>= T (UCH+1) + 2 PADB, = 32 mod 128)
constexpr int WBMAX = NPB + UCH - 1;   // input blocks a chunk can touch
constexpr int THREADS = 256;           // 8 warps: 4 row tiles x 2 column halves
constexpr int SP = 68;                 // stash row stride (int32) per output block

__host__ __device__ constexpr int smem_bytes(int MS) {
    return (WBMAX * MS * ROWB + 4 * GW) > (MS * NPB * SP * 4) ? (WBMAX * MS * ROWB + 4 * GW) : (MS * NPB * SP * 4);
}

// Everything a tile needs, already offset to its group.
struct TileArgs {
    const int8_t* planes;        // [M][S][N]
    const int8_t* g;             // [N]
    int64_t* out;                // [M][N]
    uint32_t* flags;             // [N/32] or null
    unsigned long long* nflag;   // or null
    const int64_t* fault_pos;    // faults, sorted by position (or null): output i of this
    const int32_t* fault_stream; // group is position fault_base + i of the list
    const int32_t* fault_bit;
    int64_t nfault;
    int64_t fault_base;
    int N, M, S, MS, l, r, fuse;
    int flags_atomic;            // bitmap pre-zeroed: OR in the set bits instead of storing words
    int shift[NE_MAX_DIGITS];
    // fused form (craw non-null): the raw streams [M][N] and the digit plan's
    // 32-bit split -- every input is checked against [raw_lo, raw_hi], the word
    // c_m + 2^l c_{m-1} (c_m alone if raw_plain) plus raw_off holds digit s as
    // byte raw_byte[s] XOR 0x80; an input out of range sets *status = NE_ERANGE
    const int32_t* craw;
    int32_t* status;
    uint32_t raw_off;
    int raw_lo, raw_hi, raw_plain;
    int raw_byte[4];
    // words form: the entangled words [M][N] themselves, split into the plan's
    // digits while loading; a word with y = word + 0x80..80 and
    // (y & w_nsmask) != w_nswant is outside the plan and sets *status = NE_ERANGE
    const int64_t* cwords;
    uint64_t w_nsmask, w_nswant;
    // bounded indexing (IX_LINEAR, IX_RAGGED): the inputs are [M][lin_n]
    // (inputs outside [0, lin_n) zero) and g has lin_K taps; IX_LINEAR: the
    // outputs [M][N] are the full linear convolution, N = lin_n + lin_K - 1;
    // IX_RAGGED: the circular convolution of length N = lin_n = lin_K, N not
    // a multiple of T
    int lin_n, lin_K;
};

// where a tile's digit rows come from
constexpr int LD_PLANES = 0;   // digit planes in memory (cp.async)
constexpr int LD_RAW = 1;      // the raw int32 streams: Eq. 16 and the split while loading
constexpr int LD_WORDS = 2;    // the entangled int64 words: the split while loading

// how output blocks meet input blocks
constexpr int IX_CIRC = 0;     // circular, N a multiple of T: input block (p - u) mod NB, u < NB
constexpr int IX_LINEAR = 1;   // linear: input block p - u, G_u[q][t] = g[T u + q - t] (0 outside [0, K))
constexpr int IX_RAGGED = 2;   // circular, any N: input block p - d for the signed block offsets d
                               // the tile needs, G_d[q][t] = g[(T d + q - t) mod N]

__device__ __forceinline__ int64_t shl64(int64_t x, int s) { return (int64_t)((uint64_t)x << s); }

// LT: the job's l when it is 16 or 8 (every shift below is then a constant;
// with the two digits at shifts 0 and LT of the byte-aligned plan of
// int8-valued streams, the recombination is one shift-add), else 0.
// P: positions per lane and pass, lane + 32 p (P = 2 needs npb T to be a
// multiple of 64); the stream order of the rotation and the output rows are
// formed once per thread.
template <int MT, int LT, int P>
__device__ __forceinline__ void epilogue_l(const TileArgs& a, const int32_t* stash, int p0, int npb, int nthreads) {
    constexpr int MX = MT ? MT : 32;
    const int M = MT ? MT : a.M;
    const int S = a.S;
    const int l = LT ? LT : a.l;
    const bool two = LT && S == 2 && a.shift[0] == 0 && a.shift[1] == LT;
    const int lane = threadIdx.x & 31;
    const int npos = npb * T;
    const int64_t i0 = (int64_t)p0 * T;
    const bool check = (a.fuse == NE_FUSE_EXTRACT_CHECK);
    const bool need_r = (a.fuse != NE_FUSE_RECOVER);
    // slot j holds stream (r + j) mod M: its first plane in the stash and its
    // output row, kept per thread when M is a compile-time constant
    auto stream_of = [&](int j) {
        int m = a.r + j;
        return m >= M ? m - M : m;
    };
    int soff_k[MT ? MT : 1];
    int64_t* orow_k[MT ? MT : 1];
    if constexpr (MT != 0) {
#pragma unroll
        for (int j = 0; j < MT; j++) {
            soff_k[j] = stream_of(j) * S * NPB * SP;
            orow_k[j] = a.out + (int64_t)stream_of(j) * a.N + i0;
        }
    }
    auto soff = [&](int j) {
        if constexpr (MT != 0) return soff_k[j];
        else return stream_of(j) * S * NPB * SP;
    };
    auto orow = [&](int j) -> int64_t* {
        if constexpr (MT != 0) return orow_k[j];
        else return a.out + (int64_t)stream_of(j) * a.N + i0;
    };
    auto digits = [&](const int32_t* sp, int j) {
        const int o = soff(j);
        if (two) return (int64_t)sp[o] + (int64_t)((uint64_t)(int64_t)sp[o + NPB * SP] << LT);
        int64_t v = 0;
#pragma unroll
        for (int s = 0; s < NE_MAX_DIGITS; s++)
            if (s < S) v += shl64(sp[o + s * NPB * SP], a.shift[s]);
        return v;
    };
    int64_t f0 = 0, f1 = 0;
    const int64_t key0 = a.fault_base + i0;
    if (a.nfault > 0) {
        f0 = fault_lower_bound(a.fault_pos, 0, a.nfault, key0);
        f1 = fault_lower_bound(a.fault_pos, f0, a.nfault, key0 + npos);
    }
    for (int base = (threadIdx.x & ~31) * P; base < npos; base += nthreads * P) {
        bool flag[P];
#pragma unroll
        for (int p = 0; p < P; p++) {
            flag[p] = false;
            const int bp = base + 32 * p;
            if (bp >= npos || i0 + bp >= a.N) continue;      // warp-uniform: past the end
            const int i = bp + lane;
            const int pr = i / T, q = i % T;
            const int32_t* sp = stash + pr * SP + q;
            // the last block of a linear convolution ends inside the tile
            const bool valid = i0 + i < a.N;
            if (a.fuse == NE_FUSE_NONE) {
                if (!valid) continue;
#pragma unroll
                for (int j = 0; j < MX; j++) {
                    if (!MT && j >= M) break;
                    int64_t v = digits(sp, j);
                    if (f1 > f0) v = apply_faults(v, a.fault_pos, a.fault_stream, a.fault_bit, f0, f1, key0 + i, stream_of(j));
                    orow(j)[i] = v;
                }
                continue;
            }
            int64_t rot[MX], res[MX];
#pragma unroll
            for (int j = 0; j < MX; j++) {
                if (!MT && j >= M) break;
                int64_t v = 0;
                if (valid && (j > 0 || need_r)) {
                    v = digits(sp, j);
                    if (f1 > f0) v = apply_faults(v, a.fault_pos, a.fault_stream, a.fault_bit, f0, f1, key0 + i, stream_of(j));
                }
                rot[j] = v;
            }
            if constexpr (MT == 3 && LT != 0) flag[p] = extract_rot3<LT>(rot, check, res) && valid;
            else flag[p] = extract_rot<MT>(rot, M, l, check, res) && valid;
            if (valid) {
#pragma unroll
                for (int j = 0; j < MX; j++) {
                    if (!MT && j >= M) break;
                    orow(j)[i] = res[j];
                }
            }
        }
        if (check) {
#pragma unroll
            for (int p = 0; p < P; p++) {
                const int bp = base + 32 * p;
                if (bp >= npos || i0 + bp >= a.N) continue;
                const uint32_t w = __ballot_sync(0xffffffffu, flag[p]);
                if (lane == 0 && w) {
                    if (a.flags) {
                        if (a.flags_atomic) atomicOr(&a.flags[(i0 + bp) / 32], w);
                        else a.flags[(i0 + bp) / 32] = w;
                    }
                    if (a.nflag) atomicAdd(a.nflag, (unsigned long long)__popc(w));
                } else if (lane == 0 && a.flags && !a.flags_atomic) {
                    a.flags[(i0 + bp) / 32] = 0u;
                }
            }
        }
    }
}

template <int MT, int P = 1>
__device__ __forceinline__ void epilogue(const TileArgs& a, const int32_t* stash, int p0, int npb,
                                         int nthreads = THREADS) {
    if (a.l == 16) epilogue_l<MT, 16, P>(a, stash, p0, npb, nthreads);
    else if (a.l == 8) epilogue_l<MT, 8, P>(a, stash, p0, npb, nthreads);
    else epilogue_l<MT, 0, P>(a, stash, p0, npb, nthreads);
}

// bytes t of four words, XOR 0x80: four consecutive positions of one digit plane
__device__ __forceinline__ uint32_t pick4(uint32_t y0, uint32_t y1, uint32_t y2, uint32_t y3, uint32_t t) {
    const uint32_t sel = t | ((t + 4) << 4);
    return __byte_perm(__byte_perm(y0, y1, sel), __byte_perm(y2, y3, sel), 0x5410) ^ 0x80808080u;
}

// The digit rows [WB][MS][ROWB] of input blocks (first + blk_rel) mod NB.
// From planes: 16-byte cp.async copies (a lost stream's rows zero-filled);
// the caller commits and waits.  Fused: every work item (block, stream,
// 16 positions) loads 16 inputs of c_m and c_{m-1}, forms the words of
// Eq. 16 in 32 bits and stores the S digit rows' 16 bytes.
template <int LD>
__device__ __forceinline__ void load_window(const TileArgs& a, uint8_t* sig, int WB, int first, int NB, int nthr) {
    const int N = a.N, MS = a.MS;
    const int tid = threadIdx.x;
    if constexpr (LD == LD_WORDS) {
        const int M = a.M, S = a.S;
        bool bad = false;
        for (int e = tid; e < WB * M * 4; e += nthr) {
            const int c16 = e & 3, rowm = e >> 2;
            const int blk_rel = rowm / M, m = rowm - blk_rel * M;
            int ab = (first + blk_rel) % NB;
            if (ab < 0) ab += NB;
            uint8_t* dst = sig + (blk_rel * MS + m * S) * ROWB + c16 * 16;
            if (a.fuse == NE_FUSE_RECOVER && m == a.r) {
                for (int s = 0; s < S; s++) *reinterpret_cast<uint4*>(dst + s * ROWB) = make_uint4(0u, 0u, 0u, 0u);
                continue;
            }
            const longlong2* src = reinterpret_cast<const longlong2*>(a.cwords + (int64_t)m * N + (int64_t)ab * T + c16 * 16);
            uint64_t y[16];
#pragma unroll
            for (int q = 0; q < 8; q++) {
                const longlong2 v = __ldg(src + q);
                y[2 * q] = (uint64_t)v.x + 0x8080808080808080ull;
                y[2 * q + 1] = (uint64_t)v.y + 0x8080808080808080ull;
            }
#pragma unroll
            for (int q = 0; q < 16; q++) bad |= (y[q] & a.w_nsmask) != a.w_nswant;
#pragma unroll
            for (int s = 0; s < NE_MAX_DIGITS; s++) {
                if (s >= S) break;
                const int sh = a.shift[s];
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t v0 = (uint32_t)(y[4 * q] >> sh), v1 = (uint32_t)(y[4 * q + 1] >> sh);
                    const uint32_t v2 = (uint32_t)(y[4 * q + 2] >> sh), v3 = (uint32_t)(y[4 * q + 3] >> sh);
                    w[q] = __byte_perm(__byte_perm(v0, v1, 0x0040), __byte_perm(v2, v3, 0x0040), 0x5410) ^ 0x80808080u;
                }
                *reinterpret_cast<uint4*>(dst + s * ROWB) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        if (bad && a.status) atomicExch(a.status, (int32_t)NE_ERANGE);
        return;
    } else if constexpr (LD == LD_PLANES) {
        const uint32_t sig_s = smem_u32(sig);
        for (int e = tid; e < WB * MS * 4; e += nthr) {
            const int c16 = e & 3, row = e >> 2;
            const int blk_rel = row / MS, ms = row - blk_rel * MS;
            int ab = (first + blk_rel) % NB;
            if (ab < 0) ab += NB;
            const int8_t* src = a.planes + (int64_t)ms * N + (int64_t)ab * T + c16 * 16;
            const bool lost = (a.fuse == NE_FUSE_RECOVER) && (ms / a.S == a.r);
            cp_async16(sig_s + row * ROWB + c16 * 16, src, lost ? 0 : 16);
        }
        return;
    } else {
    const int M = a.M, S = a.S;
    uint32_t worst = 0;
    // a window longer than the group holds block (first + b) mod NB twice, at
    // rows b and b + NB (WB < 2 NB): each block is formed once and stored twice
    const int WU = WB < NB ? WB : NB;
    for (int e = tid; e < WU * M * 4; e += nthr) {
        const int c16 = e & 3, rowm = e >> 2;
        const int blk_rel = rowm / M, m = rowm - blk_rel * M;
        int ab = (first + blk_rel) % NB;
        if (ab < 0) ab += NB;
        uint8_t* dst = sig + (blk_rel * MS + m * S) * ROWB + c16 * 16;
        uint8_t* dst2 = blk_rel + NB < WB ? dst + NB * MS * ROWB : nullptr;
        if (a.fuse == NE_FUSE_RECOVER && m == a.r) {
            for (int s = 0; s < S; s++) {
                *reinterpret_cast<uint4*>(dst + s * ROWB) = make_uint4(0u, 0u, 0u, 0u);
                if (dst2) *reinterpret_cast<uint4*>(dst2 + s * ROWB) = make_uint4(0u, 0u, 0u, 0u);
            }
            continue;
        }
        const int64_t pos = (int64_t)ab * T + c16 * 16;
        const int mp = m == 0 ? M - 1 : m - 1;
        // a lost stream r is never loaded as c_m, but its inputs still enter
        // the words of stream r+1 (Eq. 16): check them there
        const bool check_prev = a.fuse == NE_FUSE_RECOVER && mp == a.r;
        const int4* xm = reinterpret_cast<const int4*>(a.craw + (int64_t)m * N + pos);
        const int4* xp = reinterpret_cast<const int4*>(a.craw + (int64_t)mp * N + pos);
        uint32_t y[16];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int4 v = __ldg(xm + q);
            y[4 * q] = (uint32_t)v.x;
            y[4 * q + 1] = (uint32_t)v.y;
            y[4 * q + 2] = (uint32_t)v.z;
            y[4 * q + 3] = (uint32_t)v.w;
        }
#pragma unroll
        for (int k = 0; k < 16; k++) {
            worst = max(worst, y[k] - (uint32_t)a.raw_lo);
            y[k] += a.raw_off;
        }
        if (!a.raw_plain) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int4 v = __ldg(xp + q);
                y[4 * q] += (uint32_t)v.x << a.l;
                y[4 * q + 1] += (uint32_t)v.y << a.l;
                y[4 * q + 2] += (uint32_t)v.z << a.l;
                y[4 * q + 3] += (uint32_t)v.w << a.l;
                if (check_prev)
                    worst = max(max(max(worst, (uint32_t)v.x - (uint32_t)a.raw_lo), (uint32_t)v.y - (uint32_t)a.raw_lo),
                                max((uint32_t)v.z - (uint32_t)a.raw_lo, (uint32_t)v.w - (uint32_t)a.raw_lo));
            }
        }
#pragma unroll
        for (int s = 0; s < 4; s++) {
            if (s >= S) break;
            const uint32_t t = (uint32_t)a.raw_byte[s];
            const uint4 d = make_uint4(pick4(y[0], y[1], y[2], y[3], t), pick4(y[4], y[5], y[6], y[7], t),
                                       pick4(y[8], y[9], y[10], y[11], t), pick4(y[12], y[13], y[14], y[15], t));
            *reinterpret_cast<uint4*>(dst + s * ROWB) = d;
            if (dst2) *reinterpret_cast<uint4*>(dst2 + s * ROWB) = d;
        }
    }
    if (worst > (uint32_t)a.raw_hi - (uint32_t)a.raw_lo && a.status) atomicExch(a.status, (int32_t)NE_ERANGE);
    }
}

// The window of the bounded indexings: input blocks first .. first + WB - 1
// (no wrap), every position outside [0, n) zero -- for the raw streams the
// word 0, for words and digit planes digits 0.  An item (block, stream or
// plane, 16 positions) entirely inside its stream whose row starts aligned
// takes the vector loads, the others element by element.
template <int LD>
__device__ __forceinline__ void load_window_bounded(const TileArgs& a, uint8_t* sig, int WB, int first, int n,
                                                    int nthr) {
    const int M = a.M, S = a.S, MS = a.MS;
    auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
    if constexpr (LD == LD_PLANES) {
        const bool vec_ok = (n & 15) == 0 && al16(a.planes);
        for (int e = threadIdx.x; e < WB * MS * 4; e += nthr) {
            const int c16 = e & 3, row = e >> 2;
            const int blk_rel = row / MS, ms = row - blk_rel * MS;
            const int64_t pos = (int64_t)(first + blk_rel) * T + c16 * 16;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            const bool lost = a.fuse == NE_FUSE_RECOVER && ms / S == a.r;
            if (!lost && pos + 16 > 0 && pos < n) {
                const int8_t* src = a.planes + (int64_t)ms * n + pos;
                if (vec_ok && pos >= 0 && pos + 16 <= n) {
                    v = __ldg(reinterpret_cast<const uint4*>(src));
                } else {
                    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                    for (int b = 0; b < 16; b++)
                        if (pos + b >= 0 && pos + b < n) w[b >> 2] |= (uint32_t)(uint8_t)__ldg(src + b) << (8 * (b & 3));
                    v = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            *reinterpret_cast<uint4*>(sig + row * ROWB + c16 * 16) = v;
        }
        return;
    } else if constexpr (LD == LD_WORDS) {
        const bool vec_ok = (n & 1) == 0 && al16(a.cwords);
        bool bad = false;
        for (int e = threadIdx.x; e < WB * M * 4; e += nthr) {
            const int c16 = e & 3, rowm = e >> 2;
            const int blk_rel = rowm / M, m = rowm - blk_rel * M;
            uint8_t* dst = sig + (blk_rel * MS + m * S) * ROWB + c16 * 16;
            const int64_t pos = (int64_t)(first + blk_rel) * T + c16 * 16;
            uint64_t y[16];
#pragma unroll
            for (int q = 0; q < 16; q++) y[q] = 0x8080808080808080ull;     // the word 0: digits 0
            const bool lost = a.fuse == NE_FUSE_RECOVER && m == a.r;
            if (!lost && pos + 16 > 0 && pos < n) {
                const int64_t* src = a.cwords + (int64_t)m * n + pos;
                if (vec_ok && pos >= 0 && pos + 16 <= n) {
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const longlong2 v = __ldg(reinterpret_cast<const longlong2*>(src) + q);
                        y[2 * q] += (uint64_t)v.x;
                        y[2 * q + 1] += (uint64_t)v.y;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 16; q++)
                        if (pos + q >= 0 && pos + q < n) y[q] += (uint64_t)__ldg(src + q);
                }
#pragma unroll
                for (int q = 0; q < 16; q++) bad |= (y[q] & a.w_nsmask) != a.w_nswant;
            }
#pragma unroll
            for (int s = 0; s < NE_MAX_DIGITS; s++) {
                if (s >= S) break;
                const int sh = a.shift[s];
                uint32_t w[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t v0 = (uint32_t)(y[4 * q] >> sh), v1 = (uint32_t)(y[4 * q + 1] >> sh);
                    const uint32_t v2 = (uint32_t)(y[4 * q + 2] >> sh), v3 = (uint32_t)(y[4 * q + 3] >> sh);
                    w[q] = __byte_perm(__byte_perm(v0, v1, 0x0040), __byte_perm(v2, v3, 0x0040), 0x5410) ^ 0x80808080u;
                }
                *reinterpret_cast<uint4*>(dst + s * ROWB) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        if (bad && a.status) atomicExch(a.status, (int32_t)NE_ERANGE);
        return;
    } else {
    const bool vec_ok = (n & 3) == 0 && al16(a.craw);
    uint32_t worst = 0;
    for (int e = threadIdx.x; e < WB * M * 4; e += nthr) {
        const int c16 = e & 3, rowm = e >> 2;
        const int blk_rel = rowm / M, m = rowm - blk_rel * M;
        uint8_t* dst = sig + (blk_rel * MS + m * S) * ROWB + c16 * 16;
        const int64_t pos = (int64_t)(first + blk_rel) * T + c16 * 16;
        if ((a.fuse == NE_FUSE_RECOVER && m == a.r) || pos + 16 <= 0 || pos >= n) {
            for (int s = 0; s < S; s++) *reinterpret_cast<uint4*>(dst + s * ROWB) = make_uint4(0u, 0u, 0u, 0u);
            continue;
        }
        const int mp = m == 0 ? M - 1 : m - 1;
        const bool check_prev = a.fuse == NE_FUSE_RECOVER && mp == a.r;
        const int32_t* xm = a.craw + (int64_t)m * n;
        const int32_t* xp = a.craw + (int64_t)mp * n;
        uint32_t y[16];
        if (vec_ok && pos >= 0 && pos + 16 <= n) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int4 v = __ldg(reinterpret_cast<const int4*>(xm + pos) + q);
                y[4 * q] = (uint32_t)v.x;
                y[4 * q + 1] = (uint32_t)v.y;
                y[4 * q + 2] = (uint32_t)v.z;
                y[4 * q + 3] = (uint32_t)v.w;
            }
#pragma unroll
            for (int k = 0; k < 16; k++) {
                worst = max(worst, y[k] - (uint32_t)a.raw_lo);
                y[k] += a.raw_off;
            }
            if (!a.raw_plain) {
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int4 v = __ldg(reinterpret_cast<const int4*>(xp + pos) + q);
                    const uint32_t w[4] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z, (uint32_t)v.w};
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        y[4 * q + k] += w[k] << a.l;
                        if (check_prev) worst = max(worst, w[k] - (uint32_t)a.raw_lo);
                    }
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < 16; k++) {
                const int64_t i = pos + k;
                uint32_t v = 0;                       // zero padding: the word 0, every digit 0
                if (i >= 0 && i < n) {
                    const uint32_t x = (uint32_t)__ldg(xm + i);
                    worst = max(worst, x - (uint32_t)a.raw_lo);
                    v = x;
                    if (!a.raw_plain) {
                        const uint32_t w = (uint32_t)__ldg(xp + i);
                        if (check_prev) worst = max(worst, w - (uint32_t)a.raw_lo);
                        v += w << a.l;
                    }
                }
                y[k] = v + a.raw_off;
            }
        }
#pragma unroll
        for (int s = 0; s < 4; s++) {
            if (s >= S) break;
            const uint32_t t = (uint32_t)a.raw_byte[s];
            *reinterpret_cast<uint4*>(dst + s * ROWB) =
                make_uint4(pick4(y[0], y[1], y[2], y[3], t), pick4(y[4], y[5], y[6], y[7], t),
                           pick4(y[8], y[9], y[10], y[11], t), pick4(y[12], y[13], y[14], y[15], t));
        }
    }
    if (worst > (uint32_t)a.raw_hi - (uint32_t)a.raw_lo && a.status) atomicExch(a.status, (int32_t)NE_ERANGE);
    }
}

// The tile of output blocks [p0, p0 + npb) of one group; all 256 threads of
// the block take part.  smem: smem_bytes(MS) bytes, 128-byte aligned.
// IX_LINEAR: the shifts u run over the kernel's NU = (K + 62) / 64 + 1 blocks
// of G_u[q][t] = g[T u + q - t] (zero outside [0, K)) and input block p - u
// is zero outside the stream, so each output block sums NU products instead
// of NB (Sec. IV-A: a long stream needs only the blocks the kernel reaches).
// IX_RAGGED: the block offsets d = p - p' of the tile's outputs and every
// input block, d = ubase + u with ubase = p0 - NB + 1 and u < NB + npb - 1
// (each output block meets NB of them; the others are zero rows).
template <int NTW, int MT, int LD = LD_PLANES, int IX = IX_CIRC>
__device__ __forceinline__ void tile(const TileArgs& a, uint8_t* smem, int p0, int npb) {
    const int MS = a.MS;
    const int N = a.N;
    const int NB = IX == IX_RAGGED ? (N + T - 1) / T : N / T;
    const int NU = IX == IX_LINEAR ? (a.lin_K + 62) / T + 1 : (IX == IX_RAGGED ? NB + npb - 1 : NB);   // shifts u
    const int ubase = IX == IX_RAGGED ? p0 - NB + 1 : 0;
    const int uch = min(UCH, NU);
    const int WB = npb + uch - 1;
    const int cols = npb * MS;
    const int NT = (cols + 7) / 8;
    const int NTH = (NT + 1) / 2;

    uint8_t* sig = smem;                                  // [WB][MS][ROWB]
    uint8_t* gcp = smem + WBMAX * MS * ROWB;              // 4 x GW
    int32_t* stash = reinterpret_cast<int32_t*>(smem);    // after the main loop

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mt = warp & 3, half = warp >> 2;
    const int gq = lane >> 2, tq = lane & 3;
    const int tile0 = half * NTH;
    const int ntile = max(0, min(NT, tile0 + NTH) - tile0);
    const int kh = (lane >> 3) & 1;
    const int rho = (4 - (gq & 3)) & 3;                   // byte shift of this lane's G_u reads
    const uint32_t gcp_s = smem_u32(gcp) + rho * GW + PADB - rho;
    const uint32_t sig_s = smem_u32(sig);

    int acc[NTW][4];
#pragma unroll
    for (int j = 0; j < NTW; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0;
    // this lane's ldmatrix row of column tile tile0 (+ 8 rows per further
    // tile).  A padding column (c >= cols, last tile only) reads a row past
    // the window's used rows, still inside the shared memory of the window and
    // the filter copies after it; its result is dropped at the stash.
    const uint32_t bbase = sig_s + (8 * (tile0 + (lane >> 4)) + (lane & 7)) * ROWB + 16 * kh;

    for (int u0 = 0; u0 < NU; u0 += uch) {
        const int uc = min(uch, NU - u0);
        // digit rows of input blocks (p0 - (u0 + uch - 1) + blk_rel), mod NB for
        // the circular convolution
        if constexpr (IX == IX_CIRC) load_window<LD>(a, sig, WB, p0 - (u0 + uch - 1), NB, THREADS);
        else load_window_bounded<LD>(a, sig, WB, p0 - ubase - (u0 + uch - 1), a.lin_n, THREADS);
        cp_async_commit();
        // g copies: copy rr, byte z holds g[(T (ubase + u0 + uch) - (z + rr - PADB)) mod N]
        // (linear: g at that index, 0 outside [0, K))
        const int top = T * (ubase + u0 + uch);
        for (int e = tid; e < 4 * (GW / 4); e += THREADS) {
            const int rr = e / (GW / 4), zw = e - rr * (GW / 4);
            uint32_t w = 0;
            if constexpr (IX == IX_CIRC) {
                // N a multiple of 64: the bytes g[v], g[v-1], g[v-2], g[v-3] (mod N)
                // are one funnel shift of two aligned filter words, byte-reversed
                int v = (top - (4 * zw + rr - PADB)) % N;
                if (v < 0) v += N;
                int u = v - 3;
                if (u < 0) u += N;
                const uint32_t* g32 = reinterpret_cast<const uint32_t*>(a.g);
                const int q = u >> 2, q1 = q + 1 == N / 4 ? 0 : q + 1;
                w = __byte_perm(__funnelshift_r(__ldg(g32 + q), __ldg(g32 + q1), 8 * (u & 3)), 0u, 0x0123);
            } else {
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    int idx = top - (4 * zw + k + rr - PADB);
                    uint32_t gv;
                    if constexpr (IX == IX_LINEAR) {
                        gv = (idx >= 0 && idx < a.lin_K) ? (uint32_t)(uint8_t)__ldg(a.g + idx) : 0u;
                    } else {
                        idx %= N;
                        if (idx < 0) idx += N;
                        gv = (uint32_t)(uint8_t)__ldg(a.g + idx);
                    }
                    w |= gv << (8 * k);
                }
            }
            *reinterpret_cast<uint32_t*>(gcp + rr * GW + 4 * zw) = w;
        }
        cp_async_wait<0>();
        __syncthreads();

        for (int u = u0; u < u0 + uc; u++) {
            const int ushift = u0 + uch - 1 - u;
            const uint32_t ya = gcp_s + T * (u0 + uch - u) - 16 * mt - gq + 4 * tq;
            const uint32_t yb = bbase + MS * ushift * ROWB;
#pragma unroll
            for (int ks = 0; ks < 2; ks++) {
                uint32_t af[4];
                af[0] = lds32(ya + 32 * ks);
                af[1] = lds32(ya + 32 * ks - 8);
                af[2] = lds32(ya + 32 * ks + 16);
                af[3] = lds32(ya + 32 * ks + 8);
#pragma unroll
                for (int jj = 0; jj < NTW; jj += 2) {
                    if (jj >= ntile) break;
                    uint32_t bf[4];
                    ldsm_x4(bf, yb + 8 * jj * ROWB + 32 * ks);
                    mma_s8(acc[jj], af, bf[0], bf[1]);
                    if (jj + 1 < ntile) mma_s8(acc[jj + 1], af, bf[2], bf[3]);
                }
            }
        }
        __syncthreads();
    }

    // int32 digit sums -> stash [plane][output block][q]
#pragma unroll
    for (int jj = 0; jj < NTW; jj++) {
        if (jj >= ntile) break;
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const int c = 8 * (tile0 + jj) + 2 * tq + (h & 1);
            const int q = 16 * mt + gq + 8 * (h >> 1);
            if (c < cols) {
                const int pr = c / MS, ms = c - pr * MS;
                stash[(ms * NPB + pr) * SP + q] = acc[jj][h];
            }
        }
    }
    __syncthreads();
    epilogue<MT>(a, stash, p0, npb);
}

// ---- hybrid tile: the int8 tensor pipe and the CUDA-core dp4a pipe together -----------------
//
// On sm_103a the int8 tensor instruction and dp4a (four int8 products added
// into an int32, on the integer ALUs) have about the same throughput and run
// on separate pipes.  For groups of 9..16 blocks (N in (512, 1024]) the
// hybrid tile gives the last HW * R / 2 output blocks to HW extra warps that
// compute them with dp4a, while TW MMA warps (8 as in tile(), or 4 that each
// hold every column tile of their 16 rows) compute the other blocks; both
// finish into the same stash and the same epilogue.  A
// dp4a thread owns R outputs 4 apart, i0 + 4 r, for every digit plane.  The
// filter word that output i0 + 4 r needs at input chunk J (positions 4 J ..
// 4 J + 3) is the one output i0 needs at chunk J - r, so per 4 inputs a
// thread loads one new filter word (from four byte-shifted copies of the
// reversed filter, so that every read is aligned) and each plane's digit
// word (a broadcast, 8 inputs per load), for R x planes dp4a.
// TW tensor warps (8: two column halves of 4 row tiles; 4: one) and HW dp4a warps
__host__ __device__ constexpr int hybrid_threads(int HW, int TW = 8) { return 32 * (TW + HW); }
constexpr int GDP = 2192;                     // bytes per filter copy slot: >= 2 * 1024 + 16 + 4 * 31
constexpr int GDPW = 514;                     // words of a copy the dp4a reads reach: (2 * 1024 + 8) / 4
// Byte offset of dp4a filter copy rr for R outputs per thread (R = 2, 3, 4).
// The 8 lanes that read copy rr (the same rho) are R words apart, so their
// banks are D_rr - R k, k = 0..7, with D_rr = the copy's word offset (+1 for
// copy 0, whose reads start one word later).  D_rr = rr (R = 4), 0, 1, 16, 17
// (R = 2) or 5, 13, 21, 29 (R = 3: times 11 = 3^-1 mod 32 the sets become
// intervals of 8 banks ending at 23, 15, 7, 31) puts the four copies' lanes on
// disjoint banks.
__host__ __device__ constexpr int gdp_bank(int rr, int R) {
    return R == 4 ? rr
                  : (R == 3 ? 5 + 8 * rr : (rr == 0 ? 0 : (rr == 1 ? 1 : (rr == 2 ? 16 : 17))));
}
__host__ __device__ constexpr int gdp_off(int rr, int R) {
    return rr * GDP + 4 * (((gdp_bank(rr, R) - (rr * GDP / 4 + (rr == 0 ? 1 : 0))) % 32 + 32) % 32);
}

// [digit-plane window + tensor-pipe filter window][dp4a filter copies][stash]:
// the stash has its own space, so a warp may write its results as soon as it
// is done, while other warps still read the windows.
__host__ __device__ constexpr int hybrid_smem_bytes(int MS) {
    return WBMAX * MS * ROWB + 4 * GW + 4 * GDP + MS * NPB * SP * 4;
}

// NBC: the group's block count when the caller fixes it at compile time (every
// size below and the shape of the tensor warps' loop are then constants), else 0
template <int MT, int MSC, int HW, int R, int LD = LD_PLANES, int NBC = 0, int TW = 8>
__device__ __forceinline__ void tile_hybrid(const TileArgs& a, uint8_t* smem) {
    constexpr int MS = MSC;
    constexpr int NTHR = hybrid_threads(HW, TW);
    constexpr int HALVES = TW / 4;        // column parts of the tensor warps
    static_assert(TW == 4 || TW == 8, "4 or 8 tensor warps");
    static_assert(TW == 8 || NBC != 0, "4 tensor warps hold every column tile: compile-time groups only");
    constexpr int DT = 32 * HW;           // dp4a threads
    static_assert((DT * R) % T == 0, "dp4a outputs must be whole blocks");
    static_assert(R >= 2 && R <= 4, "the dp4a filter copies are laid out for 2 to 4 outputs per thread");
    static_assert(NBC == 0 || (NBC > DT * R / T && NBC <= NPB), "a compile-time group size must leave tensor blocks");
    const int N = NBC ? NBC * T : a.N;
    const int NB = N / T;                 // DT * R / T + 1 .. 16
    const int uch = NB;                   // a single chunk of shifts
    const int npb = NB - DT * R / T;      // output blocks on the tensor pipe
    const int WB = npb + uch - 1;
    const int cols = npb * MS;
    const int NT = (cols + 7) / 8;
    const int NTH = (NT + HALVES - 1) / HALVES;

    uint8_t* sig = smem;                                  // [WB][MS][ROWB]
    uint8_t* gcp = smem + WBMAX * MS * ROWB;              // 4 x GW (tensor-pipe filter window)
    uint8_t* gdp = gcp + 4 * GW;                          // 4 x GDP (dp4a filter copies)
    int32_t* stash = reinterpret_cast<int32_t*>(gdp + 4 * GDP);   // [MS][NPB][SP], its own space

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t sig_s = smem_u32(sig);

    // -- loads (every thread) --
    load_window<LD>(a, sig, WB, -(uch - 1), NB, NTHR);
    cp_async_commit();
    // The reversed filter rev[j] = g[(N - j) mod N] as words, staged once in the
    // stash's space (free until the stash is written), with one wrap word at
    // the end: word i is byte 0 of filter word (N/4 - i) mod (N/4) followed by
    // bytes 3, 2, 1 of the word before it (N is a multiple of 64 here).  Every
    // copy word below holds 4 consecutive bytes of rev, g[(v - k) mod N] =
    // rev[(s + k) mod N] with s = -v mod N: one funnel shift of two staged words.
    uint32_t* revw = reinterpret_cast<uint32_t*>(stash);
    const int NW = N / 4;
    for (int i = tid; i <= NW; i += NTHR) {
        const int a0 = i % NW == 0 ? 0 : NW - i % NW;
        const int a1 = a0 == 0 ? NW - 1 : a0 - 1;
        const uint32_t* gw = reinterpret_cast<const uint32_t*>(a.g);
        revw[i] = __byte_perm(__ldg(gw + a0), __ldg(gw + a1), 0x5670);
    }
    __syncthreads();
    // Both filter windows are the reversed filter shifted by rr bytes: word w of
    // tensor-pipe copy rr (byte z: g[(N - (z + rr - PADB)) mod N]) is the funnel
    // shift by 8 rr of staged words (w - 4) mod NW and the one after it, word w
    // of dp4a copy rr (byte z: g[(N + 4 - z - rr) mod N]) that of staged words
    // (w - 1) mod NW and the one after it (word NW is word 0 again).  An item
    // forms 4 consecutive words of one copy from 5 staged words.
    constexpr int GQ = GW / 16, DQ = (GDPW + 3) / 4;      // items per copy
    static_assert(GW % 16 == 0 && 16 * DQ + 4 * 31 <= GDP, "filter copies must hold whole items");
    for (int e = tid; e < 4 * (GQ + DQ); e += NTHR) {
        const bool tens = e < 4 * GQ;
        const int e2 = tens ? e : e - 4 * GQ;
        const int rr = tens ? e2 / GQ : e2 / DQ;
        const int j = tens ? e2 - rr * GQ : e2 - rr * DQ;
        int b4 = (4 * j - (tens ? 4 : 0)) % NW;
        if (b4 < 0) b4 += NW;
        const uint4 q = *reinterpret_cast<const uint4*>(revw + b4);
        const uint32_t w0 = tens ? q.x : revw[b4 == 0 ? NW - 1 : b4 - 1];
        const uint32_t w1 = tens ? q.y : q.x, w2 = tens ? q.z : q.y, w3 = tens ? q.w : q.z;
        const uint32_t w4 = tens ? revw[b4 + 4] : q.w;
        const int sh = 8 * rr;
        const uint4 o = make_uint4(__funnelshift_r(w0, w1, sh), __funnelshift_r(w1, w2, sh),
                                   __funnelshift_r(w2, w3, sh), __funnelshift_r(w3, w4, sh));
        if (tens) {
            *reinterpret_cast<uint4*>(gcp + rr * GW + 16 * j) = o;
        } else {
            uint32_t* d = reinterpret_cast<uint32_t*>(gdp + gdp_off(rr, R) + 16 * j);
            d[0] = o.x;
            d[1] = o.y;
            d[2] = o.z;
            d[3] = o.w;
        }
    }
    cp_async_wait<0>();
    __syncthreads();

    if (warp < TW) {
        // -- tensor pipe: output blocks [0, npb), as in tile() --
        const int mt = warp & 3, half = warp >> 2;
        const int gq = lane >> 2, tq = lane & 3;
        const int tile0 = half * NTH;
        // both halves hold NTH column tiles when NT is even
        const int ntile = NT == HALVES * NTH ? NTH : max(0, min(NT, tile0 + NTH) - tile0);
        const int kh = (lane >> 3) & 1;
        const int rho = (4 - (gq & 3)) & 3;
        // column tiles a warp holds: at most 16 blocks' worth, or exactly the
        // compile-time group's
        constexpr int NTW = NBC ? (((NBC - DT * R / T) * MS + 7) / 8 + HALVES - 1) / HALVES
                                : (16 * MS / 8 + HALVES - 1) / HALVES;
        int acc[NTW][4];
#pragma unroll
        for (int j = 0; j < NTW; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0;
        // this lane's ldmatrix row of column tile tile0, + 8 rows per further
        // tile (a padding column reads a row past the window's used rows,
        // still inside the window and filter copies; its result is dropped)
        const uint32_t bbase = sig_s + (8 * (tile0 + (lane >> 4)) + (lane & 7)) * ROWB + 16 * kh;
        // shift u: A words at ya - T u, B rows of window block uch - 1 - u
        const uint32_t ya0 = smem_u32(gcp) + rho * GW + PADB - rho + T * uch - 16 * mt - gq + 4 * tq;
        const uint32_t boff0 = (uch - 1) * MS * ROWB;
#pragma unroll 2
        for (int u = 0; u < uch; u++) {
            const uint32_t ya = ya0 - T * u;
            const uint32_t boff = boff0 - u * (MS * ROWB);
#pragma unroll
            for (int ks = 0; ks < 2; ks++) {
                uint32_t af[4];
                af[0] = lds32(ya + 32 * ks);
                af[1] = lds32(ya + 32 * ks - 8);
                af[2] = lds32(ya + 32 * ks + 16);
                af[3] = lds32(ya + 32 * ks + 8);
#pragma unroll
                for (int jj = 0; jj < NTW; jj += 2) {
                    if (jj >= ntile) break;
                    uint32_t bf[4];
                    ldsm_x4(bf, bbase + boff + 8 * jj * ROWB + 32 * ks);
                    mma_s8(acc[jj], af, bf[0], bf[1]);
                    if (jj + 1 < ntile) mma_s8(acc[jj + 1], af, bf[2], bf[3]);
                }
            }
        }
#pragma unroll
        for (int jj = 0; jj < NTW; jj++) {
            if (jj >= ntile) break;
#pragma unroll
            for (int h = 0; h < 4; h++) {
                const int c = 8 * (tile0 + jj) + 2 * tq + (h & 1);
                const int q = 16 * mt + gq + 8 * (h >> 1);
                if (c < cols) {
                    const int pr = c / MS, ms = c - pr * MS;
                    stash[(ms * NPB + pr) * SP + q] = acc[jj][h];
                }
            }
        }
    } else {
        // -- dp4a pipe: thread t = 4 k + rho owns outputs i0 + 4 r, i0 = npb T + rho + 4 R k --
        const int t = tid - 32 * TW;               // 0 .. DT - 1
        const int rho = t & 3, k = t >> 2;
        const int rr = (4 - rho) & 3;              // the copy whose words start at i0's byte shift
        const int i0 = npb * T + rho + 4 * R * k;
        // F(m), the word of filter bytes g[(i0 - 4 m - e) mod N], e = 0..3, sits at
        // byte gd + 4 m of copy rr (m >= 1 - R keeps every read inside the copy)
        const uint32_t gd = smem_u32(gdp) + gdp_off(rr, R) + N + 4 - rr - i0;
        int acc[R][MS];
#pragma unroll
        for (int r = 0; r < R; r++)
#pragma unroll
            for (int ms = 0; ms < MS; ms++) acc[r][ms] = 0;
        // f[w] = F(J0 - (R - 1) + w): output i0 + 4 r at chunk J0 + e takes f[R - 1 + e - r]
        uint32_t f[R + 1];
#pragma unroll
        for (int w = 0; w < R - 1; w++) f[w] = lds32(gd + 4 * (w - (R - 1)));
        for (int jb = 0; jb < NB; jb++) {
            const int blk_rel = (jb + uch - 1) % NB;     // where input block jb sits in the window
            const uint32_t srow = sig_s + blk_rel * MS * ROWB;
            // 8 inputs (chunks J0, J0 + 1) per step: every accumulator takes two
            // dependent dp4a, the R x planes accumulators are independent
#pragma unroll
            for (int jh = 0; jh < T / 8; jh++) {
                const int J0 = jb * (T / 4) + 2 * jh;
                f[R - 1] = lds32(gd + 4 * J0);
                f[R] = lds32(gd + 4 * (J0 + 1));
                uint2 x[MS];
#pragma unroll
                for (int ms = 0; ms < MS; ms++) x[ms] = lds64(srow + ms * ROWB + 8 * jh);   // the same for every lane
#pragma unroll
                for (int ms = 0; ms < MS; ms++)
#pragma unroll
                    for (int r = 0; r < R; r++) acc[r][ms] = __dp4a((int)x[ms].x, (int)f[R - 1 - r], acc[r][ms]);
#pragma unroll
                for (int ms = 0; ms < MS; ms++)
#pragma unroll
                    for (int r = 0; r < R; r++) acc[r][ms] = __dp4a((int)x[ms].y, (int)f[R - r], acc[r][ms]);
#pragma unroll
                for (int w = 0; w < R - 1; w++) f[w] = f[w + 2];
            }
        }
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int o = rho + 4 * (R * k + r);   // output index - npb * T
#pragma unroll
            for (int ms = 0; ms < MS; ms++) stash[(ms * NPB + npb + o / T) * SP + o % T] = acc[r][ms];
        }
    }
    __syncthreads();
    epilogue<MT, 2>(a, stash, 0, NB, NTHR);
}

}  // namespace cconv
}  // namespace ne
