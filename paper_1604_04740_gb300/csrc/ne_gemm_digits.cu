// Matrix product of entangled streams on the int8 tensor path (the GEMM of
// Sec. V, applied per Eq. 10) with the extraction and check of Eq. 17-20 /
// Eq. 24 fused into the epilogue.
//
// Every entangled word is held as balanced base-256 digit planes, so
//     delta_m = sum_s 2^shift_s (sigma_{m,s} G),
// where each sigma_{m,s} G is an exact int8 x int8 -> int32 product
// (|partial| <= k 2^14 < 2^31 for k <= 131071).
//
// A CTA owns a 32 x 64 output tile of ALL M*S planes, one warp per plane
// (2 x 8 mma.m16n8k32 tiles, int32 accumulators in registers), so the tile
// of every stream is on chip when the epilogue runs: the digits are
// recombined exactly in int64 and the extraction/check runs per position
// with the same device code as the stand-alone kernel; delta never reaches
// HBM.  The shared operand G tile (64 k x 64 n) is read once per stage and
// used by every plane.  mma.sync wants both operands K-major; G is stored
// n-major, so each thread loads a 4 x 4 byte block of it and transposes the
// block in registers (byte permutes) on the way into shared memory.  The
// digit-plane tiles arrive by cp.async in a 3-stage pipeline.
#include "ne_common.cuh"
#include "ne_extract.cuh"
#include "ne_faults.cuh"
#include "ne_mma.cuh"

namespace {

using namespace ne;

constexpr int BM = 32, BN = 64, BK = 64;
constexpr int STAGES = 3;
constexpr int RB = 80;                  // shared-memory row stride (bytes): 64 data + 16 pad
constexpr int A_STAGE_PER_PLANE = BM * RB;
constexpr int B_STAGE = BN * RB;
constexpr int SB = 68;                  // stash row stride (int32)
constexpr int KMAX = 131056;            // largest k with no int32 overflow (multiple of 16)

struct GemmArgs {
    const int8_t* planes;   // [M][S][rows][k]
    const int8_t* G;        // [k][cols]
    int64_t* out;           // [M][rows][cols]
    uint32_t* flags;        // bitmap over i*cols + j, or null
    unsigned long long* nflag;
    int rows, cols, k;
    int M, S, MS, l, r, fuse;
    int direct_flags;       // cols % 32 == 0: each warp owns whole bitmap words
    int shift[NE_MAX_DIGITS];
    ne_faults faults;       // flat positions i * cols + j (count 0: none)
    // words form (WORDS): the entangled words themselves [M][rows][k], split
    // into the digits of the plan while the tiles load; a word whose bytes
    // outside the plan's digits differ from the balanced split's (y & ns_mask
    // != ns_want, y = word + 0x80..80) sets *status = NE_ERANGE
    const int64_t* words;
    int32_t* status;
    uint64_t ns_mask, ns_want;
};

// The S digit bytes of 16 words (already offset by 0x80 in every byte) as S
// rows of 16 bytes: row s holds byte shift[s] / 8 of each word XOR 0x80.
__device__ __forceinline__ void store_digit_rows(const uint64_t (&y)[16], const int* shift, int S, uint8_t* dst,
                                                 int row_stride) {
#pragma unroll
    for (int s = 0; s < NE_MAX_DIGITS; s++) {
        if (s >= S) break;
        const int sh = shift[s];
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t v0 = (uint32_t)(y[4 * q] >> sh), v1 = (uint32_t)(y[4 * q + 1] >> sh);
            const uint32_t v2 = (uint32_t)(y[4 * q + 2] >> sh), v3 = (uint32_t)(y[4 * q + 3] >> sh);
            w[q] = __byte_perm(__byte_perm(v0, v1, 0x0040), __byte_perm(v2, v3, 0x0040), 0x5410) ^ 0x80808080u;
        }
        *reinterpret_cast<uint4*>(dst + s * row_stride) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

int smem_bytes(int MS) {
    const int pipe = STAGES * (MS * A_STAGE_PER_PLANE + B_STAGE);
    const int stash = MS * BM * SB * 4;
    return pipe > stash ? pipe : stash;
}

__device__ __forceinline__ int64_t shl64(int64_t x, int s) { return (int64_t)((uint64_t)x << s); }

// 4x4 byte transpose: r[e] holds row e (bytes = columns 0..3); returns columns.
__device__ __forceinline__ void transpose4x4(const uint32_t (&r)[4], uint32_t (&c)[4]) {
    const uint32_t t0 = __byte_perm(r[0], r[1], 0x5140);
    const uint32_t t1 = __byte_perm(r[0], r[1], 0x7362);
    const uint32_t t2 = __byte_perm(r[2], r[3], 0x5140);
    const uint32_t t3 = __byte_perm(r[2], r[3], 0x7362);
    c[0] = __byte_perm(t0, t2, 0x5410);
    c[1] = __byte_perm(t0, t2, 0x7632);
    c[2] = __byte_perm(t1, t3, 0x5410);
    c[3] = __byte_perm(t1, t3, 0x7632);
}

template <int MT>
__device__ __forceinline__ void gemm_epilogue(const GemmArgs& a, const int32_t* stash, int row0, int col0) {
    const int M = MT ? MT : a.M;
    const int S = a.S;
    const int nthreads = blockDim.x;
    const int lane = threadIdx.x & 31;
    const bool check = (a.fuse == NE_FUSE_EXTRACT_CHECK);
    const bool need_r = (a.fuse != NE_FUSE_RECOVER);
    const int64_t plane = (int64_t)a.rows * a.cols;
    // the faults of this tile's row band (every thread finds the same range)
    const ne_faults& F = a.faults;
    int64_t f0 = 0, f1 = 0;
    if (F.count > 0) {
        const int last_row = min(row0 + BM, a.rows) - 1;
        f0 = fault_lower_bound(F.pos, 0, F.count, (int64_t)row0 * a.cols + col0);
        f1 = fault_lower_bound(F.pos, f0, F.count, (int64_t)last_row * a.cols + min(col0 + BN, a.cols));
    }
    for (int base = threadIdx.x & ~31; base < BM * BN; base += nthreads) {
        const int idx = base + lane;
        const int i = idx / BN, j = idx % BN;
        const int gi = row0 + i, gj = col0 + j;
        const bool valid = gi < a.rows && gj < a.cols;
        const int32_t* sp = stash + i * SB + j;
        const int64_t pos = (int64_t)gi * a.cols + gj;
        bool f = false;
        if (valid) {
            if (a.fuse == NE_FUSE_NONE) {
                for (int m = 0; m < M; m++) {
                    int64_t v = 0;
#pragma unroll
                    for (int s = 0; s < NE_MAX_DIGITS; s++)
                        if (s < S) v += shl64(sp[(m * S + s) * BM * SB], a.shift[s]);
                    if (f1 > f0) v = apply_faults(v, F.pos, F.stream, F.bit, f0, f1, pos, m);
                    a.out[m * plane + pos] = v;
                }
            } else {
                int64_t rot[MT ? MT : 32], res[MT ? MT : 32];
#pragma unroll
                for (int jj = 0; jj < (MT ? MT : 32); jj++) {
                    if (!MT && jj >= M) break;
                    int m = a.r + jj;
                    if (m >= M) m -= M;
                    int64_t v = 0;
                    if (jj > 0 || need_r) {
#pragma unroll
                        for (int s = 0; s < NE_MAX_DIGITS; s++)
                            if (s < S) v += shl64(sp[(m * S + s) * BM * SB], a.shift[s]);
                        if (f1 > f0) v = apply_faults(v, F.pos, F.stream, F.bit, f0, f1, pos, m);
                    }
                    rot[jj] = v;
                }
                f = extract_rot<MT>(rot, M, a.l, check, res);
#pragma unroll
                for (int jj = 0; jj < (MT ? MT : 32); jj++) {
                    if (!MT && jj >= M) break;
                    int m = a.r + jj;
                    if (m >= M) m -= M;
                    a.out[m * plane + pos] = res[jj];
                }
            }
        }
        if (check) {
            if (a.direct_flags) {
                // the warp's 32 positions are one bitmap word (same row, 32-aligned columns)
                const uint32_t w = __ballot_sync(0xffffffffu, f);
                if (lane == 0 && gi < a.rows && col0 + (base % BN) < a.cols) {
                    if (a.flags) a.flags[((int64_t)gi * a.cols + col0 + (base % BN)) / 32] = w;
                    if (a.nflag && w) atomicAdd(a.nflag, (unsigned long long)__popc(w));
                }
            } else if (f) {
                if (a.flags) atomicOr(&a.flags[pos >> 5], 1u << (pos & 31));
                if (a.nflag) atomicAdd(a.nflag, 1ull);
            }
        }
    }
}

// RAGGED: k not a multiple of 16, cols not of 4, or an operand not aligned for
// the vector loads; the loads then go element by element
template <int MT, bool WORDS, bool RAGGED>
__global__ void __launch_bounds__(512, 1) k_gemm_digits(GemmArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int MS = a.MS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthreads = blockDim.x;
    const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
    const int K = a.k, rows = a.rows, cols = a.cols;
    const int KT = (K + BK - 1) / BK;
    const int plane = warp;   // one warp per digit plane
    const int stream_of_plane = plane / a.S;
    const bool lost_plane = (a.fuse == NE_FUSE_RECOVER) && (stream_of_plane == a.r);

    uint8_t* As = smem;                                      // [STAGES][MS][BM][RB]
    uint8_t* Bs = smem + STAGES * MS * A_STAGE_PER_PLANE;    // [STAGES][BN][RB] (G transposed)
    const uint32_t As_s = smem_u32(As), Bs_s = smem_u32(Bs);

    // A loads: MS planes x 32 rows x 4 chunks of 16 bytes
    auto load_A = [&](int stage, int kt) {
        const int k0 = kt * BK;
        if constexpr (WORDS) {
            // M streams x 32 rows x 4 chunks of 16 words, split into S digit rows each
            bool bad = false;
            for (int e = tid; e < a.M * BM * 4; e += nthreads) {
                const int c16 = e & 3, r = (e >> 2) % BM, m = (e >> 2) / BM;
                const int gi = row0 + r, gk = k0 + 16 * c16;
                const bool ok = gi < rows && gk < K && !((a.fuse == NE_FUSE_RECOVER) && m == a.r);
                uint64_t y[16];
                if (ok && RAGGED) {
                    // rows of any length: word by word, past k the word 0
                    const int64_t* src = a.words + ((int64_t)m * rows + gi) * K + gk;
#pragma unroll
                    for (int q = 0; q < 16; q++) {
                        y[q] = (gk + q < K ? (uint64_t)__ldg(src + q) : 0ull) + 0x8080808080808080ull;
                        bad |= (y[q] & a.ns_mask) != a.ns_want;
                    }
                } else if (ok) {
                    const longlong2* src =
                        reinterpret_cast<const longlong2*>(a.words + ((int64_t)m * rows + gi) * K + gk);
#pragma unroll
                    for (int q = 0; q < 8; q++) {
                        const longlong2 v = __ldg(src + q);
                        y[2 * q] = (uint64_t)v.x + 0x8080808080808080ull;
                        y[2 * q + 1] = (uint64_t)v.y + 0x8080808080808080ull;
                    }
#pragma unroll
                    for (int q = 0; q < 16; q++) bad |= (y[q] & a.ns_mask) != a.ns_want;
                } else {
#pragma unroll
                    for (int q = 0; q < 16; q++) y[q] = 0x8080808080808080ull;    // digits 0
                }
                store_digit_rows(y, a.shift, a.S, As + ((stage * MS + m * a.S) * BM + r) * RB + 16 * c16, BM * RB);
            }
            if (bad && a.status) atomicExch(a.status, (int32_t)NE_ERANGE);
            return;
        }
        const int nchunks = MS * BM * 4;
        for (int e = tid; e < nchunks; e += nthreads) {
            const int c16 = e & 3, r = (e >> 2) % BM, pl = (e >> 2) / BM;
            const int gi = row0 + r, gk = k0 + 16 * c16;
            const bool ok = gi < rows && gk < K && !((a.fuse == NE_FUSE_RECOVER) && (pl / a.S == a.r));
            const int8_t* src = a.planes + ((int64_t)pl * rows + (ok ? gi : 0)) * K + (ok ? gk : 0);
            if constexpr (RAGGED) {
                // rows that do not start 16-byte aligned: byte by byte, past k zero
                uint32_t w[4] = {0u, 0u, 0u, 0u};
                if (ok) {
#pragma unroll
                    for (int b = 0; b < 16; b++)
                        if (gk + b < K) w[b >> 2] |= (uint32_t)(uint8_t)__ldg(src + b) << (8 * (b & 3));
                }
                *reinterpret_cast<uint4*>(As + ((stage * MS + pl) * BM + r) * RB + 16 * c16) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            } else {
                cp_async16(As_s + ((stage * MS + pl) * BM + r) * RB + 16 * c16, src, ok ? 16 : 0);
            }
        }
    };
    // G loads: 4x4 byte blocks (kb, nb) -> registers
    const int nblk = (BK / 4) * (BN / 4);   // 256
    auto load_G = [&](int kt, uint32_t (&reg)[2][4]) {
        const int k0 = kt * BK;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = tid + h * nthreads;
#pragma unroll
            for (int q = 0; q < 4; q++) reg[h][q] = 0;
            if (e < nblk) {
                const int nb = e % (BN / 4), kb = e / (BN / 4);
                const int gn = col0 + 4 * nb;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int gk = k0 + 4 * kb + q;
                    if (gk < K && gn < cols) {
                        if constexpr (RAGGED) {
                            // rows of G of any length: byte by byte, past cols zero
                            uint32_t x = 0;
#pragma unroll
                            for (int c = 0; c < 4; c++)
                                if (gn + c < cols) x |= (uint32_t)(uint8_t)__ldg(a.G + (int64_t)gk * cols + gn + c) << (8 * c);
                            reg[h][q] = x;
                        } else {
                            reg[h][q] = __ldg(reinterpret_cast<const uint32_t*>(a.G + (int64_t)gk * cols + gn));
                        }
                    }
                }
            }
        }
    };
    auto store_G = [&](int stage, const uint32_t (&reg)[2][4]) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = tid + h * nthreads;
            if (e < nblk) {
                const int nb = e % (BN / 4), kb = e / (BN / 4);
                uint32_t c[4];
                transpose4x4(reg[h], c);
#pragma unroll
                for (int q = 0; q < 4; q++)
                    *reinterpret_cast<uint32_t*>(Bs + (stage * BN + 4 * nb + q) * RB + 4 * kb) = c[q];
            }
        }
    };

    int acc[2][8][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0;

    uint32_t greg[2][4];
#pragma unroll
    for (int st = 0; st < STAGES - 1; st++) {
        if (st < KT) {
            load_A(st, st);
            load_G(st, greg);
            store_G(st, greg);
        }
        cp_async_commit();
    }

    for (int kt = 0; kt < KT; kt++) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        const int pf = kt + STAGES - 1;
        if (pf < KT) {
            load_A(pf % STAGES, pf);
            load_G(pf, greg);
        }
        cp_async_commit();
        const int st = kt % STAGES;
        if (!lost_plane) {
#pragma unroll
            for (int ks = 0; ks < 2; ks++) {
                const int t0 = 32 * ks;
                uint32_t af[2][4];
#pragma unroll
                for (int mi = 0; mi < 2; mi++)
                    ldsm_x4(af[mi], As_s + ((st * MS + plane) * BM + 16 * mi + (lane & 15)) * RB + t0 + 16 * (lane >> 4));
#pragma unroll
                for (int nj = 0; nj < 8; nj += 2) {
                    uint32_t bf[4];
                    const int n = 8 * (nj + (lane >> 4)) + (lane & 7);
                    ldsm_x4(bf, Bs_s + (st * BN + n) * RB + t0 + 16 * ((lane >> 3) & 1));
#pragma unroll
                    for (int mi = 0; mi < 2; mi++) {
                        mma_s8(acc[mi][nj], af[mi], bf[0], bf[1]);
                        mma_s8(acc[mi][nj + 1], af[mi], bf[2], bf[3]);
                    }
                }
            }
        }
        if (pf < KT) store_G(pf % STAGES, greg);
    }
    cp_async_wait<0>();
    __syncthreads();

    // int32 digit products -> stash [plane][BM][SB]
    int32_t* stash = reinterpret_cast<int32_t*>(smem);
    const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; mi++)
#pragma unroll
        for (int nj = 0; nj < 8; nj++)
#pragma unroll
            for (int h = 0; h < 4; h++) {
                const int i = 16 * mi + gq + 8 * (h >> 1);
                const int j = 8 * nj + 2 * tq + (h & 1);
                stash[(plane * BM + i) * SB + j] = acc[mi][nj][h];
            }
    __syncthreads();
    gemm_epilogue<MT>(a, stash, row0, col0);
}

template <int MT, bool WORDS, bool RAGGED>
ne_status launch(const GemmArgs& a, cudaStream_t s) {
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(k_gemm_digits<MT, WORDS, RAGGED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_bytes(16)) != cudaSuccess)
            return check_launch("ne_gemm_digits: shared-memory attribute");
        attr_set[dev] = true;
    }
    dim3 grid((a.cols + BN - 1) / BN, (a.rows + BM - 1) / BM);
    k_gemm_digits<MT, WORDS, RAGGED><<<grid, a.MS * 32, smem_bytes(a.MS), s>>>(a);
    return check_launch("ne_gemm_digits");
}

template <bool WORDS, bool RAGGED>
ne_status dispatch_m(const GemmArgs& a, cudaStream_t s) {
    switch (a.M) {
        case 3: return launch<3, WORDS, RAGGED>(a, s);
        case 4: return launch<4, WORDS, RAGGED>(a, s);
        case 5: return launch<5, WORDS, RAGGED>(a, s);
        default: return launch<0, WORDS, RAGGED>(a, s);
    }
}

template <bool WORDS>
ne_status dispatch(const GemmArgs& a, cudaStream_t s) {
    const void* A = WORDS ? (const void*)a.words : (const void*)a.planes;
    const bool ragged = a.k % 16 != 0 || a.cols % 4 != 0 || !aligned(A, 16) || !aligned(a.G, 4);
    return ragged ? dispatch_m<WORDS, true>(a, s) : dispatch_m<WORDS, false>(a, s);
}


// The tensor-path product from digit planes (planes non-null) or from the
// entangled words themselves (words non-null, split in the loader).
ne_status gemm_tensor(const char* who, ne_params p, ne_digits dg, const int8_t* planes, const int64_t* words,
                      const int8_t* G, int64_t* out, uint32_t* flags, uint64_t* nflag, int32_t rows, int32_t cols,
                      int32_t k, int32_t fuse, int32_t r, const ne_faults& faults, int32_t* status, cudaStream_t s) {
    ne_status st = validate_params(p);
    if (st) return st;
    if ((st = validate_digits(dg))) return st;
    if ((st = validate_faults(faults, who))) return st;
    if (rows < 0 || cols < 0 || k < 0) return fail(NE_EINVAL, "%s: negative size", who);
    if (k > KMAX) return fail(NE_EINVAL, "%s: k=%d exceeds %d", who, k, KMAX);
    if (fuse < NE_FUSE_NONE || fuse > NE_FUSE_RECOVER) return fail(NE_EINVAL, "%s: fuse=%d", who, fuse);
    if (r < 0 || r >= p.M) return fail(NE_EINVAL, "%s: r=%d", who, r);
    const int MS = p.M * dg.S;
    if (MS > 16) return fail(NE_EINVAL, "%s: M*S=%d exceeds 16 planes", who, MS);
    if ((int64_t)(rows + BM - 1) / BM > 65535) return fail(NE_EINVAL, "%s: rows too large", who);
    unsigned long long* nf = reinterpret_cast<unsigned long long*>(nflag);
    if (nf && cudaMemsetAsync(nf, 0, sizeof(*nf), s) != cudaSuccess)
        return check_launch("digit-plane product: reset count");
    if (rows == 0 || cols == 0) return NE_OK;
    if ((!planes && !words) || !G || !out) return fail(NE_EINVAL, "%s: null pointer", who);
    if (!aligned(out, 8) || (words && !aligned(words, 8)))
        return fail(NE_EINVAL, "%s: out (and eps) must be 8-byte aligned", who);
    GemmArgs a;
    a.planes = planes;
    a.G = G;
    a.out = out;
    a.rows = rows;
    a.cols = cols;
    a.k = k;
    a.M = p.M;
    a.S = dg.S;
    a.MS = MS;
    a.l = p.l;
    a.r = r;
    a.fuse = fuse;
    a.direct_flags = (cols % 32 == 0);
    a.flags = (fuse == NE_FUSE_EXTRACT_CHECK) ? flags : nullptr;
    a.nflag = (fuse == NE_FUSE_EXTRACT_CHECK) ? nf : nullptr;
    uint64_t stored = 0;
    for (int i = 0; i < NE_MAX_DIGITS; i++) {
        a.shift[i] = i < dg.S ? dg.shift[i] : 0;
        if (i < dg.S) stored |= 0xffull << dg.shift[i];
    }
    a.faults = faults;
    a.words = words;
    a.status = status;
    a.ns_mask = ~stored;
    a.ns_want = 0x8080808080808080ull & ~stored;
    if (a.flags && !a.direct_flags) {
        const size_t nw = ((size_t)rows * cols + 31) / 32;
        if (cudaMemsetAsync(a.flags, 0, nw * 4, s) != cudaSuccess) return check_launch("digit-plane product: flags");
    }
    // k = 0 needs no special case: the tile loop is empty, every product is 0
    return words ? dispatch<true>(a, s) : dispatch<false>(a, s);
}

}  // namespace

namespace ne {

ne_status gemm_s8slice(ne_params p, ne_digits dg, const int64_t* words, const int8_t* G, int64_t* out,
                       uint32_t* flags, uint64_t* nflag, int32_t rows, int32_t cols, int32_t k, int32_t fuse,
                       int32_t r, const ne_faults& faults, int32_t* status, cudaStream_t s) {
    return gemm_tensor("ne_gemm (S8SLICE)", p, dg, nullptr, words, G, out, flags, nflag, rows, cols, k, fuse, r,
                       faults, status, s);
}

}  // namespace ne

extern "C" ne_status ne_gemm_digits(ne_params p, ne_digits dg, const int8_t* planes, const int8_t* G, int64_t* out,
                                    uint32_t* flags, uint64_t* nflag, int32_t rows, int32_t cols, int32_t k,
                                    int32_t fuse, int32_t r, ne_faults faults, cudaStream_t s) {
    return gemm_tensor("ne_gemm_digits", p, dg, planes, nullptr, G, out, flags, nflag, rows, cols, k, fuse, r, faults,
                       nullptr, s);
}
