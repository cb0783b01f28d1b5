// Batched circular convolution of the entangled streams through exact
// number-theoretic transforms for any length N in [2, 65536] (the N = 1024
// single-launch kernel is in ne_ntt.cu), with the entanglement of Eq. 16 in
// front and the extraction/check of Eq. 17-20 / Eq. 24 (or the recovery of
// Prop. 3) behind it.  Shared by ne_cconv_ntt_any (uniform groups) and the
// ragged batch runner (a table of jobs).
//
// Arithmetic.  The words themselves are transformed, modulo two primes
// P1 = 77 * 2^19 + 1 and P2 = 69 * 2^19 + 1, and the circular convolution is
// rebuilt by the Chinese remainder theorem: exact whenever the outputs lie
// below P1 P2 / 2 > 2^49 in magnitude, which the host checks from the input
// range, l and N.  A power-of-two N is transformed at length L = N (cyclic);
// any other N at the next power of two L >= 2N - 1 (linear convolution of the
// zero-padded signals), folded back as y[n] = lin[n] + lin[n + N].
//
// Transform.  Radix 2, forward by decimation in frequency (natural order in,
// bit-reversed out), inverse by decimation in time (bit-reversed in, natural
// out), so the pointwise products need no reordering.  The G = logL - 14 <= 3
// stages whose butterflies span more than LB = 2^14 elements run in one pass
// over the workspace per direction, 2^G elements per thread in registers (the
// forward pass also forms the words from the inputs).  The 14 stages inside
// a block of LB elements run in one CTA of 512 threads holding 32 elements
// each in registers, in three groups of 5, 5 and 4 stages with two exchanges
// through shared memory; shorter transforms (L < LB) run radix 2 in shared
// memory.  Twiddles come from a table laid out by stage (entry h + j = the
// j-th power of the primitive 2h-th root), so the threads of a warp read
// consecutive entries.  Residues stay below 2P: sums are reduced once per
// butterfly, differences and twiddle products through Shoup products,
// pointwise products are Montgomery products with the filter's transform
// pre-scaled by 2^32 / L.
#include <mutex>

#include "ne_common.cuh"
#include "ne_entangle.cuh"
#include "ne_extract.cuh"
#include "ne_faults.cuh"
#include "ne_ntt_any.cuh"

namespace ne {
namespace ntt2 {

__host__ __device__ constexpr uint32_t prime(int q) { return q == 0 ? 40370177u : 36175873u; }
__host__ __device__ constexpr uint32_t generator(int q) { return q == 0 ? 3u : 7u; }
constexpr int LOGMAX = 17;
constexpr int LMAX = 1 << LOGMAX;
constexpr int LOGB = 14;
constexpr int LB = 1 << LOGB;
constexpr int BTHREADS = 512;

static_assert((uint64_t)4 * 40370177u < ((uint64_t)1 << 32), "lazy residues below 4P fit 32 bits");

struct Tw {
    uint32_t w, q;
};

// [prime][direction][LMAX]: entry h + j holds the j-th power of the
// primitive 2h-th root of unity (direction 1: of its inverse) and its Shoup
// quotient, for h = 1, 2, ..., LMAX / 2 and j < h
__device__ Tw g_tw[2][2][LMAX];

__host__ __device__ inline uint32_t mulmod(uint32_t a, uint32_t b, uint32_t P) {
    return (uint32_t)((uint64_t)a * b % P);
}

__host__ __device__ inline uint32_t powmod(uint32_t a, uint64_t e, uint32_t P) {
    uint32_t r = 1;
    while (e) {
        if (e & 1) r = mulmod(r, a, P);
        a = mulmod(a, a, P);
        e >>= 1;
    }
    return r;
}

__host__ __device__ inline uint32_t neg_inv(uint32_t P) {
    uint32_t x = P;
    for (int i = 0; i < 5; i++) x *= 2u - P * x;
    return 0u - x;
}

__global__ void k_tables() {
    const int total = 2 * 2 * LMAX;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int q = idx / (2 * LMAX), dir = (idx / LMAX) & 1, e = idx % LMAX;
        if (e == 0) {
            g_tw[q][dir][0] = Tw{1u, 0u};
            continue;
        }
        const uint32_t P = prime(q);
        const int h = 1 << (31 - __clz(e));          // the stage: e in [h, 2h)
        const int j = e - h;
        // primitive 2h-th root = g^((P - 1) / 2h); the inverse direction uses its inverse
        uint32_t root = powmod(generator(q), (P - 1) / (2 * (uint64_t)h), P);
        if (dir) root = powmod(root, P - 2, P);
        const uint32_t w = powmod(root, (uint64_t)j, P);
        g_tw[q][dir][e] = Tw{w, (uint32_t)(((uint64_t)w << 32) / P)};
    }
}

std::mutex g_tables_mu;
bool g_tables_ready[64];

}  // namespace ntt2

ne_status ntt_any_init_tables(cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return check_launch("ntt tables: device");
    std::lock_guard<std::mutex> lock(ntt2::g_tables_mu);
    if (ntt2::g_tables_ready[dev]) return NE_OK;
    ntt2::k_tables<<<256, 256, 0, s>>>();
    ne_status st = check_launch("ntt tables");
    if (st) return st;
    if (cudaStreamSynchronize(s) != cudaSuccess) return check_launch("ntt tables: sync");
    ntt2::g_tables_ready[dev] = true;
    return NE_OK;
}

bool ntt_any_exact(int M, int l, int64_t N, int32_t cmax_abs, bool plain) {
    // |delta| <= N * max|word| * 128 with max|word| = max|c| (2^l + 1)
    const long double word = (long double)cmax_abs * (plain ? 1.0L : ((long double)(1ull << l) + 1.0L));
    const long double bound = (long double)N * word * 128.0L;
    const long double half = (long double)ntt2::prime(0) * (long double)ntt2::prime(1) / 2.0L;
    (void)M;
    return bound < half;
}

int ntt_any_length(int64_t N, int* logL) {
    int lg = 0;
    while ((1ll << lg) < N) lg++;
    if ((1ll << lg) != N) {                      // not a power of two: linear, then folded
        lg = 0;
        while ((1ll << lg) < 2 * N - 1) lg++;
    }
    *logL = lg;
    return 1 << lg;
}

namespace ntt2 {

__device__ __forceinline__ uint32_t red2(uint32_t x, uint32_t P) { return min(x, x - 2u * P); }
__device__ __forceinline__ uint32_t red1(uint32_t x, uint32_t P) { return min(x, x - P); }
__device__ __forceinline__ uint32_t mul_shoup(uint32_t x, uint32_t w, uint32_t wq, uint32_t P) {
    return x * w - __umulhi(x, wq) * P;
}
__device__ __forceinline__ uint32_t mont(uint32_t a, uint32_t b, uint32_t P, uint32_t pneg) {
    const uint64_t t = (uint64_t)a * b;
    const uint32_t lo = (uint32_t)t, hi = (uint32_t)(t >> 32);
    return hi + __umulhi(lo * pneg, P) + (lo != 0u ? 1u : 0u);
}

__device__ __forceinline__ NJob job_of(const NJobs& J, int64_t b) {
    if (J.table) return J.table[b];
    NJob j = J.tmpl;
    j.c_off += b * J.c_stride;
    j.g_off += b * J.g_stride;
    j.out_off += b * J.out_stride;
    j.flag_off += b * J.flag_stride;
    j.ws_off += b * J.ws_stride;
    j.fault_key0 += b * J.fault_key_stride;
    return j;
}

// plane p of prime q of a job's workspace: planes 0..M-1 the streams, M the filter
__device__ __forceinline__ uint32_t* plane_ptr(const NttAnyArgs& a, const NJob& j, int p, int q) {
    return a.ws + j.ws_off + ((int64_t)p * 2 + q) * j.L;
}

__device__ __forceinline__ Tw twiddle(const Tw* tw, int idx) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(tw) + idx);
    return Tw{v.x, v.y};
}

// DIF butterfly (u, v) -> (u + v, (u - v) w); ONE: w = 1.  Inputs and outputs below 2P.
template <bool ONE = false>
__device__ __forceinline__ void bf_dif(uint32_t& u, uint32_t& v, Tw w, uint32_t P) {
    const uint32_t a = u, b = v;
    u = red2(a + b, P);
    v = ONE ? red2(a + 2u * P - b, P) : mul_shoup(a + 2u * P - b, w.w, w.q, P);
}

// DIT butterfly (u, v) -> (u + v w, u - v w); ONE: w = 1.
template <bool ONE = false>
__device__ __forceinline__ void bf_dit(uint32_t& u, uint32_t& v, Tw w, uint32_t P) {
    const uint32_t t = ONE ? v : mul_shoup(v, w.w, w.q, P);
    const uint32_t a = u;
    u = red2(a + t, P);
    v = red2(a + 2u * P - t, P);
}

// the residue of the word of stream p (Eq. 16, or the raw value) or of the
// filter (p = M) at position i < N, modulo both primes; *worst tracks the range
template <bool FILTER>
__device__ __forceinline__ void load_residues(const NttAnyArgs& a, const NJob& j, int p, int64_t i, uint32_t& r0,
                                              uint32_t& r1, uint32_t& worst) {
    if (!FILTER) {
        const int32_t x = __ldg(a.c + j.c_off + (int64_t)p * j.N + i);
        worst = max(worst, (uint32_t)x - (uint32_t)j.lo);
        int64_t e = x;
        if (!j.plain) {
            const int mp = p == 0 ? j.M - 1 : p - 1;
            const int32_t xp = __ldg(a.c + j.c_off + (int64_t)mp * j.N + i);
            // a lost stream is never loaded itself, but its inputs enter this word
            if (j.fuse == NE_FUSE_RECOVER && mp == j.r) worst = max(worst, (uint32_t)xp - (uint32_t)j.lo);
            e = entangle_word(x, xp, j.l);
        }
        // |e| < 2^41: shift into [0, 2^42) by a multiple of both primes, then reduce
        r0 = (uint32_t)((uint64_t)(e + (int64_t)prime(0) * (int64_t)(1 << 22)) % prime(0));
        r1 = (uint32_t)((uint64_t)(e + (int64_t)prime(1) * (int64_t)(1 << 22)) % prime(1));
    } else {
        const int d = __ldg(a.g + j.g_off + i);
        r0 = (uint32_t)(d + (int)prime(0));
        r1 = (uint32_t)(d + (int)prime(1));
    }
}

// One unit of the forward pass: the 2^G elements base + k Q (Q = L >> G) of
// plane p, loaded from the inputs, then the G outermost DIF stages (half-spans
// L/2 .. Q) in registers, both primes.
template <int G>
__device__ __forceinline__ void gfwd_unit(const NttAnyArgs& a, const NJob& j, int p, int base, uint32_t& worst) {
    constexpr int E = 1 << G;
    const int Q = j.L >> G;
    uint32_t r[2][E];
#pragma unroll
    for (int k = 0; k < E; k++) {
        const int64_t i = base + (int64_t)k * Q;
        r[0][k] = r[1][k] = 0;
        if (i < j.N) {
            if (p < j.M) load_residues<false>(a, j, p, i, r[0][k], r[1][k], worst);
            else load_residues<true>(a, j, p, i, r[0][k], r[1][k], worst);
        }
    }
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const uint32_t P = prime(q);
        const Tw* tw = g_tw[q][0];
#pragma unroll
        for (int s = 0; s < G; s++) {
            const int d = E >> (s + 1);                  // half-span Q d
#pragma unroll
            for (int k = 0; k < E; k++) {
                if (k & d) continue;
                bf_dif(r[q][k], r[q][k + d], twiddle(tw, Q * d + base + Q * (k & (d - 1))), P);
            }
        }
        uint32_t* x = plane_ptr(a, j, p, q);
#pragma unroll
        for (int k = 0; k < E; k++) x[base + (int64_t)k * Q] = r[q][k];
    }
}

// The words of Eq. 16 (or the raw values) and the filter, modulo both primes,
// zero padded to L, with the stages whose butterflies span more than LB
// elements (G = logL - 14 <= 3 of them) done in the same pass.
__global__ void __launch_bounds__(256) k_gfwd(const NttAnyArgs a) {
    for (int64_t b = blockIdx.y; b < a.jobs.njobs; b += gridDim.y) {
        const NJob j = job_of(a.jobs, b);
        if (j.L == 0) continue;
        const int G = j.logL > LOGB ? j.logL - LOGB : 0;
        const int Q = j.L >> G;
        const int64_t units = (int64_t)(j.M + 1) * Q;
        uint32_t worst = 0;
        for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += (int64_t)gridDim.x * blockDim.x) {
            const int p = (int)(u / Q);
            const int base = (int)(u - (int64_t)p * Q);
            if (p < j.M && j.fuse == NE_FUSE_RECOVER && p == j.r) continue;   // never computed
            switch (G) {
                case 0: gfwd_unit<0>(a, j, p, base, worst); break;
                case 1: gfwd_unit<1>(a, j, p, base, worst); break;
                case 2: gfwd_unit<2>(a, j, p, base, worst); break;
                default: gfwd_unit<3>(a, j, p, base, worst); break;
            }
        }
        if (worst > (uint32_t)j.hi - (uint32_t)j.lo && a.status) atomicExch(a.status, (int32_t)NE_ERANGE);
    }
}

// The inverse stages spanning more than LB elements (half-spans Q .. L/2,
// DIT) for the 2^G elements base + k Q of one plane and prime, in registers.
template <int G>
__device__ __forceinline__ void ginv_unit(const NttAnyArgs& a, const NJob& j, int p, int q, int base) {
    constexpr int E = 1 << G;
    const int Q = j.L >> G;
    const uint32_t P = prime(q);
    const Tw* tw = g_tw[q][1];
    uint32_t* x = plane_ptr(a, j, p, q);
    uint32_t r[E];
#pragma unroll
    for (int k = 0; k < E; k++) r[k] = x[base + (int64_t)k * Q];
#pragma unroll
    for (int s = 0; s < G; s++) {
        const int d = 1 << s;
#pragma unroll
        for (int k = 0; k < E; k++) {
            if (k & d) continue;
            bf_dit(r[k], r[k + d], twiddle(tw, Q * d + base + Q * (k & (d - 1))), P);
        }
    }
#pragma unroll
    for (int k = 0; k < E; k++) x[base + (int64_t)k * Q] = r[k];
}

__global__ void __launch_bounds__(256) k_ginv(const NttAnyArgs a) {
    for (int64_t b = blockIdx.y; b < a.jobs.njobs; b += gridDim.y) {
        const NJob j = job_of(a.jobs, b);
        if (j.L <= LB) continue;
        const int G = j.logL - LOGB;
        const int64_t units = (int64_t)j.M * 2 * LB;
        for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += (int64_t)gridDim.x * blockDim.x) {
            const int pq = (int)(u >> LOGB);
            const int base = (int)(u & (LB - 1));
            const int p = pq >> 1, q = pq & 1;
            if (j.fuse == NE_FUSE_RECOVER && p == j.r) continue;
            switch (G) {
                case 1: ginv_unit<1>(a, j, p, q, base); break;
                case 2: ginv_unit<2>(a, j, p, q, base); break;
                default: ginv_unit<3>(a, j, p, q, base); break;
            }
        }
    }
}

// ---- the 14 innermost stages of a block of LB = 2^14 elements ---------------------------------
//
// 512 threads hold 32 elements each in registers and run the stages in three
// groups, exchanging through shared memory between groups: index bits 13..9
// (element t + 512 k of thread t), bits 8..4 (element 512 hi + 16 k + lo of
// thread 16 hi + lo) and bits 3..0 (rows 16 g + kk, g = t and t + 512).  The
// word of element i in shared memory is swz(i) = i + i / 32 (one pad word per
// 32), with which each of the three patterns reads and writes 32 distinct
// banks per warp, and every address is a per-thread base plus a constant.

constexpr int RTHREADS = 512;
__host__ __device__ constexpr int swz(int i) { return i + (i >> 5); }
constexpr int RSMEM_WORDS = swz(LB - 1) + 1;

// bits 13..9: half-spans 512 d, d = 16 .. 1 (DIF) or 1 .. 16 (DIT)
template <bool INV>
__device__ __forceinline__ void stages_hi(uint32_t (&r)[32], const Tw* tw, int t, uint32_t P) {
#pragma unroll
    for (int s = 0; s < 5; s++) {
        const int d = INV ? (1 << s) : (16 >> s);
#pragma unroll
        for (int k = 0; k < 32; k++) {
            if (k & d) continue;
            const Tw w = twiddle(tw, 512 * d + t + 512 * (k & (d - 1)));
            if (INV) bf_dit(r[k], r[k + d], w, P);
            else bf_dif(r[k], r[k + d], w, P);
        }
    }
}

// bits 8..4: half-spans 16 d
template <bool INV>
__device__ __forceinline__ void stages_mid(uint32_t (&r)[32], const Tw* tw, int lo, uint32_t P) {
#pragma unroll
    for (int s = 0; s < 5; s++) {
        const int d = INV ? (1 << s) : (16 >> s);
#pragma unroll
        for (int k = 0; k < 32; k++) {
            if (k & d) continue;
            const Tw w = twiddle(tw, 16 * d + 16 * (k & (d - 1)) + lo);
            if (INV) bf_dit(r[k], r[k + d], w, P);
            else bf_dif(r[k], r[k + d], w, P);
        }
    }
}

// bits 3..0 of two rows of 16: half-spans d = 8 .. 1 (DIF) or 1 .. 8 (DIT);
// the first butterfly of every span has twiddle 1
template <bool INV>
__device__ __forceinline__ void stages_lo(uint32_t (&r)[32], const Tw* tw, uint32_t P) {
#pragma unroll
    for (int s = 0; s < 4; s++) {
        const int d = INV ? (1 << s) : (8 >> s);
#pragma unroll
        for (int kk = 0; kk < 16; kk++) {
            if (kk & d) continue;
            const int jj = kk & (d - 1);
            if (jj == 0) {
#pragma unroll
                for (int row = 0; row < 2; row++) {
                    if (INV) bf_dit<true>(r[16 * row + kk], r[16 * row + kk + d], Tw{1u, 0u}, P);
                    else bf_dif<true>(r[16 * row + kk], r[16 * row + kk + d], Tw{1u, 0u}, P);
                }
            } else {
                const Tw w = twiddle(tw, d + jj);
#pragma unroll
                for (int row = 0; row < 2; row++) {
                    if (INV) bf_dit(r[16 * row + kk], r[16 * row + kk + d], w, P);
                    else bf_dif(r[16 * row + kk], r[16 * row + kk + d], w, P);
                }
            }
        }
    }
}

// Forward (DIF, natural order in, bit-reversed out; the filter plane scaled by
// 2^32 / L, fully reduced) or inverse (pointwise product with the filter's
// transform, then DIT) of every LB-block of the jobs with L >= LB.
template <bool INV>
__global__ void __launch_bounds__(RTHREADS, 2) k_block_r(const NttAnyArgs a) {
    extern __shared__ uint32_t sx[];
    const int t = threadIdx.x;
    const int hi = t >> 4, lo = t & 15;
    for (int64_t b = blockIdx.y; b < a.jobs.njobs; b += gridDim.y) {
        const NJob j = job_of(a.jobs, b);
        if (j.L < LB) continue;
        const int nblk = j.L >> LOGB;
        const int planes = INV ? j.M : j.M + 1;
        for (int unit = blockIdx.x; unit < planes * 2 * nblk; unit += gridDim.x) {
            const int blk = unit % nblk, pq = unit / nblk;
            const int p = pq >> 1, q = pq & 1;
            if (p < j.M && j.fuse == NE_FUSE_RECOVER && p == j.r) continue;
            const uint32_t P = prime(q);
            const Tw* tw = g_tw[q][INV ? 1 : 0];
            uint32_t* x = plane_ptr(a, j, p, q) + (int64_t)blk * LB;
            uint32_t r[32];
            if (!INV) {
#pragma unroll
                for (int k = 0; k < 32; k++) r[k] = x[t + 512 * k];
                stages_hi<false>(r, tw, t, P);
#pragma unroll
                for (int k = 0; k < 32; k++) sx[swz(t + 512 * k)] = r[k];
                __syncthreads();
#pragma unroll
                for (int k = 0; k < 32; k++) r[k] = sx[swz(512 * hi + 16 * k + lo)];
                stages_mid<false>(r, tw, lo, P);
#pragma unroll
                for (int k = 0; k < 32; k++) sx[swz(512 * hi + 16 * k + lo)] = r[k];
                __syncthreads();
#pragma unroll
                for (int row = 0; row < 2; row++)
#pragma unroll
                    for (int kk = 0; kk < 16; kk++) r[16 * row + kk] = sx[swz(16 * (t + 512 * row) + kk)];
                stages_lo<false>(r, tw, P);
                if (p == j.M) {
                    // a Montgomery product with the scaled filter transform multiplies by G / L
                    const uint32_t pneg = neg_inv(P), gs = q ? j.gscale[1] : j.gscale[0];
#pragma unroll
                    for (int k = 0; k < 32; k++) r[k] = red1(mont(r[k], gs, P, pneg), P);
                }
#pragma unroll
                for (int row = 0; row < 2; row++) {
                    uint4* dst = reinterpret_cast<uint4*>(x + 16 * (t + 512 * row));
#pragma unroll
                    for (int v = 0; v < 4; v++)
                        dst[v] = make_uint4(r[16 * row + 4 * v], r[16 * row + 4 * v + 1], r[16 * row + 4 * v + 2],
                                            r[16 * row + 4 * v + 3]);
                }
            } else {
                const uint32_t* gm = plane_ptr(a, j, j.M, q) + (int64_t)blk * LB;
                const uint32_t pneg = neg_inv(P);
#pragma unroll
                for (int row = 0; row < 2; row++) {
                    const uint4* src = reinterpret_cast<const uint4*>(x + 16 * (t + 512 * row));
                    const uint4* gsrc = reinterpret_cast<const uint4*>(gm + 16 * (t + 512 * row));
#pragma unroll
                    for (int v = 0; v < 4; v++) {
                        const uint4 xv = src[v], gv = __ldg(gsrc + v);
                        r[16 * row + 4 * v] = mont(xv.x, gv.x, P, pneg);
                        r[16 * row + 4 * v + 1] = mont(xv.y, gv.y, P, pneg);
                        r[16 * row + 4 * v + 2] = mont(xv.z, gv.z, P, pneg);
                        r[16 * row + 4 * v + 3] = mont(xv.w, gv.w, P, pneg);
                    }
                }
                stages_lo<true>(r, tw, P);
#pragma unroll
                for (int row = 0; row < 2; row++)
#pragma unroll
                    for (int kk = 0; kk < 16; kk++) sx[swz(16 * (t + 512 * row) + kk)] = r[16 * row + kk];
                __syncthreads();
#pragma unroll
                for (int k = 0; k < 32; k++) r[k] = sx[swz(512 * hi + 16 * k + lo)];
                stages_mid<true>(r, tw, lo, P);
#pragma unroll
                for (int k = 0; k < 32; k++) sx[swz(512 * hi + 16 * k + lo)] = r[k];
                __syncthreads();
#pragma unroll
                for (int k = 0; k < 32; k++) r[k] = sx[swz(t + 512 * k)];
                stages_hi<true>(r, tw, t, P);
#pragma unroll
                for (int k = 0; k < 32; k++) x[t + 512 * k] = r[k];
            }
            __syncthreads();        // the next unit reuses sx
        }
    }
}

// all stages of a job with L < LB, radix 2 in shared memory (forward:
// half-spans L/2 .. 1; inverse: the pointwise product with the filter first,
// then half-spans 1 .. L/2)
template <bool INV>
__global__ void __launch_bounds__(BTHREADS) k_block(const NttAnyArgs a) {
    extern __shared__ uint32_t sx[];
    for (int64_t b = blockIdx.y; b < a.jobs.njobs; b += gridDim.y) {
        const NJob j = job_of(a.jobs, b);
        if (j.L == 0 || j.L >= LB) continue;
        const int B = j.L;
        const int nblk = 1;
        const int planes = INV ? j.M : j.M + 1;
        for (int unit = blockIdx.x; unit < planes * 2 * nblk; unit += gridDim.x) {
            const int blk = unit % nblk, pq = unit / nblk;
            const int p = pq >> 1, q = pq & 1;
            if (p < j.M && j.fuse == NE_FUSE_RECOVER && p == j.r) continue;
            const uint32_t P = prime(q);
            uint32_t* x = plane_ptr(a, j, p, q) + (int64_t)blk * B;
            for (int i = threadIdx.x; i < B; i += blockDim.x) sx[i] = x[i];
            if (INV) {
                const uint32_t* gm = plane_ptr(a, j, j.M, q) + (int64_t)blk * B;
                const uint32_t pneg = neg_inv(P);
                for (int i = threadIdx.x; i < B; i += blockDim.x) sx[i] = mont(sx[i], gm[i], P, pneg);
            }
            __syncthreads();
            const Tw* tw = g_tw[q][INV ? 1 : 0];
            for (int st = 0; st < 31; st++) {
                const int h = INV ? (1 << st) : (B >> (st + 1));
                if (h < 1 || h >= B) break;
                for (int t = threadIdx.x; t < B / 2; t += blockDim.x) {
                    const int jj = t & (h - 1);
                    const int i0 = ((t - jj) << 1) + jj, i1 = i0 + h;
                    const Tw w = tw[h + jj];
                    const uint32_t u0 = sx[i0], v0 = sx[i1];
                    if (!INV) {
                        sx[i0] = red2(u0 + v0, P);
                        sx[i1] = mul_shoup(u0 + 2u * P - v0, w.w, w.q, P);
                    } else {
                        const uint32_t v = mul_shoup(v0, w.w, w.q, P);
                        sx[i0] = red2(u0 + v, P);
                        sx[i1] = red2(u0 + 2u * P - v, P);
                    }
                }
                __syncthreads();
            }
            if (!INV && p == j.M) {
                // the filter's transform times 2^32 / L, fully reduced: a Montgomery
                // product with it multiplies by G / L
                const uint32_t pneg = neg_inv(P);
                const uint32_t gs = q ? j.gscale[1] : j.gscale[0];
                for (int i = threadIdx.x; i < B; i += blockDim.x) x[i] = red1(mont(sx[i], gs, P, pneg), P);
            } else {
                for (int i = threadIdx.x; i < B; i += blockDim.x) x[i] = sx[i];
            }
            __syncthreads();
        }
    }
}

// fold, CRT, extraction / check / faults of one job, 32 positions per warp
template <int MT>
__device__ __forceinline__ void final_job(const NttAnyArgs& a, const NJob& j) {
    constexpr int MR = MT ? MT : 16;
    const int lane = threadIdx.x & 31;
    const uint32_t P1 = prime(0), P2 = prime(1);
    const uint32_t inv = a.crt_inv, invq = a.crt_invq;           // P1^-1 mod P2 and its Shoup quotient
    const uint64_t PP = (uint64_t)P1 * P2;
    {
        const int Mv = MT ? MT : j.M;
        const bool folded = j.L != j.N;
        for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; base < j.N;
             base += (int64_t)gridDim.x * blockDim.x) {
            const int64_t n = base + lane;
            const bool valid = n < j.N;
            int64_t f0 = 0, f1 = 0;                                   // this warp's faults
            if (a.fault_pos && j.fault_end > j.fault_begin) {
                f0 = fault_lower_bound(a.fault_pos, j.fault_begin, j.fault_end, j.fault_key0 + base);
                f1 = fault_lower_bound(a.fault_pos, f0, j.fault_end, j.fault_key0 + base + 32);
            }
            int64_t rot[MR];
#pragma unroll
            for (int jj = 0; jj < MR; jj++) {
                if (!MT && jj >= Mv) break;
                int m = j.r + jj;
                if (m >= Mv) m -= Mv;
                int64_t v = 0;
                if (valid && !(j.fuse == NE_FUSE_RECOVER && jj == 0)) {
                    uint32_t x[2];
#pragma unroll
                    for (int q = 0; q < 2; q++) {
                        const uint32_t P = prime(q);
                        const uint32_t* y = plane_ptr(a, j, m, q);
                        uint32_t r = red1(y[n], P);
                        if (folded) r = red1(r + red1(y[n + j.N], P), P);
                        x[q] = r;
                    }
                    // CRT: v = x1 + P1 ((x2 - x1) P1^-1 mod P2), centred
                    const uint32_t x1m = x[0] >= P2 ? x[0] - P2 : x[0];
                    const uint32_t d = x[1] >= x1m ? x[1] - x1m : x[1] + P2 - x1m;
                    const uint32_t t = red1(mul_shoup(d, inv, invq, P2), P2);
                    uint64_t y = (uint64_t)x[0] + (uint64_t)P1 * t;
                    v = y > PP / 2 ? (int64_t)(y - PP) : (int64_t)y;
                    if (f1 > f0)                                          // transient faults
                        v = apply_faults(v, a.fault_pos, a.fault_stream, a.fault_bit, f0, f1, j.fault_key0 + n, m);
                }
                rot[jj] = v;
            }
            bool flag = false;
            if (valid) {
                if (j.fuse != NE_FUSE_NONE) {
                    int64_t o[MR];
                    // constant shifts for the byte-aligned l of int8-valued streams
                    const bool chk = j.fuse == NE_FUSE_EXTRACT_CHECK;
                    flag = j.l == 16  ? extract_rot<MT>(rot, Mv, 16, chk, o)
                           : j.l == 8 ? extract_rot<MT>(rot, Mv, 8, chk, o)
                                      : extract_rot<MT>(rot, Mv, j.l, chk, o);
#pragma unroll
                    for (int jj = 0; jj < MR; jj++) {
                        if (!MT && jj >= Mv) break;
                        rot[jj] = o[jj];
                    }
                }
#pragma unroll
                for (int jj = 0; jj < MR; jj++) {
                    if (!MT && jj >= Mv) break;
                    int m = j.r + jj;
                    if (m >= Mv) m -= Mv;
                    a.out[j.out_off + (int64_t)m * j.N + n] = rot[jj];
                }
            }
            if (j.fuse == NE_FUSE_EXTRACT_CHECK) {
                const uint32_t w = __ballot_sync(0xffffffffu, flag);
                if (lane == 0) {
                    if (a.flags) {
                        if (a.flags_atomic) {
                            if (w) atomicOr(a.flags + j.flag_off + base / 32, w);
                        } else {
                            a.flags[j.flag_off + base / 32] = w;
                        }
                    }
                    if (a.nflag && w) atomicAdd(a.nflag, (unsigned long long)__popc(w));
                }
            }
        }
    }
}

// MT = 3, 4, 5: the jobs with that M; MT = 0: the jobs with M > 5
template <int MT>
__global__ void __launch_bounds__(256) k_final(const NttAnyArgs a) {
    for (int64_t b = blockIdx.y; b < a.jobs.njobs; b += gridDim.y) {
        const NJob j = job_of(a.jobs, b);
        if (j.L == 0 || (MT ? j.M != MT : j.M <= 5)) continue;
        final_job<MT>(a, j);
    }
}

// a table of jobs with M in 3 .. 5, each on the code for its M (one launch)
__global__ void __launch_bounds__(256) k_final_mixed(const NttAnyArgs a) {
    for (int64_t b = blockIdx.y; b < a.jobs.njobs; b += gridDim.y) {
        const NJob j = job_of(a.jobs, b);
        if (j.L == 0) continue;
        switch (j.M) {
            case 3: final_job<3>(a, j); break;
            case 4: final_job<4>(a, j); break;
            case 5: final_job<5>(a, j); break;
            default: break;            // M > 5: k_final<0>
        }
    }
}

}  // namespace ntt2

void ntt_any_job_constants(NJob& j) {
    for (int q = 0; q < 2; q++) {
        const uint32_t P = ntt2::prime(q);
        const uint32_t r1 = (uint32_t)((((uint64_t)1) << 32) % P);
        const uint32_t linv = ntt2::powmod((uint32_t)(j.L % P), P - 2, P);
        j.gscale[q] = ntt2::mulmod(ntt2::mulmod(r1, r1, P), linv, P);
    }
}

ne_status ntt_any_run(NttAnyArgs& a, int min_logL, int max_logL, int max_M, int64_t max_units_load,
                      cudaStream_t s) {
    ne_status st = ntt_any_init_tables(s);
    if (st) return st;
    const uint32_t inv = ntt2::powmod(ntt2::prime(0) % ntt2::prime(1), ntt2::prime(1) - 2, ntt2::prime(1));
    a.crt_inv = inv;
    a.crt_invq = (uint32_t)(((uint64_t)inv << 32) / ntt2::prime(1));
    const int64_t nj = a.jobs.njobs;
    const unsigned gy = (unsigned)(nj < 65535 ? nj : 65535);
    const int sms = sm_count();
    auto gx_for = [&](int64_t units, int threads) {
        int64_t want = (units + threads - 1) / threads;
        const int64_t cap = (int64_t)sms * 8 * 4 / (gy > 0 ? gy : 1) + 1;
        if (want > cap) want = cap;
        if (want < 1) want = 1;
        return (unsigned)want;
    };
    ntt2::k_gfwd<<<dim3(gx_for(max_units_load, 256), gy), 256, 0, s>>>(a);
    if ((st = check_launch("ne_cconv_ntt_any: load and outer forward stages"))) return st;
    static bool attr[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        cudaFuncSetAttribute(ntt2::k_block<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ntt2::LB / 2 * 4);
        cudaFuncSetAttribute(ntt2::k_block<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ntt2::LB / 2 * 4);
        cudaFuncSetAttribute(ntt2::k_block_r<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             ntt2::RSMEM_WORDS * 4);
        cudaFuncSetAttribute(ntt2::k_block_r<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             ntt2::RSMEM_WORDS * 4);
        attr[dev] = true;
    }
    // jobs with L >= LB: register-resident blocks of LB; shorter jobs: one block of L
    const bool big = max_logL >= ntt2::LOGB, small = min_logL < ntt2::LOGB;
    const int nblk = big ? (1 << max_logL) / ntt2::LB : 1;
    const int small_logL = max_logL < ntt2::LOGB ? max_logL : ntt2::LOGB - 1;
    const size_t rsmem = (size_t)ntt2::RSMEM_WORDS * 4, smem = ((size_t)1 << small_logL) * 4;
    if (big) {
        ntt2::k_block_r<false><<<dim3((unsigned)((max_M + 1) * 2 * nblk), gy), ntt2::RTHREADS, rsmem, s>>>(a);
        if ((st = check_launch("ne_cconv_ntt_any: forward blocks"))) return st;
    }
    if (small) {
        ntt2::k_block<false><<<dim3((unsigned)((max_M + 1) * 2), gy), ntt2::BTHREADS, smem, s>>>(a);
        if ((st = check_launch("ne_cconv_ntt_any: forward blocks"))) return st;
    }
    if (big) {
        ntt2::k_block_r<true><<<dim3((unsigned)(max_M * 2 * nblk), gy), ntt2::RTHREADS, rsmem, s>>>(a);
        if ((st = check_launch("ne_cconv_ntt_any: inverse blocks"))) return st;
    }
    if (small) {
        ntt2::k_block<true><<<dim3((unsigned)(max_M * 2), gy), ntt2::BTHREADS, smem, s>>>(a);
        if ((st = check_launch("ne_cconv_ntt_any: inverse blocks"))) return st;
    }
    if (max_logL > ntt2::LOGB) {
        ntt2::k_ginv<<<dim3(gx_for((int64_t)max_M * 2 * ntt2::LB, 256), gy), 256, 0, s>>>(a);
        if ((st = check_launch("ne_cconv_ntt_any: outer inverse stages"))) return st;
    }
    const int64_t maxN = (int64_t)1 << max_logL;
    const unsigned fx = gx_for(maxN, 256);
    if (a.jobs.table) {
        // a table may mix M: one launch for M in 3 .. 5, another for larger M
        ntt2::k_final_mixed<<<dim3(fx, gy), 256, 0, s>>>(a);
        if (max_M > 5) ntt2::k_final<0><<<dim3(fx, gy), 256, 0, s>>>(a);
        return check_launch("ne_cconv_ntt_any: final");
    }
    switch (max_M) {
        case 3: ntt2::k_final<3><<<dim3(fx, gy), 256, 0, s>>>(a); break;
        case 4: ntt2::k_final<4><<<dim3(fx, gy), 256, 0, s>>>(a); break;
        case 5: ntt2::k_final<5><<<dim3(fx, gy), 256, 0, s>>>(a); break;
        default: ntt2::k_final<0><<<dim3(fx, gy), 256, 0, s>>>(a); break;
    }
    return check_launch("ne_cconv_ntt_any: final");
}

}  // namespace ne

using namespace ne;

extern "C" int64_t ne_cconv_ntt_any_workspace(int32_t M, int64_t N, int64_t batch) {
    if (M < 1 || N < 2 || N > 65536 || batch < 0) return -1;
    int lg = 0;
    const int64_t L = ntt_any_length(N, &lg);
    return batch * (int64_t)(M + 1) * 2 * L * (int64_t)sizeof(uint32_t);
}

extern "C" ne_status ne_cconv_ntt_any(ne_params p, int32_t cmin, int32_t cmax, const int32_t* c, const int8_t* g,
                                      int64_t* out, uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t N,
                                      int32_t fuse, int32_t r, int32_t plain, ne_faults faults, int32_t* status,
                                      void* workspace, int64_t workspace_bytes, cudaStream_t s) {
    ne_status st = validate_params(p);
    if (st) return st;
    if ((st = validate_faults(faults, "ne_cconv_ntt_any"))) return st;
    if (batch < 0 || N < 2 || N > 65536) return fail(NE_EINVAL, "ne_cconv_ntt_any: N=%lld must be in [2, 65536]",
                                                     (long long)N);
    if (cmin > cmax) return fail(NE_EINVAL, "ne_cconv_ntt_any: empty input range");
    if (fuse < NE_FUSE_NONE || fuse > NE_FUSE_RECOVER) return fail(NE_EINVAL, "ne_cconv_ntt_any: fuse=%d", fuse);
    if (r < 0 || r >= p.M) return fail(NE_EINVAL, "ne_cconv_ntt_any: r=%d", r);
    if (plain && fuse != NE_FUSE_NONE) return fail(NE_EINVAL, "ne_cconv_ntt_any: the plain operation has no extraction");
    if (p.M > 16) return fail(NE_EINVAL, "ne_cconv_ntt_any: M=%d exceeds 16", p.M);
    const int32_t cabs = (int32_t)(-(int64_t)cmin > (int64_t)cmax ? -(int64_t)cmin : (int64_t)cmax);
    if (!ntt_any_exact(p.M, p.l, N, cabs, plain != 0))
        return fail(NE_ERANGE, "ne_cconv_ntt_any: outputs may exceed the two-prime range (N, l, input range)");
    unsigned long long* nf = reinterpret_cast<unsigned long long*>(nflag);
    if (nf && fuse == NE_FUSE_EXTRACT_CHECK && cudaMemsetAsync(nf, 0, sizeof(*nf), s) != cudaSuccess)
        return check_launch("ne_cconv_ntt_any: reset count");
    if (batch == 0) return NE_OK;
    if (!c || !g || !out || !workspace) return fail(NE_EINVAL, "ne_cconv_ntt_any: null pointer");
    if (batch > 65535) return fail(NE_EINVAL, "ne_cconv_ntt_any: batch %lld exceeds 65535 groups", (long long)batch);
    const int64_t need = ne_cconv_ntt_any_workspace(p.M, N, batch);
    if (workspace_bytes < need || !aligned(workspace, 16))
        return fail(NE_EINVAL, "ne_cconv_ntt_any: workspace needs %lld bytes, 16-byte aligned", (long long)need);
    NttAnyArgs a{};
    NJob& j = a.jobs.tmpl;
    int lg = 0;
    j.L = ntt_any_length(N, &lg);
    j.logL = lg;
    j.M = p.M;
    j.N = (int32_t)N;
    j.l = p.l;
    j.r = fuse == NE_FUSE_NONE ? 0 : r;
    j.fuse = fuse;
    j.plain = plain ? 1 : 0;
    j.lo = cmin;
    j.hi = cmax;
    j.fault_begin = 0;
    j.fault_end = faults.count;
    j.fault_key0 = 0;
    ntt_any_job_constants(j);
    a.jobs.table = nullptr;
    a.jobs.njobs = batch;
    a.jobs.c_stride = (int64_t)p.M * N;
    a.jobs.g_stride = N;
    a.jobs.out_stride = (int64_t)p.M * N;
    a.jobs.flag_stride = (N + 31) / 32;
    a.jobs.ws_stride = (int64_t)(p.M + 1) * 2 * j.L;
    a.jobs.fault_key_stride = N;
    a.c = c;
    a.g = g;
    a.out = out;
    a.flags = fuse == NE_FUSE_EXTRACT_CHECK ? flags : nullptr;
    a.nflag = fuse == NE_FUSE_EXTRACT_CHECK ? nf : nullptr;
    a.flags_atomic = 0;
    a.status = status;
    a.ws = static_cast<uint32_t*>(workspace);
    a.fault_pos = faults.count > 0 ? faults.pos : nullptr;
    a.fault_stream = faults.stream;
    a.fault_bit = faults.bit;
    return ntt_any_run(a, lg, lg, p.M, (int64_t)(p.M + 1) * j.L, s);
}
