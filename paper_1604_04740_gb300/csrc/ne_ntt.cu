// Batched circular convolution of the entangled streams through an exact
// number-theoretic transform: the integer-exact counterpart of the
// frequency-domain convolution the paper measures (Sec. V), fused with the
// entanglement of Eq. 16 in front and the extraction/check of Eq. 17-20 and
// Eq. 24 (or the recovery of Prop. 3) behind it.  One launch goes from the raw
// int32 streams to the extracted outputs and check flags.
//
// Arithmetic.  Every entangled word is split into the balanced base-256
// digits of the caller's digit plan (each digit in [-128, 127]; every byte of
// every word that the plan does not store is checked to be a zero digit).  The
// circular convolution of one digit plane with the int8 filter is bounded by
// N * 2^14 = 2^24 in magnitude, below P / 2 for the prime P = 77 * 2^19 + 1,
// so its residue modulo P determines it exactly.  The words are the
// shift-and-add of their digits' convolutions in wrapping 64-bit arithmetic,
// exact whenever the true outputs fit the w = 64 word (the choice of l).
//
// Transform.  N = 1024 = 32 x 32 in the four-step form: one warp owns one
// transform and lane t holds elements t, t + 32, ..., t + 992.  Each lane
// runs a radix-2 32-point transform in registers (its twiddles are
// compile-time constants), the 1024-point twiddles W^(t k) are applied from a
// shared-memory table, a padded 32 x 33 shared-memory transpose exchanges the
// two index digits, and a second 32-point register transform finishes.  The
// inverse runs the same steps backwards; the 1/N factor is folded into the
// filter's transform.  P < 2^26 leaves room for the five butterfly stages of
// a 32-point transform to run without any modular reduction: stage t maps
// residues below 2^(t+1) P to residues below 2^(t+2) P, so a transform takes
// inputs below 2P to outputs below 64P < 2^32, and only the twiddle products
// (Shoup) and pointwise products (Montgomery) bring them back below 2P.
//
// CTA: persistent over groups.  Warp w < M*S transforms digit s = w % S of
// stream m = w / S; warp M*S transforms the filter.  After the inverse
// transforms every warp writes its centred residues to shared memory and the
// whole CTA recombines the digits and extracts 32 positions per warp.
#include <type_traits>

#include "ne_common.cuh"
#include "ne_entangle.cuh"
#include "ne_extract.cuh"
#include "ne_faults.cuh"

namespace {

using namespace ne;

namespace ntt {

constexpr uint32_t P = 40370177u;    // 77 * 2^19 + 1, prime
constexpr uint32_t GEN = 3u;         // a primitive root modulo P
constexpr int N = 1024;
constexpr int PAD = 33;              // row stride of the transpose buffers (conflict-free)
constexpr int BUF = 32 * PAD;        // words per warp buffer

static_assert((uint64_t)64 * P < ((uint64_t)1 << 32), "unreduced residues below 64P must fit 32 bits");
static_assert((uint64_t)N * 128 * 128 <= P / 2, "a digit plane's convolution must be recoverable from its residue");
static_assert((P - 1) % N == 0, "P must have N-th roots of unity");

__host__ __device__ constexpr uint32_t mulmod(uint32_t a, uint32_t b) { return (uint32_t)((uint64_t)a * b % P); }

__host__ __device__ constexpr uint32_t powmod(uint32_t a, uint64_t e) {
    uint32_t r = 1;
    while (e) {
        if (e & 1) r = mulmod(r, a);
        a = mulmod(a, a);
        e >>= 1;
    }
    return r;
}

// floor(w 2^32 / P): the precomputed quotient of Shoup's modular product
__host__ __device__ constexpr uint32_t shoup(uint32_t w) { return (uint32_t)(((uint64_t)w << 32) / P); }

// -P^-1 mod 2^32 by Newton's iteration (each step doubles the correct low bits)
__host__ __device__ constexpr uint32_t neg_inv() {
    uint32_t x = P;
    for (int i = 0; i < 5; i++) x *= 2u - P * x;
    return 0u - x;
}

constexpr uint32_t W = powmod(GEN, (P - 1) / N);   // primitive N-th root of unity
constexpr uint32_t WI = powmod(W, N - 1);          // its inverse
constexpr uint32_t W32 = powmod(W, 32);            // primitive 32nd root
constexpr uint32_t W32I = powmod(WI, 32);
constexpr uint32_t PNEG = neg_inv();
constexpr uint32_t Q1 = (uint32_t)((((uint64_t)1) << 32) / P);      // Shoup quotient of 1
constexpr uint32_t R1 = (uint32_t)(((uint64_t)1 << 32) % P);          // 2^32 mod P
constexpr uint32_t NINV = powmod((uint32_t)N, P - 2);
// Montgomery product of x with GSCALE = x 2^32 / N mod P, so that a later
// Montgomery product with it multiplies by x / N
constexpr uint32_t GSCALE = mulmod(mulmod(R1, R1), NINV);

static_assert(powmod(W, N / 2) == P - 1, "W must have order exactly N");
static_assert(mulmod(W, WI) == 1, "WI must invert W");
static_assert((uint32_t)(P * (0u - PNEG)) == 1u, "PNEG must be -P^-1 mod 2^32");

// A twiddle and its Shoup quotient, read together (one 8-byte load)
struct __align__(8) Tw {
    uint32_t w, q;
};

// 1024-point twiddles of the four-step form, tw[a * 32 + b] = W^(a b), and
// their inverses
struct Tables {
    Tw tw[N], twi[N];
};

constexpr Tables make_tables() {
    Tables t{};
    uint32_t pw = 1, pwi = 1;
    uint32_t pows[N] = {}, powsi[N] = {};
    for (int i = 0; i < N; i++) {
        pows[i] = pw;
        powsi[i] = pwi;
        pw = mulmod(pw, W);
        pwi = mulmod(pwi, WI);
    }
    for (int a = 0; a < 32; a++)
        for (int b = 0; b < 32; b++) {
            const int e = (a * b) % N;
            t.tw[a * 32 + b].w = pows[e];
            t.tw[a * 32 + b].q = shoup(pows[e]);
            t.twi[a * 32 + b].w = powsi[e];
            t.twi[a * 32 + b].q = shoup(powsi[e]);
        }
    return t;
}

__device__ const Tables g_tables = make_tables();

__host__ __device__ constexpr int rev5(int k) {
    return ((k & 1) << 4) | ((k & 2) << 2) | (k & 4) | ((k & 8) >> 2) | ((k & 16) >> 4);
}

template <int I, int END, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < END) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, END>(f);
    }
}

__device__ __forceinline__ uint32_t red1(uint32_t x) { return min(x, x - P); }    // [0, 2P) -> [0, P)

// x w mod P in [0, 2P) for any 32-bit x and w < P (Shoup)
__device__ __forceinline__ uint32_t mul_shoup(uint32_t x, uint32_t w, uint32_t wq) {
    return x * w - __umulhi(x, wq) * P;
}

// a b 2^-32 mod P in [0, 2P) for a b < P 2^32 (Montgomery)
__device__ __forceinline__ uint32_t mont(uint32_t a, uint32_t b) {
    const uint64_t t = (uint64_t)a * b;
    const uint32_t lo = (uint32_t)t, hi = (uint32_t)(t >> 32);
    return hi + __umulhi(lo * PNEG, P) + (lo != 0u ? 1u : 0u);
}

// In-register 32-point transform, radix 2, decimation in frequency: on entry
// a[n] (natural order, residues below 2P); on return a[rev5(k)] holds
// sum_n w^(n k) a[n] with w = W32 (INV: W32I) as a residue below 64P.  No
// reductions: the inputs of stage t are below B = 2^(t+1) P, its sums below
// 2B, its differences u + B - v in (0, 2B), and the twiddled differences below
// 2P (Shoup).
template <bool INV>
__device__ __forceinline__ void dft32(uint32_t (&a)[32]) {
    static_for<0, 5>([&](auto st) {
        constexpr int t = decltype(st)::value;
        constexpr int h = 16 >> t;
        constexpr uint32_t B = (2u << t) * P;
        static_for<0, 16 / h>([&](auto blk) {
            constexpr int s = decltype(blk)::value * 2 * h;
            static_for<0, h>([&](auto jj) {
                constexpr int j = decltype(jj)::value;
                const uint32_t u = a[s + j], v = a[s + j + h];
                a[s + j] = u + v;
                const uint32_t d = u + B - v;
                if constexpr (j == 0) {
                    a[s + j + h] = d;
                } else {
                    constexpr uint32_t w = powmod(INV ? W32I : W32, (uint64_t)j * (16 / h));
                    constexpr uint32_t wq = shoup(w);
                    a[s + j + h] = mul_shoup(d, w, wq);
                }
            });
        });
    });
}

// Forward transform of the warp's 1024 residues (below 2P on entry).  On
// entry a[n1] = x[32 n1 + lane]; on return a[rev5(k2)] = X[lane + 32 k2] below
// 64P, X[k] = sum_n W^(n k) x[n].  Both passes share one copy of the code.
__device__ __forceinline__ void forward(uint32_t (&a)[32], uint32_t* buf, const Tw* tw, int lane) {
#pragma unroll 1
    for (int pass = 0; pass < 2; pass++) {
        dft32<false>(a);   // pass 0: a[rev5(k1)] = sum_n1 W32^(n1 k1) x[32 n1 + lane]
        if (pass == 1) break;
        static_for<0, 32>([&](auto kk) {
            constexpr int k1 = decltype(kk)::value;
            const Tw t = tw[k1 * 32 + lane];
            buf[k1 * PAD + lane] = mul_shoup(a[rev5(k1)], t.w, t.q);
        });
        __syncwarp();
        static_for<0, 32>([&](auto nn) {
            constexpr int n2 = decltype(nn)::value;
            a[n2] = buf[lane * PAD + n2];
        });
        __syncwarp();
    }
}

// Inverse transform without the 1/N factor.  On entry a[k2] = Y[lane + 32 k2]
// (natural order, below 2P); on return a[rev5(n1)] = sum_k W^(-n k) Y[k] at
// n = 32 n1 + lane, below 64P.
__device__ __forceinline__ void inverse(uint32_t (&a)[32], uint32_t* buf, const Tw* twi, int lane) {
#pragma unroll 1
    for (int pass = 0; pass < 2; pass++) {
        dft32<true>(a);    // pass 0: a[rev5(n2)] = sum_k2 W32^(-n2 k2) Y[lane + 32 k2]
        if (pass == 1) break;
        static_for<0, 32>([&](auto nn) {
            constexpr int n2 = decltype(nn)::value;
            const Tw t = twi[n2 * 32 + lane];
            buf[n2 * PAD + lane] = mul_shoup(a[rev5(n2)], t.w, t.q);
        });
        __syncwarp();
        static_for<0, 32>([&](auto kk) {
            constexpr int k1 = decltype(kk)::value;
            a[k1] = buf[lane * PAD + k1];
        });
        __syncwarp();
    }
}

}  // namespace ntt

struct NttArgs {
    const int32_t* c;           // [batch][M][N] raw streams
    const int8_t* g;            // [batch][N]
    int64_t* out;               // [batch][M][N]
    uint32_t* flags;            // [batch][N/32] or null
    unsigned long long* nflag;
    int32_t* status;
    int64_t batch;
    int M, S, MS, l, r, fuse, plain;
    int shift[NE_MAX_DIGITS];
    ne_faults faults;           // flat positions b * N + i (count 0: none)
    // generic digit split: bytes of a 64-bit word that hold no stored digit, and 0x80 in each
    uint64_t ns_mask, ns_want;
    // fast digit split (words of in-range inputs fit 32 bits): the input range
    // [lo, hi] is checked instead of every word
    uint32_t off32;
    int lo, hi;
};

constexpr size_t ntt_smem_bytes(int MS) {
    return sizeof(uint32_t) * (size_t)(5 * ntt::N + (MS + 1) * ntt::BUF);
}

// Digit s of the 32 words of this lane (positions 32 n1 + lane) as residues
// below 2P: FAST forms the words in 32 bits and checks the inputs against the
// plan's range; otherwise every 64-bit word is checked digit by digit.
// check_prev: cp is the input of a lost stream (never loaded as cm itself),
// so its range is checked here.
template <bool FAST>
__device__ __forceinline__ bool load_digits(const NttArgs& a, const int32_t* cm, const int32_t* cp, int sh,
                                            bool check_prev, uint32_t (&v)[32]) {
    using namespace ntt;
    if constexpr (FAST) {
        uint32_t worst = 0;
        const uint32_t span = (uint32_t)a.hi - (uint32_t)a.lo;
        const int up = 24 - sh;    // the digit's byte moved to the top, then sign-extended
#pragma unroll
        for (int n1 = 0; n1 < 32; n1++) {
            const int32_t x = __ldg(cm + 32 * n1);
            worst = max(worst, (uint32_t)x - (uint32_t)a.lo);
            uint32_t y = (uint32_t)x + a.off32;
            if (!a.plain) {
                const int32_t xp = __ldg(cp + 32 * n1);
                if (check_prev) worst = max(worst, (uint32_t)xp - (uint32_t)a.lo);
                y += (uint32_t)xp << a.l;
            }
            const int d = (int32_t)((y ^ 0x80808080u) << up) >> 24;
            v[n1] = (uint32_t)(d + (int)P);
        }
        return worst > span;
    } else {
        bool bad = false;
#pragma unroll
        for (int n1 = 0; n1 < 32; n1++) {
            const int32_t x = __ldg(cm + 32 * n1);
            const int64_t e = a.plain ? (int64_t)x : entangle_word(x, __ldg(cp + 32 * n1), a.l);
            const uint64_t y = (uint64_t)e + 0x8080808080808080ull;
            bad |= (y & a.ns_mask) != a.ns_want;
            const int d = (int)(int8_t)(uint8_t)(((uint32_t)(y >> sh) & 0xffu) ^ 0x80u);
            v[n1] = (uint32_t)(d + (int)P);
        }
        return bad;
    }
}

template <int MT, bool FAST>
__global__ void __launch_bounds__(448, 2) k_cconv_ntt(const NttArgs a) {
    using namespace ntt;
    constexpr int MR = MT ? MT : 16;
    extern __shared__ __align__(16) uint32_t sm[];
    Tw* tw = reinterpret_cast<Tw*>(sm);
    Tw* twi = tw + N;
    uint32_t* gm = sm + 4 * N;
    uint32_t* bufs = sm + 5 * N;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Mv = MT ? MT : a.M;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        tw[i] = g_tables.tw[i];
        twi[i] = g_tables.twi[i];
    }
    __syncthreads();
    uint32_t* buf = bufs + warp * BUF;
    const bool filter_warp = warp == a.MS;
    const bool digit_warp = warp < a.MS;
    const int m = digit_warp ? warp / a.S : 0;
    const int s = digit_warp ? warp - m * a.S : 0;
    const bool active = digit_warp && !(a.fuse == NE_FUSE_RECOVER && m == a.r);
    const int mp = m == 0 ? Mv - 1 : m - 1;
    for (int64_t b = blockIdx.x; b < a.batch; b += gridDim.x) {
        uint32_t v[32];
        if (active || filter_warp) {
            if (filter_warp) {
                const int8_t* gb = a.g + b * N + lane;
#pragma unroll
                for (int n1 = 0; n1 < 32; n1++) v[n1] = (uint32_t)((int)__ldg(gb + 32 * n1) + (int)P);
            } else {
                // Eq. 16 for the 32 positions of this lane, digit s of the plan
                const bool bad = load_digits<FAST>(a, a.c + (b * Mv + m) * N + lane, a.c + (b * Mv + mp) * N + lane,
                                                   a.shift[s], a.fuse == NE_FUSE_RECOVER && mp == a.r, v);
                if (bad && a.status) atomicExch(a.status, (int32_t)NE_ERANGE);
            }
            forward(v, buf, tw, lane);
            if (filter_warp) {
                // G 2^32 / N mod P, fully reduced, so that the Montgomery products below
                // multiply the streams' transforms by G / N
                static_for<0, 32>([&](auto kk) {
                    constexpr int k2 = decltype(kk)::value;
                    gm[lane + 32 * k2] = red1(mont(v[rev5(k2)], GSCALE));
                });
            }
        }
        __syncthreads();
        if (active) {
            uint32_t y[32];
            static_for<0, 32>([&](auto kk) {
                constexpr int k2 = decltype(kk)::value;
                y[k2] = mont(v[rev5(k2)], gm[lane + 32 * k2]);
            });
            inverse(y, buf, twi, lane);
            // the digit plane's convolution: reduce below P, centre into (-P/2, P/2]
            int32_t* res = reinterpret_cast<int32_t*>(buf);
            static_for<0, 32>([&](auto nn) {
                constexpr int n1 = decltype(nn)::value;
                const uint32_t x = red1(mul_shoup(y[rev5(n1)], 1u, Q1));
                res[32 * n1 + lane] = x > P / 2 ? (int32_t)(x - P) : (int32_t)x;
            });
        }
        __syncthreads();
        // recombine the digits of every stream and extract, 32 positions per warp
        // (l = 16 with the two digits at shifts 0 and 16, the byte-aligned plan of
        // int8-valued streams, with every shift a constant)
        const int32_t* resall = reinterpret_cast<const int32_t*>(bufs);
        const bool l16 = a.l == 16 && a.S == 2 && a.shift[0] == 0 && a.shift[1] == 16;
        const ne_faults& F = a.faults;
        int64_t f0 = 0, f1 = 0;                 // this group's faults
        if (F.count > 0) {
            f0 = fault_lower_bound(F.pos, 0, F.count, b * N);
            f1 = fault_lower_bound(F.pos, f0, F.count, (b + 1) * N);
        }
        for (int base = warp * 32; base < N; base += blockDim.x) {
            const int i = base + lane;
            int64_t rot[MR];
#pragma unroll
            for (int j = 0; j < MR; j++) {
                if (!MT && j >= Mv) break;
                int mm = a.r + j;
                if (mm >= Mv) mm -= Mv;
                uint64_t w = 0;
                if (!(a.fuse == NE_FUSE_RECOVER && j == 0)) {
                    if (l16) {
                        w = (uint64_t)(int64_t)resall[2 * mm * BUF + i] +
                            ((uint64_t)(int64_t)resall[(2 * mm + 1) * BUF + i] << 16);
                    } else {
                        for (int ss = 0; ss < a.S; ss++)
                            w += (uint64_t)(int64_t)resall[(mm * a.S + ss) * BUF + i] << a.shift[ss];
                    }
                    if (f1 > f0) w = (uint64_t)apply_faults((int64_t)w, F.pos, F.stream, F.bit, f0, f1, b * N + i, mm);
                }
                rot[j] = (int64_t)w;
            }
            uint32_t f = 0;
            if (a.fuse != NE_FUSE_NONE) {
                int64_t o[MR];
                const bool chk = a.fuse == NE_FUSE_EXTRACT_CHECK;
                f = (l16 ? extract_rot<MT>(rot, Mv, 16, chk, o) : extract_rot<MT>(rot, Mv, a.l, chk, o)) ? 1u : 0u;
#pragma unroll
                for (int j = 0; j < MR; j++) {
                    if (!MT && j >= Mv) break;
                    rot[j] = o[j];
                }
            }
#pragma unroll
            for (int j = 0; j < MR; j++) {
                if (!MT && j >= Mv) break;
                int mm = a.r + j;
                if (mm >= Mv) mm -= Mv;
                __stcs(a.out + (b * Mv + mm) * N + i, rot[j]);
            }
            if (a.fuse == NE_FUSE_EXTRACT_CHECK) {
                const uint32_t word = __ballot_sync(0xffffffffu, f != 0);
                if (lane == 0) {
                    if (a.flags) a.flags[b * (N / 32) + base / 32] = word;
                    if (a.nflag && word) atomicAdd(a.nflag, (unsigned long long)__popc(word));
                }
            }
        }
        __syncthreads();
    }
}

template <int MT, bool FAST>
ne_status launch_ntt_kernel(const NttArgs& a, cudaStream_t s) {
    const size_t smem = ntt_smem_bytes(a.MS);
    const int threads = 32 * (a.MS + 1);
    if (cudaFuncSetAttribute(k_cconv_ntt<MT, FAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return check_launch("ne_cconv_ntt: shared memory");
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cconv_ntt<MT, FAST>, threads, smem) !=
            cudaSuccess || per_sm < 1)
        return check_launch("ne_cconv_ntt: occupancy");
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (grid > a.batch) grid = a.batch;
    k_cconv_ntt<MT, FAST><<<(unsigned)grid, threads, smem, s>>>(a);
    return check_launch("ne_cconv_ntt");
}

template <int MT>
ne_status launch_ntt(const NttArgs& a, bool fast, cudaStream_t s) {
    return fast ? launch_ntt_kernel<MT, true>(a, s) : launch_ntt_kernel<MT, false>(a, s);
}

}  // namespace

extern "C" ne_status ne_cconv_ntt(ne_params p, ne_digits dg, const int32_t* c, const int8_t* g, int64_t* out,
                                  uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t N, int32_t fuse,
                                  int32_t r, int32_t plain, ne_faults faults, int32_t* status, cudaStream_t s) {
    ne_status st = validate_params(p);
    if (st) return st;
    if ((st = validate_digits(dg))) return st;
    if ((st = validate_faults(faults, "ne_cconv_ntt"))) return st;
    if (batch < 0) return fail(NE_EINVAL, "ne_cconv_ntt: batch < 0");
    if (N != ntt::N) return fail(NE_EINVAL, "ne_cconv_ntt: N=%lld; the transform length is %d", (long long)N, ntt::N);
    if (fuse < NE_FUSE_NONE || fuse > NE_FUSE_RECOVER) return fail(NE_EINVAL, "ne_cconv_ntt: fuse=%d", fuse);
    if (r < 0 || r >= p.M) return fail(NE_EINVAL, "ne_cconv_ntt: r=%d", r);
    if (plain && fuse != NE_FUSE_NONE) return fail(NE_EINVAL, "ne_cconv_ntt: the plain operation has no extraction");
    const int MS = p.M * dg.S;
    if (MS > 15) return fail(NE_EINVAL, "ne_cconv_ntt: M*S=%d exceeds 15 digit planes", MS);
    if (p.M > 16) return fail(NE_EINVAL, "ne_cconv_ntt: M=%d exceeds 16", p.M);
    unsigned long long* nf = reinterpret_cast<unsigned long long*>(nflag);
    if (nf && fuse == NE_FUSE_EXTRACT_CHECK && cudaMemsetAsync(nf, 0, sizeof(*nf), s) != cudaSuccess)
        return check_launch("ne_cconv_ntt: reset count");
    if (batch == 0) return NE_OK;
    if (!c || !g || !out) return fail(NE_EINVAL, "ne_cconv_ntt: null pointer");
    NttArgs a{};
    a.c = c;
    a.g = g;
    a.out = out;
    a.flags = fuse == NE_FUSE_EXTRACT_CHECK ? flags : nullptr;
    a.nflag = fuse == NE_FUSE_EXTRACT_CHECK ? nf : nullptr;
    a.status = status;
    a.batch = batch;
    a.M = p.M;
    a.S = dg.S;
    a.MS = MS;
    a.l = p.l;
    a.r = fuse == NE_FUSE_NONE ? 0 : r;
    a.fuse = fuse;
    a.plain = plain ? 1 : 0;
    a.faults = faults;
    uint64_t stored = 0;
    for (int i = 0; i < NE_MAX_DIGITS; i++) {
        a.shift[i] = i < dg.S ? dg.shift[i] : 0;
        if (i < dg.S) stored |= 0xffull << dg.shift[i];
    }
    a.ns_mask = ~stored;
    a.ns_want = 0x8080808080808080ull & ~stored;
    // The fast split trusts the digit set only when it is exactly the plan of its
    // recorded (l, lo, hi) (for the plain operation: one digit at shift 0 and a
    // range inside [-128, 127]); then in-range inputs form words whose digits are
    // all in the set and fit 32 bits, and checking the inputs suffices.
    bool fast = false;
    if (plain) {
        fast = dg.S == 1 && dg.shift[0] == 0 && dg.lo <= dg.hi && dg.lo >= -128 && dg.hi <= 127;
        a.off32 = 0x80808080u;
    } else if (dg.lo <= dg.hi && dg.l == p.l) {
        ne_digits ref;
        FastPlan F;
        if (ne_plan_digits(dg.l, dg.lo, dg.hi, &ref) == NE_OK && ref.S == dg.S) {
            fast = true;
            for (int i = 0; i < dg.S; i++) fast = fast && ref.shift[i] == dg.shift[i];
        }
        fast = fast && make_fast_plan(dg, p.l, &F);
        a.off32 = fast ? F.off : 0u;
    }
    a.lo = dg.lo;
    a.hi = dg.hi;
    switch (p.M) {
        case 3: return launch_ntt<3>(a, fast, s);
        case 4: return launch_ntt<4>(a, fast, s);
        case 5: return launch_ntt<5>(a, fast, s);
        default: return launch_ntt<0>(a, fast, s);
    }
}
