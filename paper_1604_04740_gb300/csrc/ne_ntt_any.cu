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
// out), so the pointwise products need no reordering.  Stages whose
// butterflies span more than LB = 2^14 elements run as passes over the
// workspace (one launch per stage); the remaining 14 stages run in shared
// memory, one CTA per contiguous block of LB elements.  Twiddles come from a
// table laid out by stage (entry h + j = the j-th power of the primitive
// 2h-th root), so the threads of a warp read consecutive entries.  Residues
// stay below 2P: sums are reduced once per butterfly, differences and
// twiddle products through Shoup products, pointwise products are Montgomery
// products with the filter's transform pre-scaled by 2^32 / L.
#include <mutex>

#include "ne_common.cuh"
#include "ne_entangle.cuh"
#include "ne_extract.cuh"
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
    return j;
}

// plane p of prime q of a job's workspace: planes 0..M-1 the streams, M the filter
__device__ __forceinline__ uint32_t* plane_ptr(const NttAnyArgs& a, const NJob& j, int p, int q) {
    return a.ws + j.ws_off + ((int64_t)p * 2 + q) * j.L;
}

// words of Eq. 16 (or the raw values) and the filter, both primes, zero padded
__global__ void __launch_bounds__(256) k_load(const NttAnyArgs a) {
    for (int64_t b = blockIdx.y; b < a.jobs.njobs; b += gridDim.y) {
        const NJob j = job_of(a.jobs, b);
        if (j.L == 0) continue;
        const int64_t units = (int64_t)(j.M + 1) * j.L;
        uint32_t worst = 0;
        for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += (int64_t)gridDim.x * blockDim.x) {
            const int p = (int)(u / j.L);
            const int i = (int)(u - (int64_t)p * j.L);
            if (p < j.M && j.fuse == NE_FUSE_RECOVER && p == j.r) continue;   // never computed
            uint32_t r0 = 0, r1 = 0;
            if (i < j.N) {
                if (p < j.M) {
                    const int32_t x = __ldg(a.c + j.c_off + (int64_t)p * j.N + i);
                    worst = max(worst, (uint32_t)x - (uint32_t)j.lo);
                    int64_t e = x;
                    if (!j.plain) {
                        const int mp = p == 0 ? j.M - 1 : p - 1;
                        e = entangle_word(x, __ldg(a.c + j.c_off + (int64_t)mp * j.N + i), j.l);
                    }
                    // |e| < 2^41: shift into [0, 2^42) by a multiple of both primes, then reduce
                    const uint64_t shifted0 = (uint64_t)(e + (int64_t)prime(0) * (int64_t)(1 << 22));
                    const uint64_t shifted1 = (uint64_t)(e + (int64_t)prime(1) * (int64_t)(1 << 22));
                    r0 = (uint32_t)(shifted0 % prime(0));
                    r1 = (uint32_t)(shifted1 % prime(1));
                } else {
                    const int d = __ldg(a.g + j.g_off + i);
                    r0 = (uint32_t)(d + (int)prime(0));
                    r1 = (uint32_t)(d + (int)prime(1));
                }
            }
            plane_ptr(a, j, p, 0)[i] = r0;
            plane_ptr(a, j, p, 1)[i] = r1;
        }
        if (worst > (uint32_t)j.hi - (uint32_t)j.lo && a.status) atomicExch(a.status, (int32_t)NE_ERANGE);
    }
}

// one butterfly stage over the workspace for every job with L > LB: forward
// DIF with half-span h = L >> (s + 1), inverse DIT with h = LB << s
template <bool INV>
__global__ void __launch_bounds__(256) k_stage(const NttAnyArgs a, int s) {
    for (int64_t b = blockIdx.y; b < a.jobs.njobs; b += gridDim.y) {
        const NJob j = job_of(a.jobs, b);
        if (j.L <= LB || s >= j.logL - LOGB) continue;
        const int h = INV ? (LB << s) : (j.L >> (s + 1));     // inverse: spans grow, forward: they shrink
        const int64_t half = j.L / 2;
        const int64_t units = (int64_t)(j.M + 1) * 2 * half;
        for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += (int64_t)gridDim.x * blockDim.x) {
            const int pq = (int)(u / half);
            const int64_t t = u - (int64_t)pq * half;
            const int p = pq >> 1, q = pq & 1;
            if (INV && p == j.M) continue;                                  // the filter has no inverse
            if (p < j.M && j.fuse == NE_FUSE_RECOVER && p == j.r) continue;
            const uint32_t P = prime(q);
            uint32_t* x = plane_ptr(a, j, p, q);
            const int jj = (int)(t & (h - 1));
            const int64_t i0 = ((t - jj) << 1) + jj, i1 = i0 + h;
            const Tw w = g_tw[q][INV ? 1 : 0][h + jj];
            const uint32_t u0 = x[i0], v0 = x[i1];
            if (!INV) {
                x[i0] = red2(u0 + v0, P);
                x[i1] = mul_shoup(u0 + 2u * P - v0, w.w, w.q, P);
            } else {
                const uint32_t v = mul_shoup(v0, w.w, w.q, P);
                x[i0] = red2(u0 + v, P);
                x[i1] = red2(u0 + 2u * P - v, P);
            }
        }
    }
}

// the stages within one block of B = min(L, LB) elements, in shared memory
// (forward: half-spans B/2 .. 1; inverse: the pointwise product with the
// filter first, then half-spans 1 .. B/2)
template <bool INV>
__global__ void __launch_bounds__(BTHREADS) k_block(const NttAnyArgs a) {
    extern __shared__ uint32_t sx[];
    for (int64_t b = blockIdx.y; b < a.jobs.njobs; b += gridDim.y) {
        const NJob j = job_of(a.jobs, b);
        if (j.L == 0) continue;
        const int B = j.L < LB ? j.L : LB;
        const int nblk = j.L / B;
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
                const uint32_t gs = j.gscale[q];
                for (int i = threadIdx.x; i < B; i += blockDim.x) x[i] = red1(mont(sx[i], gs, P, pneg), P);
            } else {
                for (int i = threadIdx.x; i < B; i += blockDim.x) x[i] = sx[i];
            }
            __syncthreads();
        }
    }
}

// first index f in [0, n) with pos[f] >= key (pos sorted ascending)
__device__ __forceinline__ int64_t fault_lower_bound(const int64_t* pos, int64_t n, int64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (pos[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// fold, CRT, extraction / check / faults, 32 positions per warp
template <int MT>
__global__ void __launch_bounds__(256) k_final(const NttAnyArgs a) {
    constexpr int MR = MT ? MT : 16;
    const int lane = threadIdx.x & 31;
    const uint32_t P1 = prime(0), P2 = prime(1);
    const uint32_t inv = a.crt_inv, invq = a.crt_invq;           // P1^-1 mod P2 and its Shoup quotient
    const uint64_t PP = (uint64_t)P1 * P2;
    for (int64_t b = blockIdx.y; b < a.jobs.njobs; b += gridDim.y) {
        const NJob j = job_of(a.jobs, b);
        if (j.L == 0 || (MT && j.M != MT) || (!MT && a.jobs.table && j.M <= 5)) continue;
        const int Mv = MT ? MT : j.M;
        const bool folded = j.L != j.N;
        for (int64_t base = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31ll; base < j.N;
             base += (int64_t)gridDim.x * blockDim.x) {
            const int64_t n = base + lane;
            const bool valid = n < j.N;
            int64_t f0 = 0, f1 = 0;                                   // this warp's faults
            if (a.fault_pos && j.fault_end > j.fault_begin) {
                f0 = j.fault_begin + fault_lower_bound(a.fault_pos + j.fault_begin, j.fault_end - j.fault_begin, base);
                f1 = j.fault_begin + fault_lower_bound(a.fault_pos + j.fault_begin, j.fault_end - j.fault_begin, base + 32);
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
                    for (int64_t f = f0; f < f1; f++)                    // transient faults (batch)
                        if (a.fault_pos[f] == n && a.fault_stream[f] == m) v ^= (int64_t)(1ull << a.fault_bit[f]);
                }
                rot[jj] = v;
            }
            bool flag = false;
            if (valid) {
                if (j.fuse != NE_FUSE_NONE) {
                    int64_t o[MR];
                    flag = extract_rot<MT>(rot, Mv, j.l, j.fuse == NE_FUSE_EXTRACT_CHECK, o);
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

}  // namespace ntt2

void ntt_any_job_constants(NJob& j) {
    for (int q = 0; q < 2; q++) {
        const uint32_t P = ntt2::prime(q);
        const uint32_t r1 = (uint32_t)((((uint64_t)1) << 32) % P);
        const uint32_t linv = ntt2::powmod((uint32_t)(j.L % P), P - 2, P);
        j.gscale[q] = ntt2::mulmod(ntt2::mulmod(r1, r1, P), linv, P);
    }
}

ne_status ntt_any_run(NttAnyArgs& a, int max_logL, int max_M, int64_t max_units_load, cudaStream_t s) {
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
    ntt2::k_load<<<dim3(gx_for(max_units_load, 256), gy), 256, 0, s>>>(a);
    if ((st = check_launch("ne_cconv_ntt_any: load"))) return st;
    const int gstages = max_logL > ntt2::LOGB ? max_logL - ntt2::LOGB : 0;
    const int64_t half_units = (int64_t)(max_M + 1) * 2 * ((int64_t)1 << (max_logL - 1));
    for (int sidx = 0; sidx < gstages; sidx++) {
        ntt2::k_stage<false><<<dim3(gx_for(half_units, 256), gy), 256, 0, s>>>(a, sidx);
        if ((st = check_launch("ne_cconv_ntt_any: stage"))) return st;
    }
    const int B = max_logL < ntt2::LOGB ? (1 << max_logL) : ntt2::LB;
    const size_t smem = (size_t)B * sizeof(uint32_t);
    static bool attr[64][2];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr[dev][0]) {
        cudaFuncSetAttribute(ntt2::k_block<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ntt2::LB * 4);
        cudaFuncSetAttribute(ntt2::k_block<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ntt2::LB * 4);
        attr[dev][0] = true;
    }
    const int nblk = (1 << max_logL) / B;
    const int fwd_units = (max_M + 1) * 2 * nblk, inv_units = max_M * 2 * nblk;
    ntt2::k_block<false><<<dim3((unsigned)fwd_units, gy), ntt2::BTHREADS, smem, s>>>(a);
    if ((st = check_launch("ne_cconv_ntt_any: forward blocks"))) return st;
    ntt2::k_block<true><<<dim3((unsigned)inv_units, gy), ntt2::BTHREADS, smem, s>>>(a);
    if ((st = check_launch("ne_cconv_ntt_any: inverse blocks"))) return st;
    for (int sidx = 0; sidx < gstages; sidx++) {
        ntt2::k_stage<true><<<dim3(gx_for(half_units, 256), gy), 256, 0, s>>>(a, sidx);
        if ((st = check_launch("ne_cconv_ntt_any: stage"))) return st;
    }
    const int64_t maxN = (int64_t)1 << max_logL;
    const unsigned fx = gx_for(maxN, 256);
    if (a.jobs.table) {
        // a table may mix M: one specialised launch per M (each skips the other jobs)
        ntt2::k_final<3><<<dim3(fx, gy), 256, 0, s>>>(a);
        ntt2::k_final<4><<<dim3(fx, gy), 256, 0, s>>>(a);
        ntt2::k_final<5><<<dim3(fx, gy), 256, 0, s>>>(a);
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
                                      int32_t fuse, int32_t r, int32_t plain, int32_t* status, void* workspace,
                                      int64_t workspace_bytes, cudaStream_t s) {
    ne_status st = validate_params(p);
    if (st) return st;
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
    j.fault_begin = j.fault_end = 0;
    ntt_any_job_constants(j);
    a.jobs.table = nullptr;
    a.jobs.njobs = batch;
    a.jobs.c_stride = (int64_t)p.M * N;
    a.jobs.g_stride = N;
    a.jobs.out_stride = (int64_t)p.M * N;
    a.jobs.flag_stride = (N + 31) / 32;
    a.jobs.ws_stride = (int64_t)(p.M + 1) * 2 * j.L;
    a.c = c;
    a.g = g;
    a.out = out;
    a.flags = fuse == NE_FUSE_EXTRACT_CHECK ? flags : nullptr;
    a.nflag = fuse == NE_FUSE_EXTRACT_CHECK ? nf : nullptr;
    a.flags_atomic = 0;
    a.status = status;
    a.ws = static_cast<uint32_t*>(workspace);
    a.fault_pos = nullptr;
    a.fault_stream = nullptr;
    a.fault_bit = nullptr;
    return ntt_any_run(a, lg, p.M, (int64_t)(p.M + 1) * j.L, s);
}
