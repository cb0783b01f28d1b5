// Disentanglement (Eq. 17-20), the reliability check (Eq. 24), fail-stop
// recovery (Prop. 3), transient-fault injection and the ABFT check/recovery
// (Eq. 6, Sec. II-A).  HBM-bound streaming kernels.
//
// Work split: a warp owns a segment of 32*VEC consecutive positions of one
// group (VEC = 2 with 16-byte loads when possible), so each segment maps to
// whole uint32 words of the flag bitmap and the flags are assembled with
// warp shuffles, not atomics.
#include "ne_bulk.cuh"
#include "ne_common.cuh"
#include "ne_extract.cuh"
#include "ne_flags.cuh"

namespace {

using namespace ne;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// U segments per warp and iteration: all their loads are issued before any
// arithmetic, so a warp keeps U * M * 32 * VEC words in flight.
template <int MT, int VEC, int U, bool WRITE_D, bool CHECK, int TH = kThreads>
__global__ void __launch_bounds__(TH) k_extract(const int64_t* __restrict__ delta, int64_t* __restrict__ dhat,
                                                      int M, int l, int r, int64_t batch, int64_t n,
                                                      uint32_t* __restrict__ flags, unsigned long long* nflag) {
    constexpr int MR = MT ? MT : 32;
    const int Mv = MT ? MT : M;
    const int lane = threadIdx.x & 31;
    const int64_t seg_len = 32 * VEC;
    const int64_t nseg = (n + seg_len - 1) / seg_len;
    const int64_t wpr = (n + 31) / 32;
    for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
        const int64_t* db = delta + b * Mv * n;
        int64_t* ob = dhat + b * Mv * n;
        uint32_t* fb = flags ? flags + b * wpr : nullptr;
        for (int64_t sp = (int64_t)blockIdx.x * (TH / 32) + (threadIdx.x >> 5); sp * U < nseg;
             sp += (int64_t)gridDim.x * (TH / 32)) {
            int64_t rot[U][VEC][MR];
            // rotate while loading: register index j is static, address is not
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t i = (sp * U + u) * seg_len + lane * VEC;
                if (i >= n) continue;
#pragma unroll
                for (int j = 0; j < MR; j++) {
                    if (!MT && j >= Mv) break;
                    if (j == 0 && !CHECK) continue;
                    int m = r + j;
                    if (m >= Mv) m -= Mv;
                    const int64_t* src = db + (int64_t)m * n + i;
                    if constexpr (VEC == 2) {
                        longlong2 v = __ldcs(reinterpret_cast<const longlong2*>(src));
                        rot[u][0][j] = v.x;
                        rot[u][1][j] = v.y;
                    } else {
                        rot[u][0][j] = __ldcs(src);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const int64_t seg = sp * U + u;
                if (seg >= nseg) break;                    // warp-uniform
                const int64_t i = seg * seg_len + lane * VEC;
                uint32_t f = 0;
                if (i < n) {
#pragma unroll
                    for (int v = 0; v < VEC; v++) {
                        int64_t out[MR];
                        if (extract_rot<MT>(rot[u][v], Mv, l, CHECK, out)) f |= 1u << v;
                        if constexpr (WRITE_D) {
#pragma unroll
                            for (int j = 0; j < MR; j++) {
                                if (!MT && j >= Mv) break;
                                rot[u][v][j] = out[j];
                            }
                        }
                    }
                    if constexpr (WRITE_D) {
#pragma unroll
                        for (int j = 0; j < MR; j++) {
                            if (!MT && j >= Mv) break;
                            int m = r + j;
                            if (m >= Mv) m -= Mv;
                            int64_t* dst = ob + (int64_t)m * n + i;
                            if constexpr (VEC == 2)
                                __stcs(reinterpret_cast<longlong2*>(dst), make_longlong2(rot[u][0][j], rot[u][1][j]));
                            else __stcs(dst, rot[u][0][j]);
                        }
                    }
                }
                if constexpr (CHECK) emit_flags<VEC>(f, lane, seg, wpr, fb, nflag);
            }
        }
    }
}

// ---- the read-only check with the reads staged in shared memory ----------------
//
// A unit is PER x TH consecutive positions of one group (all M streams).  Each
// block of a persistent launch walks the units gridDim.x apart through a ring
// of S shared-memory stages: one thread issues the M bulk copies of a unit
// (cp.async.bulk completing on the stage's mbarrier) S units ahead, so the
// block keeps them in flight however long the check of the current one takes.
// A warp checks 32 PER consecutive positions of a unit, a lane PER / 2 pairs
// of them, each pair of a stream read as one 16-byte shared-memory load.
// Requires n even and delta 16-byte aligned (every copy then starts and ends
// on 16 bytes).
constexpr uint32_t CK_WAIT_LIMIT = 1u << 22;
// polls of each block's first wait (ne_check_set_wait_limit; every other wait,
// the drain included, keeps CK_WAIT_LIMIT)
uint32_t g_first_wait_limit = CK_WAIT_LIMIT;

// TH threads, PER positions per thread and unit (2 or 4), S stages
template <int MT, int LT, int TH, int PER, int S>
__global__ void __launch_bounds__(TH, 1) k_check_staged(const int64_t* __restrict__ delta, int l, int r,
                                                        int64_t batch, int64_t n, uint32_t* __restrict__ flags,
                                                        unsigned long long* nflag, int32_t* status,
                                                        uint32_t first_limit) {
    constexpr int CK_POS = PER * TH;
    constexpr int WPOS = 32 * PER;                      // positions of a warp
    extern __shared__ __align__(128) int64_t ring[];   // [S][MT][CK_POS]
    __shared__ uint64_t full[S];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t upg = (n + CK_POS - 1) / CK_POS;      // units per group
    const int64_t nunits = batch * upg;
    const int64_t wpr = (n + 31) / 32;
    const int lv = LT ? LT : l;
    // unit u = (group b, chunk c); the walk adds gridDim.x units per step
    const int64_t sb = gridDim.x / upg, sc = gridDim.x % upg;
    auto next = [&](int64_t& b, int64_t& c) {
        b += sb;
        c += sc;
        if (c >= upg) { c -= upg; b++; }
    };
    auto issue = [&](int64_t b, int64_t c, int s) {
        const int64_t p0 = c * CK_POS;
        const int64_t len = n - p0 < CK_POS ? n - p0 : CK_POS;
        const uint32_t bytes = (uint32_t)len * 8;
        mbar_arrive_expect(&full[s], bytes * MT);
#pragma unroll
        for (int m = 0; m < MT; m++)
            bulk_copy_g2s(ring + (s * MT + m) * CK_POS, delta + (b * MT + m) * n + p0, bytes, &full[s]);
    };
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < S; s++) mbar_init(&full[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    int64_t b = blockIdx.x / upg, c = blockIdx.x % upg;
    // the issuing thread's walk runs S units ahead
    int64_t iu = blockIdx.x, ib = b, ic = c;
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < S; s++) {
            if (iu < nunits) issue(ib, ic, s);
            iu += gridDim.x;
            next(ib, ic);
        }
    }
    int it = 0;
    for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x, it++, next(b, c)) {
        const int s = it % S;
        const bool ok = mbar_wait(&full[s], (uint32_t)(it / S) & 1u, it == 0 ? first_limit : CK_WAIT_LIMIT);
        const int64_t p0 = c * CK_POS;
        const int64_t* st = ring + s * MT * CK_POS;
#pragma unroll
        for (int k = 0; k < PER / 2; k++) {
            const int q = warp * WPOS + k * 64 + lane * 2;   // position within the unit
            uint32_t f = 0;
            if (p0 + q < n) {
                if (ok) {
                    int64_t rot[2][MT];
#pragma unroll
                    for (int j = 0; j < MT; j++) {
                        int m = r + j;
                        if (m >= MT) m -= MT;
                        const longlong2 v = *reinterpret_cast<const longlong2*>(st + m * CK_POS + q);
                        rot[0][j] = v.x;
                        rot[1][j] = v.y;
                    }
#pragma unroll
                    for (int v = 0; v < 2; v++) {
                        int64_t out[MT];
                        if (extract_rot<MT>(rot[v], MT, lv, true, out)) f |= 1u << v;
                    }
                } else {
                    f = 3u;                             // not checked: reported as flagged
                }
            }
            emit_flags<2>(f, lane, (p0 + warp * WPOS + k * 64) / 64, wpr, flags ? flags + b * wpr : nullptr, nflag);
        }
        if (!__syncthreads_and(ok)) {
            // a copy did not arrive in time: report the timeout, report every
            // position of every later unit of this block flagged (none of them
            // is checked), wait (bounded) for the copies still in flight into
            // this block's stages, and leave
            if (tid == 0 && status) atomicExch(status, (int32_t)NE_ETIMEOUT);
            int64_t rb = b, rc = c;
            next(rb, rc);
            for (int64_t v = u + gridDim.x; v < nunits; v += gridDim.x, next(rb, rc)) {
#pragma unroll
                for (int k = 0; k < PER / 2; k++) {
                    const int64_t q = rc * CK_POS + warp * WPOS + k * 64 + lane * 2;
                    emit_flags<2>(q < n ? 3u : 0u, lane, (rc * CK_POS + warp * WPOS + k * 64) / 64, wpr,
                                  flags ? flags + rb * wpr : nullptr, nflag);
                }
            }
            if (tid == 0) {
                for (int k = 0; k < S; k++) {
                    const int jt = it + k;
                    if (u + (int64_t)k * gridDim.x < nunits)
                        mbar_wait(&full[jt % S], (uint32_t)(jt / S) & 1u, CK_WAIT_LIMIT);
                }
            }
            __syncthreads();
            return;
        }
        if (tid == 0) {
            if (iu < nunits) {
                fence_async_shared();
                issue(ib, ic, s);
            }
            iu += gridDim.x;
            next(ib, ic);
        }
    }
}

template <int MT, int LT, int TH, int PER, int S>
void launch_check_staged_v(const int64_t* delta, int l, int r, int64_t batch, int64_t n, uint32_t* flags,
                           unsigned long long* nflag, int32_t* status, cudaStream_t s) {
    static int per_sm = -1;                              // resident blocks per SM (once per process)
    constexpr int smem = S * MT * PER * TH * 8;
    auto kern = k_check_staged<MT, LT, TH, PER, S>;
    if (per_sm < 0) {
        // the ring plus the static barriers pass the 48 KB default
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, TH, smem) != cudaSuccess || b < 1) b = 1;
        per_sm = b;
    }
    const int64_t nunits = batch * ((n + PER * TH - 1) / (PER * TH));
    int64_t grid = (int64_t)sm_count() * per_sm;
    if (grid > nunits) grid = nunits;
    kern<<<(unsigned)grid, TH, smem, s>>>(delta, l, r, batch, n, flags, nflag, status, g_first_wait_limit);
}

// 256 threads of 4 positions and 3 stages (2 for M > 4): three blocks per SM
// for M = 3.  Measured on the check of 4096 x 3 x 1024 words against 2 x 2,
// 4 x 4 and 2 x 4 stages and 128 / 512-thread blocks: fewer resident warps
// lost up to 15 % at the smallest l (the 128-bit arithmetic then bounds it)
template <int MT, int LT>
void launch_check_staged_lt(const int64_t* delta, int l, int r, int64_t batch, int64_t n, uint32_t* flags,
                            unsigned long long* nflag, int32_t* status, cudaStream_t s) {
    launch_check_staged_v<MT, LT, 256, 4, (MT <= 4 ? 3 : 2)>(delta, l, r, batch, n, flags, nflag, status, s);
}

// true when the staged kernel took the launch
bool launch_check_staged(const int64_t* delta, int M, int l, int r, int64_t batch, int64_t n, uint32_t* flags,
                         unsigned long long* nflag, int32_t* status, cudaStream_t s) {
    if (n % 2 != 0 || !aligned(delta, 16)) return false;
    // l = 16 (the byte-aligned shift) is compiled in for M <= 4, the M for
    // which (M - 1) l fits a 64-bit word
    switch (M) {
        case 3:
            if (l == 16) launch_check_staged_lt<3, 16>(delta, l, r, batch, n, flags, nflag, status, s);
            else launch_check_staged_lt<3, 0>(delta, l, r, batch, n, flags, nflag, status, s);
            return true;
        case 4:
            if (l == 16) launch_check_staged_lt<4, 16>(delta, l, r, batch, n, flags, nflag, status, s);
            else launch_check_staged_lt<4, 0>(delta, l, r, batch, n, flags, nflag, status, s);
            return true;
        case 5: launch_check_staged_lt<5, 0>(delta, l, r, batch, n, flags, nflag, status, s); return true;
        case 6: launch_check_staged_lt<6, 0>(delta, l, r, batch, n, flags, nflag, status, s); return true;
        case 8: launch_check_staged_lt<8, 0>(delta, l, r, batch, n, flags, nflag, status, s); return true;
        default: return false;
    }
}

dim3 grid_segments(int64_t batch, int64_t nseg, int threads = kThreads) {
    int64_t gy = batch < 65535 ? batch : 65535;
    int64_t want = (int64_t)wave_blocks(threads, 4);
    int64_t gx = (nseg + threads / 32 - 1) / (threads / 32);
    int64_t cap = want / gy;
    if (cap < 1) cap = 1;
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    return dim3((unsigned)gx, (unsigned)gy, 1);
}

template <int MT, bool WRITE_D, bool CHECK>
void launch_extract_vec(const int64_t* delta, int64_t* dhat, int M, int l, int r, int64_t batch, int64_t n,
                        uint32_t* flags, unsigned long long* nflag, cudaStream_t s) {
    constexpr int U = MT ? 2 : 1;      // the generic-M kernel keeps one segment (register budget)
    const bool vec2 = (n % 2 == 0) && aligned(delta, 16) && (!WRITE_D || aligned(dhat, 16));
    if constexpr (MT != 0 && !WRITE_D) {
        if (vec2) {
            // the read-only check: four segments per warp in flight (no stores
            // to overlap with), 128-thread blocks
            dim3 g = grid_segments(batch, ((n + 63) / 64 + 3) / 4, 128);
            k_extract<MT, 2, 4, WRITE_D, CHECK, 128><<<g, 128, 0, s>>>(delta, dhat, M, l, r, batch, n, flags, nflag);
            return;
        }
    }
    if (vec2) {
        dim3 g = grid_segments(batch, ((n + 63) / 64 + U - 1) / U);
        k_extract<MT, 2, U, WRITE_D, CHECK><<<g, kThreads, 0, s>>>(delta, dhat, M, l, r, batch, n, flags, nflag);
    } else {
        dim3 g = grid_segments(batch, ((n + 31) / 32 + U - 1) / U);
        k_extract<MT, 1, U, WRITE_D, CHECK><<<g, kThreads, 0, s>>>(delta, dhat, M, l, r, batch, n, flags, nflag);
    }
}

template <bool WRITE_D, bool CHECK>
void launch_extract(const int64_t* delta, int64_t* dhat, int M, int l, int r, int64_t batch, int64_t n,
                    uint32_t* flags, unsigned long long* nflag, cudaStream_t s) {
    switch (M) {
        case 3: launch_extract_vec<3, WRITE_D, CHECK>(delta, dhat, M, l, r, batch, n, flags, nflag, s); break;
        case 4: launch_extract_vec<4, WRITE_D, CHECK>(delta, dhat, M, l, r, batch, n, flags, nflag, s); break;
        case 5: launch_extract_vec<5, WRITE_D, CHECK>(delta, dhat, M, l, r, batch, n, flags, nflag, s); break;
        case 6: launch_extract_vec<6, WRITE_D, CHECK>(delta, dhat, M, l, r, batch, n, flags, nflag, s); break;
        case 8: launch_extract_vec<8, WRITE_D, CHECK>(delta, dhat, M, l, r, batch, n, flags, nflag, s); break;
        default: launch_extract_vec<0, WRITE_D, CHECK>(delta, dhat, M, l, r, batch, n, flags, nflag, s); break;
    }
}

ne_status common_args(const ne_params& p, int64_t batch, int64_t n, int32_t r, const char* who) {
    ne_status st = validate_params(p);
    if (st) return st;
    if (batch < 0 || n < 0) return fail(NE_EINVAL, "%s: batch=%lld n=%lld", who, (long long)batch, (long long)n);
    if (r < 0 || r >= p.M) return fail(NE_EINVAL, "%s: r=%d not in [0, M)", who, r);
    return NE_OK;
}

// ---- fault injection ---------------------------------------------------------

__global__ void k_inject(int64_t* delta, int P, int64_t batch, int64_t n, const int64_t* group, const int64_t* pos,
                         const int64_t* stream, const int64_t* bit, int64_t count, int32_t* status) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < count; f += (int64_t)gridDim.x * blockDim.x) {
        int64_t g = group[f], i = pos[f], j = stream[f], b = bit[f];
        if (g < 0 || g >= batch || i < 0 || i >= n || j < 0 || j >= P || b < 0 || b > 63) {
            if (status) atomicExch(status, (int32_t)NE_EINVAL);
            continue;
        }
        atomicXor(reinterpret_cast<unsigned long long*>(delta + (g * P + j) * n + i), 1ull << b);
    }
}

// the fault hook of the unfused operations: entry f XORs bit (bit[f] mod 64)
// into delta_{stream[f]} at flat position pos[f] = group * n + i; streams
// outside [0, M), streams in skip_mask (never computed) and positions outside
// the array hit nothing
__global__ void k_apply_faults(int64_t* delta, int M, int64_t batch, int64_t n, ne_faults F, uint32_t skip_mask) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < F.count; f += (int64_t)gridDim.x * blockDim.x) {
        const int64_t key = F.pos[f];
        const int m = F.stream[f];
        if (key < 0 || key >= batch * n || m < 0 || m >= M || ((skip_mask >> m) & 1u)) continue;
        const int64_t g = key / n, i = key - g * n;
        atomicXor(reinterpret_cast<unsigned long long*>(delta + (g * M + m) * n + i), 1ull << (F.bit[f] & 63));
    }
}

// ---- checksum ABFT check / recovery -----------------------------------------------

__global__ void __launch_bounds__(kThreads) k_abft_check(const int64_t* __restrict__ d, int M, int64_t batch, int64_t n,
                                                         uint32_t* __restrict__ flags, unsigned long long* nflag) {
    const int lane = threadIdx.x & 31;
    const int64_t nseg = (n + 31) / 32;
    const int64_t wpr = nseg;
    for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
        const int64_t* db = d + b * (M + 1) * n;
        uint32_t* fb = flags ? flags + b * wpr : nullptr;
        for (int64_t seg = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); seg < nseg;
             seg += (int64_t)gridDim.x * kWarps) {
            const int64_t i = seg * 32 + lane;
            uint32_t f = 0;
            if (i < n) {
                i128 sum = 0;
                for (int m = 0; m < M; m++) sum += (i128)__ldcs(db + (int64_t)m * n + i);
                f = (sum != (i128)__ldcs(db + (int64_t)M * n + i));
            }
            emit_flags<1>(f, lane, seg, wpr, fb, nflag);
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_abft_recover(int64_t* d, int M, int64_t batch, int64_t n, int j) {
    for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
        int64_t* db = d + b * (M + 1) * n;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            uint64_t v = (uint64_t)db[(int64_t)M * n + i];
            for (int m = 0; m < M; m++)
                if (m != j) v -= (uint64_t)db[(int64_t)m * n + i];
            db[(int64_t)j * n + i] = (int64_t)v;
        }
    }
}

}  // namespace

namespace ne {

// Internal launches for the operations' unfused epilogues (arguments checked
// by the caller).  The extraction reads every stream of a position before it
// writes any, and no position twice, so d_hat may be delta itself.
ne_status faults_launch(int64_t* delta, int M, int64_t batch, int64_t n, const ne_faults& F, uint32_t skip_mask,
                        cudaStream_t s) {
    if (F.count <= 0) return NE_OK;
    int blocks = (int)((F.count + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_apply_faults<<<blocks, 256, 0, s>>>(delta, M, batch, n, F, skip_mask);
    return check_launch("fault hook");
}

ne_status extract_launch(const ne_params& p, const int64_t* delta, int64_t* d_hat, int64_t batch, int64_t n, int r,
                         bool check, uint32_t* flags, unsigned long long* nflag, cudaStream_t s) {
    if (batch == 0 || n == 0) return NE_OK;
    if (check) launch_extract<true, true>(delta, d_hat, p.M, p.l, r, batch, n, flags, nflag, s);
    else launch_extract<true, false>(delta, d_hat, p.M, p.l, r, batch, n, nullptr, nullptr, s);
    return check_launch("extraction");
}

}  // namespace ne

extern "C" ne_status ne_extract(ne_params p, const int64_t* delta, int64_t* d_hat, int64_t batch, int64_t n,
                                int32_t r, uint32_t* flags, uint64_t* nflag, cudaStream_t s) {
    ne_status st = common_args(p, batch, n, r, "ne_extract");
    if (st) return st;
    if (!delta || !d_hat) return fail(NE_EINVAL, "ne_extract: null pointer");
    unsigned long long* nf = reinterpret_cast<unsigned long long*>(nflag);
    if (nf && cudaMemsetAsync(nf, 0, sizeof(*nf), s) != cudaSuccess) return check_launch("ne_extract: reset count");
    if (batch == 0 || n == 0) return NE_OK;
    if (flags || nflag) launch_extract<true, true>(delta, d_hat, p.M, p.l, r, batch, n, flags, nf, s);
    else launch_extract<true, false>(delta, d_hat, p.M, p.l, r, batch, n, nullptr, nullptr, s);
    return check_launch("ne_extract");
}

extern "C" ne_status ne_check(ne_params p, const int64_t* delta, int64_t batch, int64_t n, int32_t r,
                              uint32_t* flags, uint64_t* nflag, int32_t* status, cudaStream_t s) {
    ne_status st = common_args(p, batch, n, r, "ne_check");
    if (st) return st;
    if (!delta || (!flags && !nflag)) return fail(NE_EINVAL, "ne_check: null pointer");
    unsigned long long* nf = reinterpret_cast<unsigned long long*>(nflag);
    if (nf && cudaMemsetAsync(nf, 0, sizeof(*nf), s) != cudaSuccess) return check_launch("ne_check: reset count");
    if (batch == 0 || n == 0) return NE_OK;
    if (!launch_check_staged(delta, p.M, p.l, r, batch, n, flags, nf, status, s))
        launch_extract<false, true>(delta, nullptr, p.M, p.l, r, batch, n, flags, nf, s);
    return check_launch("ne_check");
}

extern "C" ne_status ne_check_set_wait_limit(uint32_t polls) {
    if (polls > CK_WAIT_LIMIT) return fail(NE_EINVAL, "ne_check_set_wait_limit: %u polls exceed %u", polls, CK_WAIT_LIMIT);
    g_first_wait_limit = polls;
    return NE_OK;
}

extern "C" ne_status ne_recover(ne_params p, const int64_t* delta, int64_t* d_hat, int64_t batch, int64_t n,
                                int32_t r_lost, cudaStream_t s) {
    ne_status st = common_args(p, batch, n, r_lost, "ne_recover");
    if (st) return st;
    if (!delta || !d_hat) return fail(NE_EINVAL, "ne_recover: null pointer");
    if (batch == 0 || n == 0) return NE_OK;
    launch_extract<true, false>(delta, d_hat, p.M, p.l, r_lost, batch, n, nullptr, nullptr, s);
    return check_launch("ne_recover");
}

extern "C" ne_status ne_inject(int64_t* delta, int32_t P, int64_t batch, int64_t n, const int64_t* group,
                               const int64_t* pos, const int64_t* stream, const int64_t* bit, int64_t count,
                               int32_t* status, cudaStream_t s) {
    if (P < 1 || batch < 0 || n < 0 || count < 0) return fail(NE_EINVAL, "ne_inject: bad sizes");
    if (count == 0) return NE_OK;
    if (!delta || !group || !pos || !stream || !bit) return fail(NE_EINVAL, "ne_inject: null pointer");
    int blocks = (int)((count + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_inject<<<blocks, 256, 0, s>>>(delta, P, batch, n, group, pos, stream, bit, count, status);
    return check_launch("ne_inject");
}

extern "C" ne_status ne_abft_check(int32_t M, const int64_t* d, int64_t batch, int64_t n, uint32_t* flags,
                                   uint64_t* nflag, cudaStream_t s) {
    if (M < 1 || M > 64 || batch < 0 || n < 0) return fail(NE_EINVAL, "ne_abft_check: bad sizes");
    if (!d || (!flags && !nflag)) return fail(NE_EINVAL, "ne_abft_check: null pointer");
    unsigned long long* nf = reinterpret_cast<unsigned long long*>(nflag);
    if (nf && cudaMemsetAsync(nf, 0, sizeof(*nf), s) != cudaSuccess) return check_launch("ne_abft_check: reset");
    if (batch == 0 || n == 0) return NE_OK;
    k_abft_check<<<grid_segments(batch, (n + 31) / 32), kThreads, 0, s>>>(d, M, batch, n, flags, nf);
    return check_launch("ne_abft_check");
}

extern "C" ne_status ne_abft_recover(int32_t M, int64_t* d, int64_t batch, int64_t n, int32_t j, cudaStream_t s) {
    if (M < 1 || M > 64 || batch < 0 || n < 0 || j < 0 || j >= M) return fail(NE_EINVAL, "ne_abft_recover: bad args");
    if (!d) return fail(NE_EINVAL, "ne_abft_recover: null pointer");
    if (batch == 0 || n == 0) return NE_OK;
    int64_t gy = batch < 65535 ? batch : 65535;
    int64_t gx = (n + 255) / 256;
    int64_t cap = wave_blocks(256, 4) / gy;
    if (cap < 1) cap = 1;
    if (gx > cap) gx = cap;
    k_abft_recover<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(d, M, batch, n, j);
    return check_launch("ne_abft_recover");
}
