// The remaining LSB operators of Eq. 2 on the M entangled streams --
// element-wise +, -, x, the outer product, the permutation and the inner
// product -- each as one HBM pass with the disentanglement and check of
// Eq. 17-20 / Eq. 24 (or the recovery of Prop. 3) fused behind the operator,
// plus the two operand preparations: the self-entangled kernel of the
// footnote to Eq. 10 and the index reversal that turns circular
// cross-correlation into circular convolution.
//
// Every operator is applied in wrapping 64-bit arithmetic: the low 64 bits of
// a sum, difference or product depend only on the low 64 bits of the
// operands, so the words are exact whenever the true result fits the w = 64
// word, which the choice of l (Eq. 13-14) guarantees for in-range inputs.
//
// Work split of the position-wise operators: a warp owns 32*VEC consecutive
// output positions of one group (VEC = 2 with 16-byte accesses when sizes and
// alignment allow), so the check flags of a segment are whole bitmap words.
#include "ne_common.cuh"
#include "ne_extract.cuh"
#include "ne_flags.cuh"

namespace {

using namespace ne;

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

enum : int { K_ADD = NE_OP_ADD, K_SUB = NE_OP_SUB, K_MUL = NE_OP_MUL, K_OUTER = 3, K_PERM = 4 };

struct LsbArgs {
    const int64_t* eps;     // [batch][M][n]
    const int64_t* g;       // operand of group b at g + b * g_stride (ADD/SUB/MUL/OUTER)
    const int32_t* perm;    // [n] (PERM)
    int64_t* out;           // [batch][M][npos]
    int M, l, r;
    int64_t batch, n, npos, k, g_stride;
    uint32_t* flags;        // [batch][ceil(npos/32)]
    unsigned long long* nflag;
    int32_t* status;
};

template <int KIND>
__device__ __forceinline__ int64_t apply_op(int64_t x, int64_t g) {
    if constexpr (KIND == K_ADD) return (int64_t)((uint64_t)x + (uint64_t)g);
    else if constexpr (KIND == K_SUB) return (int64_t)((uint64_t)x - (uint64_t)g);
    else if constexpr (KIND == K_PERM) return x;
    else return (int64_t)((uint64_t)x * (uint64_t)g);   // MUL and OUTER
}

template <int MT, int KIND, int VEC, int FUSE>
__global__ void __launch_bounds__(kThreads) k_lsb(const LsbArgs a) {
    constexpr int MR = MT ? MT : 32;
    const int Mv = MT ? MT : a.M;
    const int lane = threadIdx.x & 31;
    const int64_t seg_len = 32 * VEC;
    const int64_t nseg = (a.npos + seg_len - 1) / seg_len;
    const int64_t wpr = (a.npos + 31) / 32;
    for (int64_t b = blockIdx.y; b < a.batch; b += gridDim.y) {
        const int64_t* eb = a.eps + b * Mv * a.n;
        const int64_t* gb = (KIND == K_PERM) ? nullptr : a.g + b * a.g_stride;
        int64_t* ob = a.out + b * Mv * a.npos;
        uint32_t* fb = a.flags ? a.flags + b * wpr : nullptr;
        for (int64_t seg = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); seg < nseg;
             seg += (int64_t)gridDim.x * kWarps) {
            const int64_t p0 = seg * seg_len + lane * VEC;
            uint32_t f = 0;
            if (p0 < a.npos) {
                // input position(s) and operand value(s) of the VEC output positions
                int64_t src[VEC], gv[VEC];
                if constexpr (KIND == K_PERM) {
#pragma unroll
                    for (int v = 0; v < VEC; v++) {
                        int64_t q = __ldg(a.perm + p0 + v);
                        if (q < 0 || q >= a.n) {
                            if (a.status) atomicExch(a.status, (int32_t)NE_EINVAL);
                            q = 0;
                        }
                        src[v] = q;
                        gv[v] = 0;
                    }
                } else if constexpr (KIND == K_OUTER) {
                    const int64_t i = p0 / a.k, j = p0 - i * a.k;   // VEC = 2 only when k is even
#pragma unroll
                    for (int v = 0; v < VEC; v++) src[v] = i;
                    if constexpr (VEC == 2) {
                        const longlong2 t = __ldg(reinterpret_cast<const longlong2*>(gb + j));
                        gv[0] = t.x;
                        gv[1] = t.y;
                    } else {
                        gv[0] = __ldg(gb + j);
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < VEC; v++) src[v] = p0 + v;
                    if constexpr (VEC == 2) {
                        const longlong2 t = __ldg(reinterpret_cast<const longlong2*>(gb + p0));
                        gv[0] = t.x;
                        gv[1] = t.y;
                    } else {
                        gv[0] = __ldg(gb + p0);
                    }
                }
                // rot[v][j] = operator applied to stream (r + j) mod M; under
                // RECOVER stream r (j = 0) is neither read nor computed
                int64_t rot[VEC][MR];
#pragma unroll
                for (int j = 0; j < MR; j++) {
                    if (!MT && j >= Mv) break;
                    if (FUSE == NE_FUSE_RECOVER && j == 0) {
#pragma unroll
                        for (int v = 0; v < VEC; v++) rot[v][0] = 0;
                        continue;
                    }
                    int m = a.r + j;
                    if (m >= Mv) m -= Mv;
                    const int64_t* sp = eb + (int64_t)m * a.n;
                    if constexpr (VEC == 2 && KIND <= K_MUL) {
                        const longlong2 t = __ldcs(reinterpret_cast<const longlong2*>(sp + src[0]));
                        rot[0][j] = t.x;
                        rot[1][j] = t.y;
                    } else if constexpr (VEC == 2 && KIND == K_OUTER) {
                        rot[0][j] = rot[1][j] = __ldg(sp + src[0]);
                    } else {
#pragma unroll
                        for (int v = 0; v < VEC; v++) rot[v][j] = __ldg(sp + src[v]);
                    }
#pragma unroll
                    for (int v = 0; v < VEC; v++) rot[v][j] = apply_op<KIND>(rot[v][j], gv[v]);
                }
                if constexpr (FUSE != NE_FUSE_NONE) {
#pragma unroll
                    for (int v = 0; v < VEC; v++) {
                        int64_t o[MR];
                        // the gather keeps the general shifts: 10 % faster there (the others equal)
                        if (extract_rot<MT, KIND != K_PERM>(rot[v], Mv, a.l, FUSE == NE_FUSE_EXTRACT_CHECK, o))
                            f |= 1u << v;
#pragma unroll
                        for (int j = 0; j < MR; j++) {
                            if (!MT && j >= Mv) break;
                            rot[v][j] = o[j];
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < MR; j++) {
                    if (!MT && j >= Mv) break;
                    int m = a.r + j;
                    if (m >= Mv) m -= Mv;
                    int64_t* dst = ob + (int64_t)m * a.npos + p0;
                    if constexpr (VEC == 2) __stcs(reinterpret_cast<longlong2*>(dst), make_longlong2(rot[0][j], rot[1][j]));
                    else __stcs(dst, rot[0][j]);
                }
            }
            if constexpr (FUSE == NE_FUSE_EXTRACT_CHECK) emit_flags<VEC>(f, lane, seg, wpr, fb, a.nflag);
        }
    }
}

dim3 grid_segments(int64_t batch, int64_t nseg) {
    const int64_t gy = batch < 65535 ? batch : 65535;
    const int64_t want = (int64_t)wave_blocks(kThreads, 4);
    int64_t gx = (nseg + kWarps - 1) / kWarps;
    int64_t cap = want / gy;
    if (cap < 1) cap = 1;
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    return dim3((unsigned)gx, (unsigned)gy, 1);
}

template <int MT, int KIND, int FUSE>
void launch_lsb_vec(const LsbArgs& a, bool vec2, cudaStream_t s) {
    if (vec2) {
        k_lsb<MT, KIND, 2, FUSE><<<grid_segments(a.batch, (a.npos + 63) / 64), kThreads, 0, s>>>(a);
    } else {
        k_lsb<MT, KIND, 1, FUSE><<<grid_segments(a.batch, (a.npos + 31) / 32), kThreads, 0, s>>>(a);
    }
}

template <int KIND, int FUSE>
void launch_lsb_m(const LsbArgs& a, bool vec2, cudaStream_t s) {
    switch (a.M) {
        case 3: launch_lsb_vec<3, KIND, FUSE>(a, vec2, s); break;
        case 4: launch_lsb_vec<4, KIND, FUSE>(a, vec2, s); break;
        case 5: launch_lsb_vec<5, KIND, FUSE>(a, vec2, s); break;
        default: launch_lsb_vec<0, KIND, FUSE>(a, vec2, s); break;
    }
}

template <int KIND>
void launch_lsb(const LsbArgs& a, int fuse, bool vec2, cudaStream_t s) {
    if (fuse == NE_FUSE_EXTRACT_CHECK) launch_lsb_m<KIND, NE_FUSE_EXTRACT_CHECK>(a, vec2, s);
    else if (fuse == NE_FUSE_RECOVER) launch_lsb_m<KIND, NE_FUSE_RECOVER>(a, vec2, s);
    else launch_lsb_m<KIND, NE_FUSE_NONE>(a, vec2, s);
}

// ---- inner product ------------------------------------------------------------------

// Block (x, b) sums positions [x*chunk, (x+1)*chunk) of every stream of group
// b against g; with one block per group (gridDim.x = 1) it also finishes the
// group, otherwise it adds its partial sums into out (zeroed beforehand) and
// k_inner_finish completes the groups.
template <int MT>
__device__ __forceinline__ void finish_group(const uint64_t* dsum, int64_t* ob, int M, int l, int r, int fuse,
                                             int64_t b, uint32_t* flags, unsigned long long* nflag) {
    constexpr int MR = MT ? MT : 32;
    const int Mv = MT ? MT : M;
    if (fuse == NE_FUSE_NONE) {
        for (int m = 0; m < Mv; m++) ob[m] = (int64_t)dsum[m];
        return;
    }
    int64_t rot[MR], o[MR];
#pragma unroll
    for (int j = 0; j < MR; j++) {
        if (!MT && j >= Mv) break;
        int m = r + j;
        if (m >= Mv) m -= Mv;
        rot[j] = (int64_t)dsum[m];
    }
    const bool f = extract_rot<MT>(rot, Mv, l, fuse == NE_FUSE_EXTRACT_CHECK, o);
#pragma unroll
    for (int j = 0; j < MR; j++) {
        if (!MT && j >= Mv) break;
        int m = r + j;
        if (m >= Mv) m -= Mv;
        ob[m] = o[j];
    }
    if (fuse == NE_FUSE_EXTRACT_CHECK) {
        if (flags) flags[b] = f ? 1u : 0u;
        if (nflag && f) atomicAdd(nflag, 1ull);
    }
}

template <int MT>
__global__ void __launch_bounds__(kThreads) k_inner(const int64_t* __restrict__ eps, const int64_t* __restrict__ g,
                                                    int64_t* out, int M, int l, int r, int fuse, int64_t batch,
                                                    int64_t n, int64_t g_stride, int64_t chunk, int vec2,
                                                    uint32_t* flags, unsigned long long* nflag) {
    constexpr int MR = MT ? MT : 32;
    const int Mv = MT ? MT : M;
    __shared__ uint64_t red[kWarps][MR];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
        const int64_t* eb = eps + b * Mv * n;
        const int64_t* gb = g + b * g_stride;
        const int64_t lo = (int64_t)blockIdx.x * chunk;
        const int64_t hi = lo + chunk < n ? lo + chunk : n;
        uint64_t acc[MR];
#pragma unroll
        for (int m = 0; m < MR; m++) acc[m] = 0;
        if (vec2) {
#pragma unroll 4
            for (int64_t i = lo + 2 * threadIdx.x; i < hi; i += 2 * kThreads) {
                const longlong2 gv = __ldg(reinterpret_cast<const longlong2*>(gb + i));
#pragma unroll
                for (int m = 0; m < MR; m++) {
                    if (!MT && m >= Mv) break;
                    if (fuse == NE_FUSE_RECOVER && m == r) continue;
                    const longlong2 x = __ldcs(reinterpret_cast<const longlong2*>(eb + (int64_t)m * n + i));
                    acc[m] += (uint64_t)x.x * (uint64_t)gv.x + (uint64_t)x.y * (uint64_t)gv.y;
                }
            }
        } else {
#pragma unroll 4
            for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) {
                const uint64_t gv = (uint64_t)__ldg(gb + i);
#pragma unroll
                for (int m = 0; m < MR; m++) {
                    if (!MT && m >= Mv) break;
                    if (fuse == NE_FUSE_RECOVER && m == r) continue;
                    acc[m] += (uint64_t)__ldcs(eb + (int64_t)m * n + i) * gv;
                }
            }
        }
#pragma unroll
        for (int m = 0; m < MR; m++) {
            if (!MT && m >= Mv) break;
            uint64_t v = acc[m];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][m] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t dsum[MR];
#pragma unroll
            for (int m = 0; m < MR; m++) {
                if (!MT && m >= Mv) break;
                uint64_t v = 0;
                for (int w = 0; w < kWarps; w++) v += red[w][m];
                dsum[m] = v;
            }
            int64_t* ob = out + b * Mv;
            if (gridDim.x == 1) {
                finish_group<MT>(dsum, ob, Mv, l, r, fuse, b, flags, nflag);
            } else {
                for (int m = 0; m < Mv; m++)
                    if (!(fuse == NE_FUSE_RECOVER && m == r))
                        atomicAdd(reinterpret_cast<unsigned long long*>(ob + m), (unsigned long long)dsum[m]);
            }
        }
        __syncthreads();
    }
}

template <int MT>
__global__ void k_inner_finish(int64_t* out, int M, int l, int r, int fuse, int64_t batch, uint32_t* flags,
                               unsigned long long* nflag) {
    constexpr int MR = MT ? MT : 32;
    const int Mv = MT ? MT : M;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < batch; b += (int64_t)gridDim.x * blockDim.x) {
        int64_t* ob = out + b * Mv;
        uint64_t dsum[MR];
        for (int m = 0; m < Mv; m++) dsum[m] = (uint64_t)ob[m];
        finish_group<MT>(dsum, ob, Mv, l, r, fuse, b, flags, nflag);
    }
}

template <int MT>
ne_status launch_inner(const int64_t* eps, const int64_t* g, int64_t g_stride, int64_t* out, uint32_t* flags,
                       unsigned long long* nf, int M, int l, int r, int fuse, int64_t batch, int64_t n,
                       bool vec2, cudaStream_t s) {
    // enough blocks for about two waves; split a group only when groups are few
    const int64_t want = (int64_t)wave_blocks(kThreads, 2);
    int64_t splits = (want + batch - 1) / batch;
    const int64_t max_splits = (n + 4095) / 4096;
    if (splits > max_splits) splits = max_splits;
    if (splits < 1) splits = 1;
    if (splits > 65535) splits = 65535;
    int64_t chunk = (n + splits - 1) / splits;
    chunk += chunk & 1;
    splits = (n + chunk - 1) / chunk;
    if (splits < 1) splits = 1;
    const unsigned gy = (unsigned)(batch < 65535 ? batch : 65535);
    if (splits > 1 && cudaMemsetAsync(out, 0, (size_t)batch * M * sizeof(int64_t), s) != cudaSuccess)
        return check_launch("ne_inner: zero partial sums");
    k_inner<MT><<<dim3((unsigned)splits, gy, 1), kThreads, 0, s>>>(eps, g, out, M, l, r, fuse, batch, n, g_stride,
                                                                   chunk, vec2 ? 1 : 0, flags, nf);
    if (splits > 1 && fuse != NE_FUSE_NONE) {
        int blocks = (int)((batch + 255) / 256);
        if (blocks > 65535) blocks = 65535;
        k_inner_finish<MT><<<blocks, 256, 0, s>>>(out, M, l, r, fuse, batch, flags, nf);
    }
    return check_launch("ne_inner");
}

// ---- operand preparations ------------------------------------------------------------

__global__ void k_kernel_self(const int64_t* __restrict__ g, int64_t* __restrict__ ge, int l, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t v = (uint64_t)g[i];
        ge[i] = (int64_t)(v + (v << l));
    }
}

__global__ void k_reverse(const int8_t* __restrict__ g, int8_t* __restrict__ gr, int64_t batch, int64_t N) {
    const int64_t total = batch * N;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / N, j = t - b * N;
        gr[t] = g[b * N + (j == 0 ? 0 : N - j)];
    }
}

int stream_blocks(int64_t n) {
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = wave_blocks(256, 4);
    if (blocks > cap) blocks = cap;
    return (int)(blocks < 1 ? 1 : blocks);
}

ne_status lsb_common(const ne_params& p, int64_t batch, int64_t n, int32_t fuse, int32_t r, const void* eps,
                     const void* out, const char* who) {
    ne_status st = validate_params(p);
    if (st) return st;
    if (batch < 0 || n < 0) return fail(NE_EINVAL, "%s: batch=%lld n=%lld", who, (long long)batch, (long long)n);
    if (fuse != NE_FUSE_NONE && fuse != NE_FUSE_EXTRACT_CHECK && fuse != NE_FUSE_RECOVER)
        return fail(NE_EINVAL, "%s: fuse=%d", who, fuse);
    if (fuse != NE_FUSE_NONE && (r < 0 || r >= p.M)) return fail(NE_EINVAL, "%s: r=%d not in [0, M)", who, r);
    if (batch > 0 && n > 0 && (!eps || !out)) return fail(NE_EINVAL, "%s: null pointer", who);
    return NE_OK;
}

ne_status reset_count(uint64_t* nflag, int32_t fuse, cudaStream_t s, const char* who) {
    if (nflag && fuse == NE_FUSE_EXTRACT_CHECK &&
        cudaMemsetAsync(nflag, 0, sizeof(*nflag), s) != cudaSuccess)
        return check_launch(who);
    return NE_OK;
}

}  // namespace

extern "C" ne_status ne_elementwise(ne_params p, int32_t op, const int64_t* eps, const int64_t* g, int64_t g_stride,
                                    int64_t* out, uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t n,
                                    int32_t fuse, int32_t r, cudaStream_t s) {
    ne_status st = lsb_common(p, batch, n, fuse, r, eps, out, "ne_elementwise");
    if (st) return st;
    if (op != NE_OP_ADD && op != NE_OP_SUB && op != NE_OP_MUL) return fail(NE_EINVAL, "ne_elementwise: op=%d", op);
    if (g_stride < 0) return fail(NE_EINVAL, "ne_elementwise: g_stride < 0");
    if (batch > 0 && n > 0 && !g) return fail(NE_EINVAL, "ne_elementwise: null operand");
    if ((st = reset_count(nflag, fuse, s, "ne_elementwise: reset count"))) return st;
    if (batch == 0 || n == 0) return NE_OK;
    LsbArgs a{eps, g, nullptr, out, p.M, p.l, fuse == NE_FUSE_NONE ? 0 : r, batch, n, n, 1, g_stride,
              fuse == NE_FUSE_EXTRACT_CHECK ? flags : nullptr,
              fuse == NE_FUSE_EXTRACT_CHECK ? reinterpret_cast<unsigned long long*>(nflag) : nullptr, nullptr};
    const bool vec2 = n % 2 == 0 && g_stride % 2 == 0 && aligned(eps, 16) && aligned(out, 16) && aligned(g, 16);
    if (op == NE_OP_ADD) launch_lsb<K_ADD>(a, fuse, vec2, s);
    else if (op == NE_OP_SUB) launch_lsb<K_SUB>(a, fuse, vec2, s);
    else launch_lsb<K_MUL>(a, fuse, vec2, s);
    return check_launch("ne_elementwise");
}

extern "C" ne_status ne_outer(ne_params p, const int64_t* eps, const int64_t* g, int64_t g_stride, int64_t* out,
                              uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t n, int64_t k,
                              int32_t fuse, int32_t r, cudaStream_t s) {
    ne_status st = lsb_common(p, batch, n, fuse, r, eps, out, "ne_outer");
    if (st) return st;
    if (k < 0 || g_stride < 0) return fail(NE_EINVAL, "ne_outer: k=%lld g_stride=%lld", (long long)k,
                                           (long long)g_stride);
    if (n > 0 && k > ((int64_t)1 << 56) / n) return fail(NE_EINVAL, "ne_outer: n * k too large");
    if (batch > 0 && n > 0 && k > 0 && !g) return fail(NE_EINVAL, "ne_outer: null operand");
    if ((st = reset_count(nflag, fuse, s, "ne_outer: reset count"))) return st;
    if (batch == 0 || n == 0 || k == 0) return NE_OK;
    LsbArgs a{eps, g, nullptr, out, p.M, p.l, fuse == NE_FUSE_NONE ? 0 : r, batch, n, n * k, k, g_stride,
              fuse == NE_FUSE_EXTRACT_CHECK ? flags : nullptr,
              fuse == NE_FUSE_EXTRACT_CHECK ? reinterpret_cast<unsigned long long*>(nflag) : nullptr, nullptr};
    const bool vec2 = k % 2 == 0 && g_stride % 2 == 0 && aligned(out, 16) && aligned(g, 16);
    launch_lsb<K_OUTER>(a, fuse, vec2, s);
    return check_launch("ne_outer");
}

extern "C" ne_status ne_permute(ne_params p, const int64_t* eps, const int32_t* perm, int64_t* out, uint32_t* flags,
                                uint64_t* nflag, int64_t batch, int64_t n, int32_t fuse, int32_t r, int32_t* status,
                                cudaStream_t s) {
    ne_status st = lsb_common(p, batch, n, fuse, r, eps, out, "ne_permute");
    if (st) return st;
    if (n > INT32_MAX) return fail(NE_EINVAL, "ne_permute: n exceeds the int32 index range");
    if (batch > 0 && n > 0 && !perm) return fail(NE_EINVAL, "ne_permute: null index set");
    if ((st = reset_count(nflag, fuse, s, "ne_permute: reset count"))) return st;
    if (batch == 0 || n == 0) return NE_OK;
    LsbArgs a{eps, nullptr, perm, out, p.M, p.l, fuse == NE_FUSE_NONE ? 0 : r, batch, n, n, 1, 0,
              fuse == NE_FUSE_EXTRACT_CHECK ? flags : nullptr,
              fuse == NE_FUSE_EXTRACT_CHECK ? reinterpret_cast<unsigned long long*>(nflag) : nullptr, status};
    const bool vec2 = n % 2 == 0 && aligned(out, 16);
    launch_lsb<K_PERM>(a, fuse, vec2, s);
    return check_launch("ne_permute");
}

extern "C" ne_status ne_inner(ne_params p, const int64_t* eps, const int64_t* g, int64_t g_stride, int64_t* out,
                              uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t n, int32_t fuse, int32_t r,
                              cudaStream_t s) {
    ne_status st = lsb_common(p, batch, n, fuse, r, eps, out, "ne_inner");
    if (st) return st;
    if (g_stride < 0) return fail(NE_EINVAL, "ne_inner: g_stride < 0");
    if (batch > 0 && !out) return fail(NE_EINVAL, "ne_inner: null output");
    if (batch > 0 && n > 0 && !g) return fail(NE_EINVAL, "ne_inner: null operand");
    if ((st = reset_count(nflag, fuse, s, "ne_inner: reset count"))) return st;
    if (batch == 0) return NE_OK;
    unsigned long long* nf = fuse == NE_FUSE_EXTRACT_CHECK ? reinterpret_cast<unsigned long long*>(nflag) : nullptr;
    uint32_t* fl = fuse == NE_FUSE_EXTRACT_CHECK ? flags : nullptr;
    const int rr = fuse == NE_FUSE_NONE ? 0 : r;
    const bool vec2 = n % 2 == 0 && g_stride % 2 == 0 && aligned(eps, 16) && aligned(g, 16);
    switch (p.M) {
        case 3: return launch_inner<3>(eps, g, g_stride, out, fl, nf, p.M, p.l, rr, fuse, batch, n, vec2, s);
        case 4: return launch_inner<4>(eps, g, g_stride, out, fl, nf, p.M, p.l, rr, fuse, batch, n, vec2, s);
        case 5: return launch_inner<5>(eps, g, g_stride, out, fl, nf, p.M, p.l, rr, fuse, batch, n, vec2, s);
        default: return launch_inner<0>(eps, g, g_stride, out, fl, nf, p.M, p.l, rr, fuse, batch, n, vec2, s);
    }
}

extern "C" ne_status ne_entangle_kernel_self(int32_t l, const int64_t* g, int64_t* ge, int64_t n, cudaStream_t s) {
    if (l < 1 || l > 62 || n < 0) return fail(NE_EINVAL, "ne_entangle_kernel_self: l=%d n=%lld", l, (long long)n);
    if (n == 0) return NE_OK;
    if (!g || !ge) return fail(NE_EINVAL, "ne_entangle_kernel_self: null pointer");
    k_kernel_self<<<stream_blocks(n), 256, 0, s>>>(g, ge, l, n);
    return check_launch("ne_entangle_kernel_self");
}

extern "C" ne_status ne_reverse_operand(const int8_t* g, int8_t* g_rev, int64_t batch, int64_t N, cudaStream_t s) {
    if (batch < 0 || N < 0) return fail(NE_EINVAL, "ne_reverse_operand: batch=%lld N=%lld", (long long)batch,
                                        (long long)N);
    if (batch == 0 || N == 0) return NE_OK;
    if (!g || !g_rev || g == g_rev) return fail(NE_EINVAL, "ne_reverse_operand: null or aliased pointer");
    k_reverse<<<stream_blocks(batch * N), 256, 0, s>>>(g, g_rev, batch, N);
    return check_launch("ne_reverse_operand");
}
