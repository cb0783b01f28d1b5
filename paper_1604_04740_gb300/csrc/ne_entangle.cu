// Entanglement (Eq. 7 for M = 3, Eq. 15-16 for general M) and the checksum
// encoder of the ABFT comparator (Eq. 4).  All three are streaming,
// HBM-bound kernels: one pass over the int32 input planes, 16-byte loads,
// every output written once.
//
// Traversal: blockIdx.y walks the groups (batch rows) and blockIdx.x/threads
// walk the positions of a row in chunks of VEC, so no division is needed to
// split a flat index into (group, position).
#include "ne_common.cuh"
#include "ne_entangle.cuh"

namespace {

using namespace ne;

// ---- int64 words -------------------------------------------------------------

template <int VEC>
__global__ void __launch_bounds__(256) k_entangle(const int32_t* __restrict__ c, int64_t* __restrict__ eps,
                                                  int M, int l, int64_t batch, int64_t n) {
    const int64_t nchunk = n / VEC;
    for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
        const int32_t* cb = c + b * M * n;
        int64_t* eb = eps + b * M * n;
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nchunk;
             q += (int64_t)gridDim.x * blockDim.x) {
            if constexpr (VEC == 4) {
                // the previous stream's chunk stays in registers: M + 1 loads per chunk
                int4 prev = __ldcs(reinterpret_cast<const int4*>(cb + (int64_t)(M - 1) * n + q * 4));
                for (int m = 0; m < M; m++) {
                    int4 cur = __ldcs(reinterpret_cast<const int4*>(cb + (int64_t)m * n + q * 4));
                    longlong2 lo, hi;
                    lo.x = entangle_word(cur.x, prev.x, l);
                    lo.y = entangle_word(cur.y, prev.y, l);
                    hi.x = entangle_word(cur.z, prev.z, l);
                    hi.y = entangle_word(cur.w, prev.w, l);
                    longlong2* dst = reinterpret_cast<longlong2*>(eb + (int64_t)m * n + q * 4);
                    __stcs(dst, lo);
                    __stcs(dst + 1, hi);
                    prev = cur;
                }
            } else {
                int32_t prev = cb[(int64_t)(M - 1) * n + q];
                for (int m = 0; m < M; m++) {
                    int32_t cur = cb[(int64_t)m * n + q];
                    eb[(int64_t)m * n + q] = entangle_word(cur, prev, l);
                    prev = cur;
                }
            }
        }
    }
}

// ---- digit planes --------------------------------------------------------------

struct DigitPlan {
    int S;
    int top;           // index of the highest digit that is computed (shift/8)
    uint32_t stored;   // bit t set: digit t is stored
    int slot[8];       // plane index of digit t (valid where stored)
};

// Balanced base-256 digits: digit t of a word is the signed low byte of the
// running remainder, and the remainder becomes (x - digit) / 256, exactly.
// Each thread takes VEC consecutive positions of a group (two 16-byte loads
// per input stream when VEC = 8) and writes one VEC-byte word per stored
// digit plane.  A non-zero digit that the plan does not store, or a
// remainder left after the top planned digit, reports NE_ERANGE.
template <int VEC>
__global__ void __launch_bounds__(256) k_entangle_digits(const int32_t* __restrict__ c, int8_t* __restrict__ planes,
                                                         int M, int l, DigitPlan P, int64_t batch, int64_t n,
                                                         int32_t* status) {
    const int64_t nchunk = n / VEC;
    bool ok = true;
    for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
        const int32_t* cb = c + b * M * n;
        int8_t* pb = planes + b * M * P.S * n;
        for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nchunk;
             q += (int64_t)gridDim.x * blockDim.x) {
            int32_t prev[VEC], cur[VEC];
            if constexpr (VEC == 8) {
                const int4* src = reinterpret_cast<const int4*>(cb + (int64_t)(M - 1) * n + q * 8);
                int4 a = __ldcs(src), bb = __ldcs(src + 1);
                prev[0] = a.x; prev[1] = a.y; prev[2] = a.z; prev[3] = a.w;
                prev[4] = bb.x; prev[5] = bb.y; prev[6] = bb.z; prev[7] = bb.w;
            } else {
                prev[0] = cb[(int64_t)(M - 1) * n + q];
            }
            for (int m = 0; m < M; m++) {
                if constexpr (VEC == 8) {
                    const int4* src = reinterpret_cast<const int4*>(cb + (int64_t)m * n + q * 8);
                    int4 a = __ldcs(src), bb = __ldcs(src + 1);
                    cur[0] = a.x; cur[1] = a.y; cur[2] = a.z; cur[3] = a.w;
                    cur[4] = bb.x; cur[5] = bb.y; cur[6] = bb.z; cur[7] = bb.w;
                } else {
                    cur[0] = cb[(int64_t)m * n + q];
                }
                int64_t x[VEC];
#pragma unroll
                for (int v = 0; v < VEC; v++) x[v] = entangle_word(cur[v], prev[v], l);
                int8_t* mp = pb + (int64_t)m * P.S * n + q * VEC;
#pragma unroll
                for (int t = 0; t < 8; t++) {
                    if (t > P.top) break;
                    uint32_t w0 = 0, w1 = 0;
                    bool nz = false;
#pragma unroll
                    for (int v = 0; v < VEC; v++) {
                        const int8_t d = (int8_t)(x[v] & 0xff);
                        nz |= (d != 0);
                        if (v < 4) w0 |= (uint32_t)(uint8_t)d << (8 * v);
                        else w1 |= (uint32_t)(uint8_t)d << (8 * (v - 4));
                        x[v] = (x[v] - d) >> 8;
                    }
                    if (P.stored & (1u << t)) {
                        int8_t* dst = mp + (int64_t)P.slot[t] * n;
                        if constexpr (VEC == 8) __stcs(reinterpret_cast<uint2*>(dst), make_uint2(w0, w1));
                        else dst[0] = (int8_t)w0;
                    } else {
                        ok = ok && !nz;
                    }
                }
#pragma unroll
                for (int v = 0; v < VEC; v++) {
                    ok = ok && (x[v] == 0);
                    prev[v] = cur[v];
                }
            }
        }
    }
    if (!ok && status) atomicExch(status, (int32_t)NE_ERANGE);
}

// Walks the flat space of (group, chunk) pairs with a grid stride, keeping
// the pair up to date by constant increments instead of a division per step.
struct FlatWalk {
    int64_t b, q, db, dq, nchunk;
    __device__ FlatWalk(int64_t start, int64_t stride, int64_t nchunk_) : nchunk(nchunk_) {
        b = start / nchunk;
        q = start - b * nchunk;
        db = stride / nchunk;
        dq = stride - db * nchunk;
    }
    __device__ void next() {
        q += dq;
        b += db;
        if (q >= nchunk) {
            q -= nchunk;
            b++;
        }
    }
};

// The common case (compile-time M, n a multiple of 8, aligned planes): every
// thread owns 8 positions of one group, issues the 2 x 16-byte loads of all
// M streams before any arithmetic, and writes one 8-byte word per stored
// digit plane and stream.
template <int MT>
__global__ void __launch_bounds__(256, 3) k_entangle_digits8(const int32_t* __restrict__ c, int8_t* __restrict__ planes,
                                                          int l, DigitPlan P, int64_t batch, int64_t n,
                                                          int32_t* status) {
    const int64_t nchunk = n / 8;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool ok = true;
    for (FlatWalk w((int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride, nchunk); w.b < batch; w.next()) {
        const int32_t* cb = c + w.b * MT * n + w.q * 8;
        int32_t v[MT][8];
#pragma unroll
        for (int m = 0; m < MT; m++) {
            const int4* src = reinterpret_cast<const int4*>(cb + (int64_t)m * n);
            const int4 a = __ldcs(src), bb = __ldcs(src + 1);
            v[m][0] = a.x; v[m][1] = a.y; v[m][2] = a.z; v[m][3] = a.w;
            v[m][4] = bb.x; v[m][5] = bb.y; v[m][6] = bb.z; v[m][7] = bb.w;
        }
        int8_t* pb = planes + w.b * MT * P.S * n + w.q * 8;
#pragma unroll
        for (int m = 0; m < MT; m++) {
            const int pm = (m + MT - 1) % MT;
            int64_t x[8];
#pragma unroll
            for (int e = 0; e < 8; e++) x[e] = entangle_word(v[m][e], v[pm][e], l);
#pragma unroll
            for (int t = 0; t < 8; t++) {
                if (t > P.top) break;
                uint32_t w0 = 0, w1 = 0;
                bool nz = false;
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    const int8_t d = (int8_t)(x[e] & 0xff);
                    nz |= (d != 0);
                    if (e < 4) w0 |= (uint32_t)(uint8_t)d << (8 * e);
                    else w1 |= (uint32_t)(uint8_t)d << (8 * (e - 4));
                    x[e] = (x[e] - d) >> 8;
                }
                if (P.stored & (1u << t))
                    __stcs(reinterpret_cast<uint2*>(pb + ((int64_t)m * P.S + P.slot[t]) * n), make_uint2(w0, w1));
                else
                    ok = ok && !nz;
            }
#pragma unroll
            for (int e = 0; e < 8; e++) ok = ok && (x[e] == 0);
        }
    }
    if (!ok && status) atomicExch(status, (int32_t)NE_ERANGE);
}

// Digit planes on the range-checked fast path (ne_entangle.cuh): eight
// positions per thread over the flat (group, chunk) space.
// PLAIN: the digits of the raw streams (no predecessor term).
template <int MT, bool PLAIN = false>
__global__ void __launch_bounds__(256) k_entangle_digits_fast(const int32_t* __restrict__ c, int8_t* __restrict__ planes,
                                                              int l, FastPlan F, int64_t batch, int64_t n,
                                                              int32_t* status) {
    const int64_t nchunk = n / 8;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t worst = 0;
    for (FlatWalk w((int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride, nchunk); w.b < batch; w.next())
        worst = max(worst, entangle_chunk8<MT, PLAIN>(c + w.b * MT * n + w.q * 8, planes + w.b * MT * F.S * n + w.q * 8,
                                                      n, l, F));
    if (worst > (uint32_t)F.hi - (uint32_t)F.lo && status) atomicExch(status, (int32_t)NE_ERANGE);
}

// int64 words with the same flat traversal: four positions per thread, the
// M 16-byte loads issued before the arithmetic.
template <int MT>
__global__ void __launch_bounds__(256) k_entangle_words4(const int32_t* __restrict__ c, int64_t* __restrict__ eps, int l,
                                                         int64_t batch, int64_t n) {
    const int64_t nchunk = n / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (FlatWalk w((int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride, nchunk); w.b < batch; w.next()) {
        const int32_t* cb = c + w.b * MT * n + w.q * 4;
        int4 v[MT];
#pragma unroll
        for (int m = 0; m < MT; m++) v[m] = __ldcs(reinterpret_cast<const int4*>(cb + (int64_t)m * n));
        int64_t* eb = eps + w.b * MT * n + w.q * 4;
#pragma unroll
        for (int m = 0; m < MT; m++) {
            const int4 cur = v[m], prev = v[(m + MT - 1) % MT];
            longlong2* dst = reinterpret_cast<longlong2*>(eb + (int64_t)m * n);
            __stcs(dst, make_longlong2(entangle_word(cur.x, prev.x, l), entangle_word(cur.y, prev.y, l)));
            __stcs(dst + 1, make_longlong2(entangle_word(cur.z, prev.z, l), entangle_word(cur.w, prev.w, l)));
        }
    }
}

int flat_blocks(int64_t chunks, int threads) {
    int64_t blocks = (chunks + threads - 1) / threads;
    const int64_t cap = (int64_t)wave_blocks(threads, 8);
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

// ---- checksum encoder (Eq. 4) -------------------------------------------------

__global__ void __launch_bounds__(256) k_abft_encode(const int32_t* __restrict__ c, int64_t* __restrict__ x,
                                                     int M, int64_t batch, int64_t n) {
    for (int64_t b = blockIdx.y; b < batch; b += gridDim.y) {
        const int32_t* cb = c + b * M * n;
        int64_t* xb = x + b * (M + 1) * n;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            int64_t sum = 0;
            for (int m = 0; m < M; m++) {
                int64_t v = cb[(int64_t)m * n + i];
                xb[(int64_t)m * n + i] = v;
                sum += v;
            }
            xb[(int64_t)M * n + i] = sum;
        }
    }
}

dim3 grid_rows(int64_t batch, int64_t chunks, int threads) {
    int64_t gy = batch < 65535 ? batch : 65535;
    int64_t want = (int64_t)wave_blocks(threads, 4);
    int64_t gx = (chunks + threads - 1) / threads;
    int64_t cap = want / gy;
    if (cap < 1) cap = 1;
    if (gx > cap) gx = cap;
    if (gx < 1) gx = 1;
    return dim3((unsigned)gx, (unsigned)gy, 1);
}

}  // namespace

extern "C" ne_status ne_entangle(ne_params p, const int32_t* c, int64_t* eps, int64_t batch, int64_t n,
                                 cudaStream_t s) {
    ne_status st = validate_params(p);
    if (st) return st;
    if (batch < 0 || n < 0) return fail(NE_EINVAL, "ne_entangle: batch=%lld n=%lld", (long long)batch, (long long)n);
    if (batch == 0 || n == 0) return NE_OK;
    if (!c || !eps) return fail(NE_EINVAL, "ne_entangle: null pointer");
    const int T = 256;
    if (n % 4 == 0 && aligned(c, 16) && aligned(eps, 16) && p.M <= 5) {
        const int blocks = flat_blocks(batch * (n / 4), T);
        switch (p.M) {
            case 3: k_entangle_words4<3><<<blocks, T, 0, s>>>(c, eps, p.l, batch, n); break;
            case 4: k_entangle_words4<4><<<blocks, T, 0, s>>>(c, eps, p.l, batch, n); break;
            default: k_entangle_words4<5><<<blocks, T, 0, s>>>(c, eps, p.l, batch, n); break;
        }
    } else if (n % 4 == 0 && aligned(c, 16) && aligned(eps, 16)) {
        k_entangle<4><<<grid_rows(batch, n / 4, T), T, 0, s>>>(c, eps, p.M, p.l, batch, n);
    } else {
        k_entangle<1><<<grid_rows(batch, n, T), T, 0, s>>>(c, eps, p.M, p.l, batch, n);
    }
    return check_launch("ne_entangle");
}

extern "C" ne_status ne_entangle_digits(ne_params p, ne_digits dg, const int32_t* c, int8_t* planes,
                                        int64_t batch, int64_t n, int32_t* status, cudaStream_t s) {
    ne_status st = validate_params(p);
    if (st) return st;
    if ((st = validate_digits(dg))) return st;
    if (batch < 0 || n < 0) return fail(NE_EINVAL, "ne_entangle_digits: batch=%lld n=%lld", (long long)batch, (long long)n);
    if (batch == 0 || n == 0) return NE_OK;
    if (!c || !planes) return fail(NE_EINVAL, "ne_entangle_digits: null pointer");
    DigitPlan P;
    P.S = dg.S;
    P.stored = 0;
    P.top = 0;
    for (int t = 0; t < 8; t++) P.slot[t] = 0;
    for (int s2 = 0; s2 < dg.S; s2++) {
        int t = dg.shift[s2] / 8;
        P.stored |= 1u << t;
        P.slot[t] = s2;
    }
    P.top = dg.shift[dg.S - 1] / 8;   // digits above the top planned one must be 0
    const int T = 256;
    const bool vec8 = n % 8 == 0 && aligned(c, 16) && aligned(planes, 8);
    // The fast path trusts the digit set only when it is exactly the plan of
    // its recorded (l, lo, hi): then every in-range input forms words whose
    // digits are in the set, and checking the inputs suffices.
    FastPlan F;
    bool planned = false;
    if (dg.lo <= dg.hi && dg.l == p.l) {
        ne_digits ref;
        if (ne_plan_digits(dg.l, dg.lo, dg.hi, &ref) == NE_OK && ref.S == dg.S) {
            planned = true;
            for (int s2 = 0; s2 < dg.S; s2++) planned = planned && ref.shift[s2] == dg.shift[s2];
        }
    }
    if (vec8 && p.M <= 5 && planned && make_fast_plan(dg, p.l, &F)) {
        const int blocks = flat_blocks(batch * (n / 8), T);
        switch (p.M) {
            case 3: k_entangle_digits_fast<3><<<blocks, T, 0, s>>>(c, planes, p.l, F, batch, n, status); break;
            case 4: k_entangle_digits_fast<4><<<blocks, T, 0, s>>>(c, planes, p.l, F, batch, n, status); break;
            default: k_entangle_digits_fast<5><<<blocks, T, 0, s>>>(c, planes, p.l, F, batch, n, status); break;
        }
    } else if (vec8 && p.M >= 3 && p.M <= 5) {
        const int64_t chunks = batch * (n / 8);
        int64_t blocks = (chunks + T - 1) / T;
        const int64_t cap = (int64_t)wave_blocks(T, 8);
        if (blocks > cap) blocks = cap;
        switch (p.M) {
            case 3: k_entangle_digits8<3><<<(unsigned)blocks, T, 0, s>>>(c, planes, p.l, P, batch, n, status); break;
            case 4: k_entangle_digits8<4><<<(unsigned)blocks, T, 0, s>>>(c, planes, p.l, P, batch, n, status); break;
            default: k_entangle_digits8<5><<<(unsigned)blocks, T, 0, s>>>(c, planes, p.l, P, batch, n, status); break;
        }
    } else if (n % 8 == 0 && aligned(c, 16) && aligned(planes, 8)) {
        k_entangle_digits<8><<<grid_rows(batch, n / 8, T), T, 0, s>>>(c, planes, p.M, p.l, P, batch, n, status);
    } else {
        k_entangle_digits<1><<<grid_rows(batch, n, T), T, 0, s>>>(c, planes, p.M, p.l, P, batch, n, status);
    }
    return check_launch("ne_entangle_digits");
}

extern "C" ne_status ne_split_digits_raw(ne_params p, ne_digits dg, const int32_t* c, int8_t* planes,
                                         int64_t batch, int64_t n, int32_t* status, cudaStream_t s) {
    ne_status st = validate_params(p);
    if (st) return st;
    if ((st = validate_digits(dg))) return st;
    if (batch < 0 || n < 0) return fail(NE_EINVAL, "ne_split_digits_raw: batch=%lld n=%lld", (long long)batch, (long long)n);
    if (p.M > 5) return fail(NE_EINVAL, "ne_split_digits_raw: M=%d exceeds 5", p.M);
    // the raw value c_m is the word of Eq. 16 with a zero predecessor, so its
    // digits are in the plan whenever 0 lies in the plan's range
    FastPlan F;
    bool planned = false;
    if (dg.S == 1 && dg.shift[0] == 0 && dg.lo <= dg.hi && dg.lo >= -128 && dg.hi <= 127) {
        // one digit: int8-valued streams as they are
        F.off = 0x80u;
        F.ns_mask = F.ns_want = 0;
        F.lim = 256u;
        F.S = 1;
        F.lo = dg.lo;
        F.hi = dg.hi;
        for (int t = 0; t < 4; t++) F.byte_of[t] = 0;
        F.pmask = 0;
        planned = true;
    } else if (dg.lo <= 0 && 0 <= dg.hi && dg.l == p.l) {
        ne_digits ref;
        planned = ne_plan_digits(dg.l, dg.lo, dg.hi, &ref) == NE_OK && ref.S == dg.S;
        for (int s2 = 0; planned && s2 < dg.S; s2++) planned = ref.shift[s2] == dg.shift[s2];
        planned = planned && make_fast_plan(dg, p.l, &F);
    }
    if (!planned)
        return fail(NE_EINVAL, "ne_split_digits_raw: dg must be one digit of values in [-128, 127] or the plan of "
                               "(l, lo, hi) with lo <= 0 <= hi and words of at most 4 digits");
    if (n % 8 != 0 || !aligned(c, 16) || !aligned(planes, 8))
        return fail(NE_EINVAL, "ne_split_digits_raw: n must be a multiple of 8, c 16-byte and planes 8-byte aligned");
    if (batch == 0 || n == 0) return NE_OK;
    if (!c || !planes) return fail(NE_EINVAL, "ne_split_digits_raw: null pointer");
    const int T = 256;
    const int blocks = flat_blocks(batch * (n / 8), T);
    switch (p.M) {
        case 3: k_entangle_digits_fast<3, true><<<blocks, T, 0, s>>>(c, planes, p.l, F, batch, n, status); break;
        case 4: k_entangle_digits_fast<4, true><<<blocks, T, 0, s>>>(c, planes, p.l, F, batch, n, status); break;
        default: k_entangle_digits_fast<5, true><<<blocks, T, 0, s>>>(c, planes, p.l, F, batch, n, status); break;
    }
    return check_launch("ne_split_digits_raw");
}

extern "C" ne_status ne_abft_encode(int32_t M, const int32_t* c, int64_t* x, int64_t batch, int64_t n,
                                    cudaStream_t s) {
    if (M < 1 || M > 64 || batch < 0 || n < 0) return fail(NE_EINVAL, "ne_abft_encode: M=%d", M);
    if (batch == 0 || n == 0) return NE_OK;
    if (!c || !x) return fail(NE_EINVAL, "ne_abft_encode: null pointer");
    const int T = 256;
    k_abft_encode<<<grid_rows(batch, n, T), T, 0, s>>>(c, x, M, batch, n);
    return check_launch("ne_abft_encode");
}

// ---- digit planes of existing int64 words -------------------------------------

namespace {

__global__ void __launch_bounds__(256) k_split_digits(const int64_t* __restrict__ x, int8_t* __restrict__ planes,
                                                      DigitPlan P, int64_t batch, int Pl, int64_t n, int32_t* status) {
    bool ok = true;
    const int64_t rows = batch * Pl;
    for (int64_t row = blockIdx.y; row < rows; row += gridDim.y) {
        const int64_t* xr = x + row * n;
        int8_t* pr = planes + row * P.S * n;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            int64_t v = xr[i];
#pragma unroll
            for (int t = 0; t < 8; t++) {
                if (t > P.top) break;
                const int8_t d = (int8_t)(v & 0xff);
                if (P.stored & (1u << t)) pr[(int64_t)P.slot[t] * n + i] = d;
                else ok = ok && (d == 0);
                v = (v - d) >> 8;
            }
            ok = ok && (v == 0);
        }
    }
    if (!ok && status) atomicExch(status, (int32_t)NE_ERANGE);
}

}  // namespace

extern "C" ne_status ne_split_digits(ne_digits dg, const int64_t* x, int8_t* planes, int64_t batch, int32_t Pl,
                                     int64_t n, int32_t* status, cudaStream_t s) {
    ne_status st = validate_digits(dg);
    if (st) return st;
    if (batch < 0 || n < 0 || Pl < 1) return fail(NE_EINVAL, "ne_split_digits: bad sizes");
    if (batch == 0 || n == 0) return NE_OK;
    if (!x || !planes) return fail(NE_EINVAL, "ne_split_digits: null pointer");
    DigitPlan P;
    P.S = dg.S;
    P.stored = 0;
    for (int t = 0; t < 8; t++) P.slot[t] = 0;
    for (int s2 = 0; s2 < dg.S; s2++) {
        P.stored |= 1u << (dg.shift[s2] / 8);
        P.slot[dg.shift[s2] / 8] = s2;
    }
    P.top = dg.shift[dg.S - 1] / 8;
    k_split_digits<<<grid_rows(batch * Pl, n, 256), 256, 0, s>>>(x, planes, P, batch, Pl, n, status);
    return check_launch("ne_split_digits");
}
