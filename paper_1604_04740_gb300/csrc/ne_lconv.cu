// Linear convolution of long entangled streams with a short kernel, the
// convolution of the paper's second experiment (Sec. V: streams of 10^6
// samples, kernels of 100 to 4500 taps), on the int8 tensor path in one
// launch from the raw streams to the extracted outputs.
//
// Sec. IV-A processes a long stream as overlapping blocks of about the
// kernel's length (overlap-save).  Here every tile of 1024 outputs is such a
// block: it reads the input blocks its outputs reach (K + 1023 inputs, the
// overlap being the kernel's K - 1) and sums the block-Toeplitz products of
// the kernel blocks G_u[q][t] = g[64 u + q - t], so no output is computed
// twice and nothing is discarded; Eq. 16 and the digit split are done while
// the window loads and the extraction/check of Eq. 17-20 / Eq. 24 runs in
// the epilogue (ne_cconv_tile.cuh, IX_LINEAR).
#include "ne_cconv_tile.cuh"
#include "ne_entangle.cuh"

namespace {

using namespace ne;

constexpr int KMAX = 131071;    // |digit-plane sum| <= K 2^14 < 2^31

struct LconvArgs {
    const int32_t* c;           // [batch][M][n]
    const int8_t* g;            // [batch][K]
    int64_t* out;               // [batch][M][n + K - 1]
    uint32_t* flags;            // [batch][ceil((n + K - 1) / 32)] or null
    unsigned long long* nflag;
    int n, K, n_out;
    int M, S, MS, l, r, fuse;
    int shift[NE_MAX_DIGITS];
    ne_faults faults;           // flat positions b * (n + K - 1) + i
    int32_t* status;
    uint32_t raw_off;
    int raw_lo, raw_hi, raw_plain;
    int raw_byte[4];
};

template <int NTW, int MT>
__global__ void __launch_bounds__(cconv::THREADS, (NTW <= 6 ? 4 : (NTW <= 10 ? 3 : 2)))
    k_lconv(LconvArgs a, int64_t b_off) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int64_t b = b_off + blockIdx.y;
    const int64_t wpr = (a.n_out + 31) / 32;
    cconv::TileArgs t;
    t.planes = nullptr;
    t.g = a.g + b * a.K;
    t.out = a.out + b * a.M * (int64_t)a.n_out;
    t.flags = a.flags ? a.flags + b * wpr : nullptr;
    t.nflag = a.nflag;
    t.fault_pos = a.faults.pos;
    t.fault_stream = a.faults.stream;
    t.fault_bit = a.faults.bit;
    t.nfault = a.faults.count;
    t.fault_base = b * a.n_out;
    t.N = a.n_out;
    t.M = a.M;
    t.S = a.S;
    t.MS = a.MS;
    t.l = a.l;
    t.r = a.r;
    t.fuse = a.fuse;
    t.flags_atomic = 0;
#pragma unroll
    for (int i = 0; i < NE_MAX_DIGITS; i++) t.shift[i] = a.shift[i];
    t.craw = a.c + b * a.M * (int64_t)a.n;
    t.status = a.status;
    t.raw_off = a.raw_off;
    t.raw_lo = a.raw_lo;
    t.raw_hi = a.raw_hi;
    t.raw_plain = a.raw_plain;
#pragma unroll
    for (int i = 0; i < 4; i++) t.raw_byte[i] = a.raw_byte[i];
    t.cwords = nullptr;
    t.w_nsmask = t.w_nswant = 0;
    t.lin_n = a.n;
    t.lin_K = a.K;
    const int NBo = (a.n_out + cconv::T - 1) / cconv::T;
    const int p0 = blockIdx.x * cconv::NPB;
    cconv::tile<NTW, MT, cconv::LD_RAW, cconv::IX_LINEAR>(t, smem, p0, min(cconv::NPB, NBo - p0));
}

template <int NTW, int MT>
ne_status launch(const LconvArgs& a, int64_t batch, cudaStream_t s) {
    const int smem = cconv::smem_bytes(a.MS);
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(k_lconv<NTW, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 cconv::smem_bytes(16)) != cudaSuccess)
            return check_launch("ne_lconv: shared-memory attribute");
        attr_set[dev] = true;
    }
    const int64_t NBo = (a.n_out + cconv::T - 1) / cconv::T;
    const int64_t tiles = (NBo + cconv::NPB - 1) / cconv::NPB;
    for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
        const int64_t nb = batch - b0 < 65535 ? batch - b0 : 65535;
        k_lconv<NTW, MT><<<dim3((unsigned)tiles, (unsigned)nb), cconv::THREADS, smem, s>>>(a, b0);
        ne_status st = check_launch("ne_lconv");
        if (st) return st;
    }
    return NE_OK;
}

ne_status dispatch(const LconvArgs& a, int64_t batch, cudaStream_t s) {
    const int MS = a.MS;
    switch (a.M) {
        case 3:
            if (MS <= 4) return launch<4, 3>(a, batch, s);
            if (MS <= 6) return launch<6, 3>(a, batch, s);
            return launch<10, 3>(a, batch, s);
        case 4:
            if (MS <= 4) return launch<4, 4>(a, batch, s);
            if (MS <= 8) return launch<8, 4>(a, batch, s);
            return launch<12, 4>(a, batch, s);
        case 5:
            if (MS <= 6) return launch<6, 5>(a, batch, s);
            if (MS <= 10) return launch<10, 5>(a, batch, s);
            return launch<16, 5>(a, batch, s);
        case 8:   // the paper's other stream count (Sec. V: M in {3, 8})
            if (MS <= 8) return launch<8, 8>(a, batch, s);
            return launch<16, 8>(a, batch, s);
        default:
            return launch<16, 0>(a, batch, s);
    }
}

}  // namespace

extern "C" ne_status ne_lconv(ne_params p, ne_digits dg, const int32_t* c, const int8_t* g, int64_t* out,
                              uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t n, int64_t K, int32_t fuse,
                              int32_t r, int32_t plain, ne_faults faults, int32_t* status, cudaStream_t s) {
    ne_status st = validate_params(p);
    if (st) return st;
    if ((st = validate_digits(dg))) return st;
    if ((st = validate_faults(faults, "ne_lconv"))) return st;
    if (batch < 0) return fail(NE_EINVAL, "ne_lconv: batch < 0");
    if (n < 1 || K < 1 || K > KMAX) return fail(NE_EINVAL, "ne_lconv: n=%lld, K=%lld (1 <= K <= %d)", (long long)n,
                                                (long long)K, KMAX);
    if (n + K - 1 > ((int64_t)1 << 30)) return fail(NE_EINVAL, "ne_lconv: n + K - 1 exceeds 2^30 outputs");
    if (fuse < NE_FUSE_NONE || fuse > NE_FUSE_RECOVER) return fail(NE_EINVAL, "ne_lconv: fuse=%d", fuse);
    if (r < 0 || r >= p.M) return fail(NE_EINVAL, "ne_lconv: r=%d", r);
    if (p.M * dg.S > 16) return fail(NE_EINVAL, "ne_lconv: M*S=%d exceeds 16 planes", p.M * dg.S);
    if (plain && fuse != NE_FUSE_NONE) return fail(NE_EINVAL, "ne_lconv: the plain operation has no extraction");
    uint32_t off = 0;
    int byte_of[4] = {0, 0, 0, 0};
    if (plain && dg.S == 1 && dg.shift[0] == 0 && dg.lo <= dg.hi && dg.lo >= -128 && dg.hi <= 127) {
        off = 0x80u;
    } else {
        ne_digits ref;
        FastPlan F;
        bool planned = dg.lo <= dg.hi && dg.l == p.l && ne_plan_digits(dg.l, dg.lo, dg.hi, &ref) == NE_OK &&
                       ref.S == dg.S && (!plain || (dg.lo <= 0 && 0 <= dg.hi));
        for (int i = 0; planned && i < dg.S; i++) planned = ref.shift[i] == dg.shift[i];
        if (!planned || !make_fast_plan(dg, p.l, &F))
            return fail(NE_EINVAL, "ne_lconv: dg must be the plan of (l, lo, hi) with words of at most 4 digits "
                                   "(plain: or one digit of values in [-128, 127])");
        off = F.off;
        for (int i = 0; i < 4; i++) byte_of[i] = F.byte_of[i];
    }
    unsigned long long* nf = reinterpret_cast<unsigned long long*>(nflag);
    if (nf && cudaMemsetAsync(nf, 0, sizeof(*nf), s) != cudaSuccess) return check_launch("ne_lconv: reset");
    if (batch == 0) return NE_OK;
    if (!c || !g || !out) return fail(NE_EINVAL, "ne_lconv: null pointer");
    if (!aligned(c, 16) || !aligned(out, 8)) return fail(NE_EINVAL, "ne_lconv: c must be 16-byte aligned");
    LconvArgs a;
    a.c = c;
    a.g = g;
    a.out = out;
    a.flags = fuse == NE_FUSE_EXTRACT_CHECK ? flags : nullptr;
    a.nflag = fuse == NE_FUSE_EXTRACT_CHECK ? nf : nullptr;
    a.n = (int)n;
    a.K = (int)K;
    a.n_out = (int)(n + K - 1);
    a.M = p.M;
    a.S = dg.S;
    a.MS = p.M * dg.S;
    a.l = p.l;
    a.r = r;
    a.fuse = fuse;
    for (int i = 0; i < NE_MAX_DIGITS; i++) a.shift[i] = i < dg.S ? dg.shift[i] : 0;
    a.faults = faults;
    a.status = status;
    a.raw_off = off;
    a.raw_lo = dg.lo;
    a.raw_hi = dg.hi;
    a.raw_plain = plain ? 1 : 0;
    for (int i = 0; i < 4; i++) a.raw_byte[i] = byte_of[i];
    return dispatch(a, batch, s);
}
