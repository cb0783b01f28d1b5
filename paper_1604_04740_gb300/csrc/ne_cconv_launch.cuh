// Launch plumbing of the batched circular convolution on the int8 tensor path
// (the circular-convolution member of Eq. 2, applied per Eq. 10, with Eq.
// 17-20 / Eq. 24 fused into the epilogue), shared by the three entry points:
// ne_cconv_digits (digit planes in memory), ne_cconv_entangled (raw streams,
// Eq. 16 and the digit split while loading) and ne_cconv's S8SLICE mode (the
// entangled words split while loading), each compiled in its own translation
// unit.  One CTA computes one tile (up to 1024 outputs of one group, all
// streams and digits); the tiles are in ne_cconv_tile.cuh.
#pragma once

#include "ne_cconv_tile.cuh"
#include "ne_entangle.cuh"

namespace ne {
namespace cconv_launch {

// the process-wide tensor / dp4a split (ne_set_cconv_split; -1: the default)
extern int g_split;

namespace {


using namespace ne;

struct CconvArgs {
    const int8_t* planes;   // [batch][M][S][N]
    const int8_t* g;        // [batch][N]
    int64_t* out;           // [batch][M][N]
    uint32_t* flags;        // [batch][N/32] or null
    unsigned long long* nflag;
    int64_t N;
    int M, S, MS, l, r, fuse;
    int shift[NE_MAX_DIGITS];
    ne_faults faults;       // flat positions b * N + i (count 0: none)
    // words form: entangled words [batch][M][N] instead of planes (see TileArgs)
    const int64_t* cwords;
    uint64_t w_nsmask, w_nswant;
    // fused form: raw streams [batch][M][N] instead of planes (see TileArgs)
    const int32_t* craw;
    int32_t* status;
    uint32_t raw_off;
    int raw_lo, raw_hi, raw_plain;
    int raw_byte[4];
};

__device__ __forceinline__ void fault_fields(const CconvArgs& a, int64_t b, cconv::TileArgs& t) {
    t.fault_pos = a.faults.pos;
    t.fault_stream = a.faults.stream;
    t.fault_bit = a.faults.bit;
    t.nfault = a.faults.count;
    t.fault_base = b * a.N;
}

__device__ __forceinline__ void raw_fields(const CconvArgs& a, int64_t b, cconv::TileArgs& t) {
    t.cwords = a.cwords ? a.cwords + b * a.M * a.N : nullptr;
    t.w_nsmask = a.w_nsmask;
    t.w_nswant = a.w_nswant;
    t.craw = a.craw ? a.craw + b * a.M * a.N : nullptr;
    t.status = a.status;
    t.raw_off = a.raw_off;
    t.raw_lo = a.raw_lo;
    t.raw_hi = a.raw_hi;
    t.raw_plain = a.raw_plain;
#pragma unroll
    for (int i = 0; i < 4; i++) t.raw_byte[i] = a.raw_byte[i];
}

// IX: cconv::IX_CIRC for N a multiple of 64, cconv::IX_RAGGED otherwise
template <int NTW, int MT, int LD, int IX>
__global__ void __launch_bounds__(cconv::THREADS, (NTW <= 6 ? 4 : (NTW <= 10 ? 3 : 2)))
    k_cconv_digits(CconvArgs a, int64_t b_off) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int64_t b = b_off + blockIdx.y;
    const int64_t N = a.N;
    cconv::TileArgs t;
    t.planes = a.planes + b * a.MS * N;
    t.g = a.g + b * N;
    t.out = a.out + b * a.M * N;
    t.flags = a.flags ? a.flags + b * ((N + 31) / 32) : nullptr;
    t.nflag = a.nflag;
    fault_fields(a, b, t);
    t.N = (int)N;
    t.M = a.M;
    t.S = a.S;
    t.MS = a.MS;
    t.l = a.l;
    t.r = a.r;
    t.fuse = a.fuse;
    t.flags_atomic = 0;
#pragma unroll
    for (int i = 0; i < NE_MAX_DIGITS; i++) t.shift[i] = a.shift[i];
    raw_fields(a, b, t);
    t.lin_n = t.lin_K = (int)N;
    const int NB = (int)((N + cconv::T - 1) / cconv::T);
    const int p0 = blockIdx.x * cconv::NPB;
    cconv::tile<NTW, MT, LD, IX>(t, smem, p0, min(cconv::NPB, NB - p0));
}

// The hybrid tile (tensor pipe + dp4a pipe) for groups of 9..16 blocks
// (NBC: 16 for groups of exactly 16 blocks, compiled for that size; 0: any).
template <int MT, int MSC, int HW, int R, int LD, int NBC, int TW>
__global__ void __launch_bounds__(cconv::hybrid_threads(HW, TW),
                                  cconv::hybrid_threads(HW, TW) <= 256 ? 4 : (cconv::hybrid_threads(HW, TW) <= 384 ? 3 : 2))
    k_cconv_digits_hybrid(CconvArgs a, int64_t b_off) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int64_t b = b_off + blockIdx.y;
    const int64_t N = a.N;
    cconv::TileArgs t;
    t.planes = a.planes + b * a.MS * N;
    t.g = a.g + b * N;
    t.out = a.out + b * a.M * N;
    t.flags = a.flags ? a.flags + b * (N / 32) : nullptr;
    t.nflag = a.nflag;
    fault_fields(a, b, t);
    t.N = (int)N;
    t.M = a.M;
    t.S = a.S;
    t.MS = a.MS;
    t.l = a.l;
    t.r = a.r;
    t.fuse = a.fuse;
    t.flags_atomic = 0;
#pragma unroll
    for (int i = 0; i < NE_MAX_DIGITS; i++) t.shift[i] = a.shift[i];
    raw_fields(a, b, t);
    cconv::tile_hybrid<MT, MSC, HW, R, LD, NBC, TW>(t, smem);
}

template <int MT, int MSC, int HW, int R, int LD, int NBC, int TW = 8>
ne_status launch_hybrid(const CconvArgs& a, int64_t batch, cudaStream_t s) {
    if (a.N / cconv::T <= 32 * HW * R / cconv::T) return NE_EINVAL;   // needs a block left for the tensor pipe
    const int smem = cconv::hybrid_smem_bytes(MSC);
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(k_cconv_digits_hybrid<MT, MSC, HW, R, LD, NBC, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem) != cudaSuccess)
            return check_launch("ne_cconv_digits: shared-memory attribute");
        attr_set[dev] = true;
    }
    for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
        const int64_t nb = batch - b0 < 65535 ? batch - b0 : 65535;
        k_cconv_digits_hybrid<MT, MSC, HW, R, LD, NBC, TW>
            <<<dim3(1, (unsigned)nb), cconv::hybrid_threads(HW, TW), smem, s>>>(a, b0);
        ne_status st = check_launch("ne_cconv_digits (hybrid)");
        if (st) return st;
    }
    return NE_OK;
}

// Split of a group between the tensor pipe and the dp4a pipe (variant -1:
// the default).  Default for groups of 16 blocks (measured on GB300 at 4096
// groups of N = 1024): 8 blocks on 4 tensor warps and 8 on 4 dp4a warps of 4
// outputs per thread (variant 444: 4 CTAs per SM for 6 planes; M = 3 0.250 ms
// against 0.259 ms with 8 tensor warps (44) and 0.270 ms for 43; M = 4 0.330
// ms against 0.333 ms for 43).
// ne_set_cconv_split overrides it: 0 tensor pipe only; HR (23, 24, 34, 42,
// 43, 44) 8 tensor warps and H dp4a warps of R outputs per thread (H * R / 2
// blocks on dp4a), for any group of at most 16 blocks; 443, 444 the same
// dp4a share with 4 tensor warps (groups of 16 blocks; others take 43, 44).

int hybrid_variant(int64_t NB, int MS) {
    if (g_split == -1) return NB == 16 ? 444 : 0;
    return g_split;
}

// groups of 16 blocks from raw streams or planes take the tile compiled for that size
template <int MT, int MSC, int HW, int R, int LD>
ne_status launch_hybrid_n(const CconvArgs& a, int64_t batch, cudaStream_t s) {
    if constexpr (LD != cconv::LD_WORDS) {
        if (a.N == 16 * cconv::T) return launch_hybrid<MT, MSC, HW, R, LD, 16>(a, batch, s);
    }
    return launch_hybrid<MT, MSC, HW, R, LD, 0>(a, batch, s);
}

template <int MT, int MSC, int LD>
ne_status launch_hybrid_variant(int var, const CconvArgs& a, int64_t batch, cudaStream_t s) {
    switch (var) {
        case 23: return launch_hybrid_n<MT, MSC, 2, 3, LD>(a, batch, s);
        case 24: return launch_hybrid_n<MT, MSC, 2, 4, LD>(a, batch, s);
        case 34: return launch_hybrid_n<MT, MSC, 3, 4, LD>(a, batch, s);
        case 42: return launch_hybrid_n<MT, MSC, 4, 2, LD>(a, batch, s);
        case 43: return launch_hybrid_n<MT, MSC, 4, 3, LD>(a, batch, s);
        case 44: return launch_hybrid_n<MT, MSC, 4, 4, LD>(a, batch, s);
        // 4 tensor warps + 4 dp4a warps (4 CTAs per SM when shared memory
        // allows), groups of 16 blocks from raw streams or planes; otherwise
        // the same dp4a share with 8 tensor warps
        case 444:
        case 443:
            if constexpr (LD != cconv::LD_WORDS) {
                if (a.N == 16 * cconv::T)
                    return var == 444 ? launch_hybrid<MT, MSC, 4, 4, LD, 16, 4>(a, batch, s)
                                      : launch_hybrid<MT, MSC, 4, 3, LD, 16, 4>(a, batch, s);
            }
            return var == 444 ? launch_hybrid_n<MT, MSC, 4, 4, LD>(a, batch, s)
                              : launch_hybrid_n<MT, MSC, 4, 3, LD>(a, batch, s);
        default: return NE_EINVAL;
    }
}

template <int NTW, int MT, int LD, int IX>
ne_status launch_ix(const CconvArgs& a, int64_t batch, cudaStream_t s) {
    const int smem = cconv::smem_bytes(a.MS);
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(k_cconv_digits<NTW, MT, LD, IX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 cconv::smem_bytes(16)) != cudaSuccess)
            return check_launch("ne_cconv_digits: shared-memory attribute");
        attr_set[dev] = true;
    }
    const int NB = (int)((a.N + cconv::T - 1) / cconv::T);
    for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
        const int64_t nb = batch - b0 < 65535 ? batch - b0 : 65535;
        dim3 grid((NB + cconv::NPB - 1) / cconv::NPB, (unsigned)nb);
        k_cconv_digits<NTW, MT, LD, IX><<<grid, cconv::THREADS, smem, s>>>(a, b0);
        ne_status st = check_launch("ne_cconv_digits");
        if (st) return st;
    }
    return NE_OK;
}

// the aligned block form when N is a multiple of 64 and the streams start
// 16-byte aligned, else the ragged form
template <int NTW, int MT, int LD>
ne_status launch(const CconvArgs& a, int64_t batch, cudaStream_t s) {
    const void* src = LD == cconv::LD_PLANES ? (const void*)a.planes
                      : (LD == cconv::LD_RAW ? (const void*)a.craw : (const void*)a.cwords);
    if (a.N % cconv::T == 0 && aligned(src, 16) && aligned(a.g, 4))
        return launch_ix<NTW, MT, LD, cconv::IX_CIRC>(a, batch, s);
    return launch_ix<NTW, MT, LD, cconv::IX_RAGGED>(a, batch, s);
}

template <int LD>
ne_status dispatch(const CconvArgs& a, int64_t batch, cudaStream_t s) {
    const int64_t NB = a.N / cconv::T;
    const int var = hybrid_variant(NB, a.MS);
    const void* src = LD == cconv::LD_PLANES ? (const void*)a.planes
                      : (LD == cconv::LD_RAW ? (const void*)a.craw : (const void*)a.cwords);
    if (var && NB <= 16 && a.N % cconv::T == 0 && aligned(src, 16) && aligned(a.g, 4)) {
        ne_status hs = NE_EINVAL;
        if (a.M == 3 && a.MS == 6) hs = launch_hybrid_variant<3, 6, LD>(var, a, batch, s);
        else if (a.M == 4 && a.MS == 8) hs = launch_hybrid_variant<4, 8, LD>(var, a, batch, s);
        if (hs != NE_EINVAL) return hs;    // NE_EINVAL: this shape stays on the tensor pipe
    }
    const int MS = a.MS;
    // a warp holds at most MS column tiles (16 output blocks x MS planes / 8 / 2)
    switch (a.M) {
        case 3:
            if (MS <= 4) return launch<4, 3, LD>(a, batch, s);
            if (MS <= 6) return launch<6, 3, LD>(a, batch, s);
            return launch<10, 3, LD>(a, batch, s);
        case 4:
            if (MS <= 4) return launch<4, 4, LD>(a, batch, s);
            if (MS <= 8) return launch<8, 4, LD>(a, batch, s);
            return launch<12, 4, LD>(a, batch, s);
        case 5:
            if (MS <= 6) return launch<6, 5, LD>(a, batch, s);
            if (MS <= 10) return launch<10, 5, LD>(a, batch, s);
            return launch<16, 5, LD>(a, batch, s);
        case 8:   // the paper's other stream count (Sec. V: M in {3, 8})
            if (MS <= 8) return launch<8, 8, LD>(a, batch, s);
            return launch<16, 8, LD>(a, batch, s);
        default:
            return launch<16, 0, LD>(a, batch, s);
    }
}

ne_status common_args(const ne_params& p, const ne_digits& dg, int64_t batch, int64_t N, int32_t fuse, int32_t r,
                      const ne_faults& faults, const char* who) {
    ne_status st = validate_params(p);
    if (st) return st;
    if ((st = validate_digits(dg))) return st;
    if ((st = validate_faults(faults, who))) return st;
    if (batch < 0) return fail(NE_EINVAL, "%s: batch < 0", who);
    if (N < 1 || N > 65536) return fail(NE_EINVAL, "%s: N=%lld must be in [1, 65536]", who, (long long)N);
    if (fuse < NE_FUSE_NONE || fuse > NE_FUSE_RECOVER) return fail(NE_EINVAL, "%s: fuse=%d", who, fuse);
    if (r < 0 || r >= p.M) return fail(NE_EINVAL, "%s: r=%d", who, r);
    if (p.M * dg.S > 16) return fail(NE_EINVAL, "%s: M*S=%d exceeds 16 planes", who, p.M * dg.S);
    return NE_OK;
}

void fill_args(CconvArgs& a, const ne_params& p, const ne_digits& dg, const int8_t* g, int64_t* out, uint32_t* flags,
               unsigned long long* nf, int64_t N, int32_t fuse, int32_t r, const ne_faults& faults) {
    a.planes = nullptr;
    a.faults = faults;
    a.g = g;
    a.out = out;
    a.flags = (fuse == NE_FUSE_EXTRACT_CHECK) ? flags : nullptr;
    a.nflag = (fuse == NE_FUSE_EXTRACT_CHECK) ? nf : nullptr;
    a.N = N;
    a.M = p.M;
    a.S = dg.S;
    a.MS = p.M * dg.S;
    a.l = p.l;
    a.r = r;
    a.fuse = fuse;
    for (int i = 0; i < NE_MAX_DIGITS; i++) a.shift[i] = i < dg.S ? dg.shift[i] : 0;
    a.cwords = nullptr;
    a.w_nsmask = a.w_nswant = 0;
    a.craw = nullptr;
    a.status = nullptr;
    a.raw_off = 0;
    a.raw_lo = a.raw_hi = a.raw_plain = 0;
    for (int i = 0; i < 4; i++) a.raw_byte[i] = 0;
}


}  // namespace
}  // namespace cconv_launch
}  // namespace ne
