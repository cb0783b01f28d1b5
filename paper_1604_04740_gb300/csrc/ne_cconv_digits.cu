// Batched circular convolution of entangled streams on the int8 tensor path
// (the circular-convolution member of Eq. 2, applied per Eq. 10), with the
// extraction and check of Eq. 17-20 / Eq. 24 fused into the epilogue.
//
// Every entangled word is held as balanced base-256 digit planes sigma_s
// (ne_entangle_digits), so that
//     delta_m[i] = sum_s 2^shift_s  sum_j sigma_{m,s}[j] g[(i - j) mod N]
// and each inner sum is an exact int8 x int8 -> int32 contraction (|sum| <=
// N 2^14 < 2^31 for N <= 65536).
//
// Block-Toeplitz form.  With i = T p + q and j = T p' + t (T = 64),
//     sum_j sigma[j] g[(i - j) mod N] = sum_u sum_t G_u[q][t] sigma[T (p - u) + t],
//     G_u[q][t] = g[(T u + q - t) mod N],
// so for each shift u the block G_u (T x T, Toeplitz) multiplies a matrix
// whose columns are the input blocks p - u of every digit plane.  One CTA
// owns NPB = 16 output blocks (1024 outputs) of one group and all planes:
//   D[q][(p, plane)] += sum_t G_u[q][t] B_u[t][(p, plane)],
// a dense T x (16 * planes) x T product per u, on mma.sync.m16n8k32.
// G_u is read from four byte-shifted copies of a reversed window of g in
// shared memory (every lane reads aligned words); the digit planes of the
// input blocks a u-chunk needs sit in shared memory, block-major, 80-byte
// rows, so the ldmatrix rows of any 8 consecutive columns hit distinct banks.
// The epilogue recombines the digits in int64, then extracts/checks per
// position exactly like the stand-alone kernel (shared code).
#include "ne_common.cuh"
#include "ne_extract.cuh"
#include "ne_mma.cuh"

namespace {

using namespace ne;

constexpr int T = 64;                  // Toeplitz block
constexpr int NPB = 16;                // output blocks per CTA
constexpr int UCH = 16;                // shifts u per chunk
constexpr int ROWB = 80;               // bytes per (block, plane) row in shared memory
constexpr int PADB = 16;               // margin of each g copy
constexpr int GW = 1184;               // bytes per g copy (>= T (UCH+1) + 2 PADB, = 32 mod 128)
constexpr int WBMAX = NPB + UCH - 1;   // input blocks a chunk can touch
constexpr int THREADS = 256;           // 8 warps: 4 row tiles x 2 column halves
constexpr int SP = 68;                 // stash row stride (int32) per output block

struct CconvArgs {
    const int8_t* planes;   // [batch][M][S][N]
    const int8_t* g;        // [batch][N]
    int64_t* out;           // [batch][M][N]
    uint32_t* flags;        // [batch][N/32] or null
    unsigned long long* nflag;
    int64_t N;
    int M, S, MS, l, r, fuse;
    int shift[NE_MAX_DIGITS];
};

__host__ __device__ constexpr int smem_bytes(int MS) {
    return (WBMAX * MS * ROWB + 4 * GW) > (MS * NPB * SP * 4) ? (WBMAX * MS * ROWB + 4 * GW) : (MS * NPB * SP * 4);
}

__device__ __forceinline__ int64_t shl64(int64_t x, int s) { return (int64_t)((uint64_t)x << s); }

template <int MT>
__device__ __forceinline__ void cconv_epilogue(const CconvArgs& a, const int32_t* stash, int64_t b, int p0, int npb) {
    const int M = MT ? MT : a.M;
    const int S = a.S;
    const int lane = threadIdx.x & 31;
    const int npos = npb * T;
    const int64_t N = a.N;
    const bool check = (a.fuse == NE_FUSE_EXTRACT_CHECK);
    const bool need_r = (a.fuse != NE_FUSE_RECOVER);
    int64_t* ob = a.out + b * M * N + (int64_t)p0 * T;
    for (int base = threadIdx.x & ~31; base < npos; base += THREADS) {
        const int i = base + lane;
        const int pr = i / T, q = i % T;
        const int32_t* sp = stash + pr * SP + q;
        if (a.fuse == NE_FUSE_NONE) {
            for (int m = 0; m < M; m++) {
                int64_t v = 0;
                
#pragma unroll
                    for (int s = 0; s < NE_MAX_DIGITS; s++)
                        if (s < S) v += shl64(sp[(m * S + s) * NPB * SP], a.shift[s]);
                ob[(int64_t)m * N + i] = v;
            }
            continue;
        }
        int64_t rot[MT ? MT : 32], res[MT ? MT : 32];
#pragma unroll
        for (int j = 0; j < (MT ? MT : 32); j++) {
            if (!MT && j >= M) break;
            int m = a.r + j;
            if (m >= M) m -= M;
            int64_t v = 0;
            if (j > 0 || need_r)
                
#pragma unroll
                    for (int s = 0; s < NE_MAX_DIGITS; s++)
                        if (s < S) v += shl64(sp[(m * S + s) * NPB * SP], a.shift[s]);
            rot[j] = v;
        }
        const bool f = extract_rot<MT>(rot, M, a.l, check, res);
#pragma unroll
        for (int j = 0; j < (MT ? MT : 32); j++) {
            if (!MT && j >= M) break;
            int m = a.r + j;
            if (m >= M) m -= M;
            ob[(int64_t)m * N + i] = res[j];
        }
        if (check) {
            const uint32_t w = __ballot_sync(0xffffffffu, f);
            if (lane == 0) {
                if (a.flags) a.flags[b * (N / 32) + ((int64_t)p0 * T + base) / 32] = w;
                if (a.nflag && w) atomicAdd(a.nflag, (unsigned long long)__popc(w));
            }
        }
    }
}

template <int NTW, int MT>
__global__ void __launch_bounds__(THREADS, (NTW <= 6 ? 4 : (NTW <= 10 ? 3 : 2))) k_cconv_digits(CconvArgs a, int64_t b_off) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int MS = a.MS;
    const int64_t N = a.N;
    const int NB = (int)(N / T);
    const int64_t b = b_off + blockIdx.y;
    const int p0 = blockIdx.x * NPB;
    const int npb = min(NPB, NB - p0);
    const int uch = min(UCH, NB);
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

    const int8_t* gb = a.g + b * N;
    const int8_t* pb = a.planes + b * MS * N;

    for (int u0 = 0; u0 < NB; u0 += uch) {
        const int uc = min(uch, NB - u0);
        // digit planes of input blocks (p0 - (u0 + uch - 1) + blk_rel) mod NB
        const int nchunks = WB * MS * 4;
        for (int e = tid; e < nchunks; e += THREADS) {
            const int c16 = e & 3, row = e >> 2;
            const int blk_rel = row / MS, ms = row - blk_rel * MS;
            int ab = (p0 - (u0 + uch - 1) + blk_rel) % NB;
            if (ab < 0) ab += NB;
            const int8_t* src = pb + (int64_t)ms * N + (int64_t)ab * T + c16 * 16;
            const bool lost = (a.fuse == NE_FUSE_RECOVER) && (ms / a.S == a.r);
            cp_async16(sig_s + row * ROWB + c16 * 16, src, lost ? 0 : 16);
        }
        cp_async_commit();
        // g copies: copy rr, byte z holds g[(T (u0 + uch) - (z + rr - PADB)) mod N]
        const int64_t top = (int64_t)T * (u0 + uch);
        for (int e = tid; e < 4 * (GW / 4); e += THREADS) {
            const int rr = e / (GW / 4), zw = e - rr * (GW / 4);
            uint32_t w = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                int64_t idx = (top - (4 * zw + k + rr - PADB)) % N;
                if (idx < 0) idx += N;
                w |= (uint32_t)(uint8_t)__ldg(gb + idx) << (8 * k);
            }
            *reinterpret_cast<uint32_t*>(gcp + rr * GW + 4 * zw) = w;
        }
        cp_async_wait<0>();
        __syncthreads();

        for (int u = u0; u < u0 + uc; u++) {
            const int ushift = u0 + uch - 1 - u;
            const int Y0 = T * (u0 + uch - u) - 16 * mt - gq;
#pragma unroll
            for (int ks = 0; ks < 2; ks++) {
                const int t0 = 32 * ks;
                const uint32_t ya = gcp_s + Y0 + t0 + 4 * tq;
                uint32_t af[4];
                af[0] = lds32(ya);
                af[1] = lds32(ya - 8);
                af[2] = lds32(ya + 16);
                af[3] = lds32(ya + 8);
#pragma unroll
                for (int jj = 0; jj < NTW; jj += 2) {
                    if (jj >= ntile) break;
                    int c = 8 * (tile0 + jj + (lane >> 4)) + (lane & 7);
                    if (c >= cols) c = 0;    // padding column: any valid row, result dropped
                    uint32_t bf[4];
                    ldsm_x4(bf, sig_s + (c + MS * ushift) * ROWB + t0 + 16 * kh);
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
    cconv_epilogue<MT>(a, stash, b, p0, npb);
}

template <int NTW, int MT>
ne_status launch(const CconvArgs& a, int64_t batch, cudaStream_t s) {
    const int smem = smem_bytes(a.MS);
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        if (cudaFuncSetAttribute(k_cconv_digits<NTW, MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_bytes(16)) != cudaSuccess)
            return check_launch("ne_cconv_digits: shared-memory attribute");
        attr_set[dev] = true;
    }
    const int NB = (int)(a.N / T);
    for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
        const int64_t nb = batch - b0 < 65535 ? batch - b0 : 65535;
        dim3 grid((NB + NPB - 1) / NPB, (unsigned)nb);
        k_cconv_digits<NTW, MT><<<grid, THREADS, smem, s>>>(a, b0);
        ne_status st = check_launch("ne_cconv_digits");
        if (st) return st;
    }
    return NE_OK;
}

}  // namespace

extern "C" ne_status ne_cconv_digits(ne_params p, ne_digits dg, const int8_t* planes, const int8_t* g, int64_t* out,
                                     uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t N, int32_t fuse,
                                     int32_t r, cudaStream_t s) {
    ne_status st = validate_params(p);
    if (st) return st;
    if ((st = validate_digits(dg))) return st;
    if (batch < 0) return fail(NE_EINVAL, "ne_cconv_digits: batch < 0");
    if (N < 64 || N % 64 != 0 || N > 65536)
        return fail(NE_EINVAL, "ne_cconv_digits: N=%lld must be a multiple of 64 in [64, 65536]", (long long)N);
    if (fuse < NE_FUSE_NONE || fuse > NE_FUSE_RECOVER) return fail(NE_EINVAL, "ne_cconv_digits: fuse=%d", fuse);
    if (r < 0 || r >= p.M) return fail(NE_EINVAL, "ne_cconv_digits: r=%d", r);
    const int MS = p.M * dg.S;
    if (MS > 16) return fail(NE_EINVAL, "ne_cconv_digits: M*S=%d exceeds 16 planes", MS);
    unsigned long long* nf = reinterpret_cast<unsigned long long*>(nflag);
    if (nf && cudaMemsetAsync(nf, 0, sizeof(*nf), s) != cudaSuccess) return check_launch("ne_cconv_digits: reset");
    if (batch == 0) return NE_OK;
    if (!planes || !g || !out) return fail(NE_EINVAL, "ne_cconv_digits: null pointer");
    if (!aligned(planes, 16) || !aligned(out, 8)) return fail(NE_EINVAL, "ne_cconv_digits: planes must be 16-byte aligned");
    CconvArgs a;
    a.planes = planes;
    a.g = g;
    a.out = out;
    a.flags = (fuse == NE_FUSE_EXTRACT_CHECK) ? flags : nullptr;
    a.nflag = (fuse == NE_FUSE_EXTRACT_CHECK) ? nf : nullptr;
    a.N = N;
    a.M = p.M;
    a.S = dg.S;
    a.MS = MS;
    a.l = p.l;
    a.r = r;
    a.fuse = fuse;
    for (int i = 0; i < NE_MAX_DIGITS; i++) a.shift[i] = i < dg.S ? dg.shift[i] : 0;
    // a warp holds at most MS column tiles (16 output blocks x MS planes / 8 / 2)
    switch (p.M) {
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
        default:
            return launch<16, 0>(a, batch, s);
    }
}
