// The LSB operations of Eq. 10 on CUDA cores in 64-bit integer arithmetic:
// the same kernel computes the plain operation on raw streams (widened to
// int64) and the entangled operation on entangled words, unaware of which
// it is given (Sec. II-B: the operation is unchanged by entanglement).
//
//   ne_gemm : out[p] = x[p] * G        (the GEMM experiment of Sec. V)
//   ne_cconv: out[b][p] = x[b][p] (*) g[b]  circular convolution (Eq. 2)
#include "ne_common.cuh"

namespace {

using namespace ne;

// ---- GEMM: 64x64 output tile, 256 threads, 4x4 int64 accumulators each -----

constexpr int GBM = 64, GBN = 64, GBK = 32;

__global__ void __launch_bounds__(256) k_gemm_i64(const int64_t* __restrict__ x, const int8_t* __restrict__ G,
                                                  int64_t* __restrict__ out, int rows, int cols, int k,
                                                  uint32_t skip_mask) {
    const int p = blockIdx.z;
    if (skip_mask & (1u << p)) return;   // fail-stopped plane: not computed
    __shared__ int64_t As[GBK][GBM + 1];
    __shared__ __align__(16) int32_t Bs[GBK][GBN];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int row0 = blockIdx.y * GBM, col0 = blockIdx.x * GBN;
    const int64_t* xp = x + (int64_t)p * rows * k;
    int64_t acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0;

    for (int k0 = 0; k0 < k; k0 += GBK) {
        // A tile: 64 rows x 32 k, coalesced along k, stored transposed
#pragma unroll
        for (int e = 0; e < (GBM * GBK) / 256; e++) {
            int idx = tid + e * 256;
            int r = idx / GBK, kk = idx % GBK;
            int gr = row0 + r, gk = k0 + kk;
            As[kk][r] = (gr < rows && gk < k) ? xp[(int64_t)gr * k + gk] : 0;
        }
        // B tile: 32 k x 64 cols, int8 widened to int32
#pragma unroll
        for (int e = 0; e < (GBK * GBN) / 256; e++) {
            int idx = tid + e * 256;
            int kk = idx / GBN, c = idx % GBN;
            int gk = k0 + kk, gc = col0 + c;
            Bs[kk][c] = (gk < k && gc < cols) ? (int32_t)G[(int64_t)gk * cols + gc] : 0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < GBK; kk++) {
            int64_t a[4];
            int4 bv = *reinterpret_cast<const int4*>(&Bs[kk][tx * 4]);
            int32_t b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] += a[i] * (int64_t)b[j];
        }
        __syncthreads();
    }
    int64_t* op = out + (int64_t)p * rows * cols;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int gr = row0 + ty * 4 + i;
        if (gr >= rows) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int gc = col0 + tx * 4 + j;
            if (gc < cols) op[(int64_t)gr * cols + gc] = acc[i][j];
        }
    }
}

// ---- circular convolution, direct form ----------------------------------------
//
// A block computes CI = 128 * 8 consecutive outputs of one plane; thread t
// owns outputs i0 + 8t .. i0 + 8t + 7.  Inputs are consumed in tiles of CJ
// values.  For the tile, the kernel values needed are
//   g[(i - j) mod N]  for il = i - i0 in [0, CI), jl = j - j0 in [0, CJ),
// stored once in shared memory as gw[u] = g[(i0 - j0 - CJ + u) mod N] so that
// g[(i - j) mod N] = gw[il - jl + CJ].  For 8 consecutive jl the thread's 64
// products use the 16 bytes gw[8t - jl + CJ - 8 ...], loaded as two aligned
// 8-byte words, so shared-memory traffic is two 8-byte loads (one of them
// reused from the previous step) plus broadcast loads of x per 64 products.
constexpr int CT = 128, CR = 8, CI = CT * CR, CJ = 1024;

__global__ void __launch_bounds__(CT) k_cconv_i64(const int64_t* __restrict__ x, const int8_t* __restrict__ g,
                                                  int64_t* __restrict__ out, int P, int64_t N, uint32_t skip_mask) {
    const int p = blockIdx.y;
    if (skip_mask & (1u << p)) return;
    const int64_t b = blockIdx.z;
    const int64_t i0 = (int64_t)blockIdx.x * CI;
    const int64_t* xb = x + (b * P + p) * N;
    const int8_t* gb = g + b * N;
    __shared__ __align__(16) int64_t xs[CJ];
    __shared__ __align__(16) int8_t gw[CI + CJ];
    const int t = threadIdx.x;
    int64_t acc[CR];
#pragma unroll
    for (int r = 0; r < CR; r++) acc[r] = 0;

    for (int64_t j0 = 0; j0 < N; j0 += CJ) {
        for (int u = t; u < CJ; u += CT) xs[u] = (j0 + u < N) ? xb[j0 + u] : 0;
        const int64_t base = i0 - j0 - CJ;
        for (int u = t; u < CI + CJ; u += CT) {
            int64_t idx = (base + u) % N;
            if (idx < 0) idx += N;
            gw[u] = gb[idx];
        }
        __syncthreads();
        const int8_t* gt = gw + CR * t + CJ;     // gt[rr - jl] = g[(i - j) mod N]
        int64_t hi = *reinterpret_cast<const int64_t*>(gt);
#pragma unroll 1
        for (int q = 0; q < CJ / 8; q++) {
            const int64_t lo = *reinterpret_cast<const int64_t*>(gt - 8 * q - 8);
            // w[8 + d] = gt[d - 8q] for d in [-8, 8)
            int32_t w[16];
#pragma unroll
            for (int d = 0; d < 8; d++) {
                w[d] = (int32_t)(int8_t)(lo >> (8 * d));
                w[8 + d] = (int32_t)(int8_t)(hi >> (8 * d));
            }
            int64_t xv[8];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                longlong2 v = *reinterpret_cast<const longlong2*>(&xs[8 * q + e]);
                xv[e] = v.x;
                xv[e + 1] = v.y;
            }
#pragma unroll
            for (int e = 0; e < 8; e++)
#pragma unroll
                for (int r = 0; r < CR; r++) acc[r] += xv[e] * (int64_t)w[8 + r - e];
            hi = lo;
        }
        __syncthreads();
    }
    int64_t* ob = out + (b * P + p) * N;
#pragma unroll
    for (int r = 0; r < CR; r++) {
        int64_t i = i0 + CR * t + r;
        if (i < N) ob[i] = acc[r];
    }
}

}  // namespace

namespace ne {

// The plain launches of the two kernels (argument checks are the caller's):
// planes whose bit is set in skip_mask are not computed and not written.
ne_status gemm_i64_launch(int32_t P, const int64_t* x, const int8_t* G, int64_t* out, int32_t rows, int32_t cols,
                          int32_t k, uint32_t skip_mask, cudaStream_t s) {
    if (rows == 0 || cols == 0) return NE_OK;
    if (k == 0) {
        for (int p = 0; p < P; p++)
            if (!(skip_mask & (1u << p)) &&
                cudaMemsetAsync(out + (int64_t)p * rows * cols, 0, (size_t)rows * cols * 8, s) != cudaSuccess)
                return check_launch("ne_gemm: zero fill");
        return NE_OK;
    }
    dim3 grid((cols + GBN - 1) / GBN, (rows + GBM - 1) / GBM, P);
    if (grid.y > 65535) return fail(NE_EINVAL, "ne_gemm: rows too large");
    k_gemm_i64<<<grid, 256, 0, s>>>(x, G, out, rows, cols, k, skip_mask);
    return check_launch("ne_gemm");
}

ne_status cconv_i64_launch(int32_t P, const int64_t* x, const int8_t* g, int64_t* out, int64_t batch, int64_t N,
                           uint32_t skip_mask, cudaStream_t s) {
    if (batch == 0 || N == 0) return NE_OK;
    if ((N + CI - 1) / CI > 2147483647LL) return fail(NE_EINVAL, "ne_cconv: N too large");
    for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
        int64_t nb = batch - b0 < 65535 ? batch - b0 : 65535;
        dim3 grid((unsigned)((N + CI - 1) / CI), P, (unsigned)nb);
        k_cconv_i64<<<grid, CT, 0, s>>>(x + b0 * P * N, g + b0 * N, out + b0 * P * N, P, N, skip_mask);
        ne_status st = check_launch("ne_cconv");
        if (st) return st;
    }
    return NE_OK;
}

}  // namespace ne
