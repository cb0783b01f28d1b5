// Measurement probes of the benchmark (not part of the library's ABI): the
// throughput ceilings the roofline fractions of the kernels are reported
// against.  First the int8 tensor path on this GPU: every warp issues
// independent mma.sync.m16n8k32 s8 instructions on register operands, so the
// launch measures the instruction's peak rate, the denominator of the
// roofline fraction reported for the digit-plane kernels.
#include <cuda_runtime.h>

#include "ne_mma.cuh"
#include "ne_probe.h"

namespace {

using namespace ne;

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

int32_t launched() { return cudaGetLastError() == cudaSuccess ? NE_PROBE_OK : NE_PROBE_ECUDA; }

constexpr int kChains = 8;   // independent accumulators per warp

__device__ int g_probe_sink;

__global__ void __launch_bounds__(256) k_probe_mma(int iters) {
    uint32_t a[4] = {threadIdx.x * 0x01010101u, threadIdx.x ^ 0x5a5a5a5au, threadIdx.x + 3u, threadIdx.x * 7u};
    const uint32_t b0 = threadIdx.x ^ 0x3c3c3c3cu, b1 = threadIdx.x + 11u;
    int d[kChains][4];
#pragma unroll
    for (int i = 0; i < kChains; i++) d[i][0] = d[i][1] = d[i][2] = d[i][3] = 0;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < kChains; i++) mma_s8(d[i], a, b0, b1);
    }
    int s = 0;
#pragma unroll
    for (int i = 0; i < kChains; i++) s += d[i][0] + d[i][1] + d[i][2] + d[i][3];
    if (s == 0x7fffffff) g_probe_sink = s;   // keeps the chains live
}

}  // namespace

extern "C" int32_t ne_probe_mma_peak(int32_t iters, int64_t* ops, cudaStream_t s) {
    if (iters < 1 || !ops) return NE_PROBE_EINVAL;
    const int blocks = sm_count() * 8, threads = 256;
    k_probe_mma<<<blocks, threads, 0, s>>>(iters);
    *ops = (int64_t)blocks * (threads / 32) * (int64_t)iters * kChains * (16LL * 8 * 32 * 2);
    return launched();
}

// The CUDA-core counterpart: dp4a (four int8 products into an int32) on
// register operands, eight independent accumulators per thread.
namespace {

__global__ void __launch_bounds__(256) k_probe_dp4a(int iters) {
    int d[8];
    const int b = (int)(threadIdx.x ^ 0x55u);
#pragma unroll
    for (int i = 0; i < 8; i++) d[i] = (int)(i * 0x10001u + threadIdx.x);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) d[i] = __dp4a(d[(i + 1) & 7], b, d[i]);
    }
    int s = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) s += d[i];
    if (s == 0x7fffffff) g_probe_sink = s;
}

}  // namespace

extern "C" int32_t ne_probe_dp4a_peak(int32_t iters, int64_t* ops, cudaStream_t s) {
    if (iters < 1 || !ops) return NE_PROBE_EINVAL;
    const int blocks = sm_count() * 8, threads = 256;
    k_probe_dp4a<<<blocks, threads, 0, s>>>(iters);
    *ops = (int64_t)blocks * threads * (int64_t)iters * 8 * 8;   // 8 dp4a x 8 int8 operations each
    return launched();
}

// Both int8 pipes at once: in every block the first mma_warps warps run the
// tensor chains of k_probe_mma and the remaining warps the dp4a chains of
// k_probe_dp4a, each for its own iteration count, so the ratio of the two
// pipes' work can be set to that of a kernel that splits its work between
// them.  The launch time is the ceiling of that instruction mix.
namespace {

__global__ void __launch_bounds__(512) k_probe_mixed(int iters_mma, int iters_dp4a, int mma_warps) {
    const int warp = threadIdx.x >> 5;
    int s = 0;
    if (warp < mma_warps) {
        uint32_t a[4] = {threadIdx.x * 0x01010101u, threadIdx.x ^ 0x5a5a5a5au, threadIdx.x + 3u, threadIdx.x * 7u};
        const uint32_t b0 = threadIdx.x ^ 0x3c3c3c3cu, b1 = threadIdx.x + 11u;
        int d[kChains][4];
#pragma unroll
        for (int i = 0; i < kChains; i++) d[i][0] = d[i][1] = d[i][2] = d[i][3] = 0;
        for (int it = 0; it < iters_mma; it++) {
#pragma unroll
            for (int i = 0; i < kChains; i++) mma_s8(d[i], a, b0, b1);
        }
#pragma unroll
        for (int i = 0; i < kChains; i++) s += d[i][0] + d[i][1] + d[i][2] + d[i][3];
    } else {
        int d[8];
        const int b = (int)(threadIdx.x ^ 0x55u);
#pragma unroll
        for (int i = 0; i < 8; i++) d[i] = (int)(i * 0x10001u + threadIdx.x);
        for (int it = 0; it < iters_dp4a; it++) {
#pragma unroll
            for (int i = 0; i < 8; i++) d[i] = __dp4a(d[(i + 1) & 7], b, d[i]);
        }
#pragma unroll
        for (int i = 0; i < 8; i++) s += d[i];
    }
    if (s == 0x7fffffff) g_probe_sink = s;
}

}  // namespace

extern "C" int32_t ne_probe_mixed_peak(int32_t iters_mma, int32_t iters_dp4a, int32_t mma_warps,
                                         int32_t dp4a_warps, int32_t blocks_per_sm, int64_t* ops,
                                         cudaStream_t s) {
    if (iters_mma < 0 || iters_dp4a < 0 || mma_warps < 0 || dp4a_warps < 0 || mma_warps + dp4a_warps < 1 ||
        mma_warps + dp4a_warps > 16 || blocks_per_sm < 1 || blocks_per_sm > 8 || !ops)
        return NE_PROBE_EINVAL;
    const int blocks = sm_count() * blocks_per_sm, threads = 32 * (mma_warps + dp4a_warps);
    k_probe_mixed<<<blocks, threads, 0, s>>>(iters_mma, iters_dp4a, mma_warps);
    *ops = (int64_t)blocks * ((int64_t)mma_warps * iters_mma * kChains * (16LL * 8 * 32 * 2) +
                              (int64_t)dp4a_warps * 32 * iters_dp4a * 8 * 8);
    return launched();
}

// The 32-bit integer multiply-add rate of the CUDA cores (IMAD, the unit the
// modular arithmetic of the number-theoretic transform is bound by):
// eight independent multiply-add chains per thread on register operands.
namespace {

__global__ void __launch_bounds__(256) k_probe_imad(int iters) {
    uint32_t d[8];
    const uint32_t b = threadIdx.x * 2654435761u + 1u, c = threadIdx.x ^ 0x9e3779b9u;
#pragma unroll
    for (int i = 0; i < 8; i++) d[i] = i * 0x01000193u + threadIdx.x;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) d[i] = d[i] * b + c;
    }
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) s ^= d[i];
    if (s == 0x7fffffffu) g_probe_sink = (int)s;
}

}  // namespace

extern "C" int32_t ne_probe_imad_peak(int32_t iters, int64_t* ops, cudaStream_t s) {
    if (iters < 1 || !ops) return NE_PROBE_EINVAL;
    const int blocks = sm_count() * 8, threads = 256;
    k_probe_imad<<<blocks, threads, 0, s>>>(iters);
    *ops = (int64_t)blocks * threads * (int64_t)iters * 8;   // 32-bit multiply-adds
    return launched();
}
