// Throughput ceiling of the int8 tensor path on this GPU: every warp issues
// independent mma.sync.m16n8k32 s8 instructions on register operands, so the
// launch measures the instruction's peak rate, the denominator of the
// roofline fraction reported for the digit-plane kernels.
#include "ne_common.cuh"
#include "ne_mma.cuh"

namespace {

using namespace ne;

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

extern "C" ne_status ne_probe_mma_peak(int32_t iters, int64_t* ops, cudaStream_t s) {
    if (iters < 1 || !ops) return fail(NE_EINVAL, "ne_probe_mma_peak: bad arguments");
    const int blocks = sm_count() * 8, threads = 256;
    k_probe_mma<<<blocks, threads, 0, s>>>(iters);
    *ops = (int64_t)blocks * (threads / 32) * (int64_t)iters * kChains * (16LL * 8 * 32 * 2);
    return check_launch("ne_probe_mma_peak");
}
