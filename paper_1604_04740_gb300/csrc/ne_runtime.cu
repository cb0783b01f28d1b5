// Serving runtime support: the host->device copies of one micro-batch issued
// from native code (one cudaMemcpyAsync per request region).
#include "ne_common.cuh"

using namespace ne;

extern "C" ne_status ne_copy_regions_h2d(void* dst_base, const void* src_base, const int64_t* dst_off,
                                         const int64_t* src_off, const int64_t* nbytes, int64_t count,
                                         cudaStream_t s) {
    if (count < 0 || (count > 0 && (!dst_base || !src_base || !dst_off || !src_off || !nbytes)))
        return fail(NE_EINVAL, "ne_copy_regions_h2d: bad arguments");
    char* dst = static_cast<char*>(dst_base);
    const char* src = static_cast<const char*>(src_base);
    for (int64_t i = 0; i < count; i++) {
        if (nbytes[i] < 0 || dst_off[i] < 0 || src_off[i] < 0) return fail(NE_EINVAL, "ne_copy_regions_h2d: region %lld", (long long)i);
        if (nbytes[i] == 0) continue;
        const cudaError_t e = cudaMemcpyAsync(dst + dst_off[i], src + src_off[i], (size_t)nbytes[i],
                                              cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail(NE_ECUDA, "ne_copy_regions_h2d: %s", cudaGetErrorString(e));
    }
    return NE_OK;
}
