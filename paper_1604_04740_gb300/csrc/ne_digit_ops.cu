// Tensor-path (mma.sync s8) operations on digit planes.
#include "ne_common.cuh"

using namespace ne;

extern "C" ne_status ne_gemm_digits(ne_params p, ne_digits dg, const int8_t* planes, const int8_t* G, int64_t* out,
                                    uint32_t* flags, uint64_t* nflag, int32_t rows, int32_t cols, int32_t k,
                                    int32_t fuse, int32_t r, cudaStream_t s) {
    return fail(NE_EINVAL, "ne_gemm_digits: not built yet");
}

extern "C" ne_status ne_cconv_digits(ne_params p, ne_digits dg, const int8_t* planes, const int8_t* g, int64_t* out,
                                     uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t N, int32_t fuse,
                                     int32_t r, cudaStream_t s) {
    return fail(NE_EINVAL, "ne_cconv_digits: not built yet");
}
