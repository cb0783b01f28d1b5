// Batched circular convolution on the int8 tensor path from digit planes
// already in memory (the circular-convolution member of Eq. 2, applied per
// Eq. 10, with the extraction and check of Eq. 17-20 / Eq. 24 fused into the
// epilogue), and the process-wide tensor / dp4a split of its tiles.
#include "ne_cconv_launch.cuh"

using namespace ne;
using namespace ne::cconv_launch;

namespace ne {
namespace cconv_launch {
int g_split = -1;
}  // namespace cconv_launch
}  // namespace ne

extern "C" ne_status ne_cconv_digits(ne_params p, ne_digits dg, const int8_t* planes, const int8_t* g, int64_t* out,
                                     uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t N, int32_t fuse,
                                     int32_t r, ne_faults faults, cudaStream_t s) {
    ne_status st = common_args(p, dg, batch, N, fuse, r, faults, "ne_cconv_digits");
    if (st) return st;
    unsigned long long* nf = reinterpret_cast<unsigned long long*>(nflag);
    if (nf && cudaMemsetAsync(nf, 0, sizeof(*nf), s) != cudaSuccess) return check_launch("ne_cconv_digits: reset");
    if (batch == 0) return NE_OK;
    if (!planes || !g || !out) return fail(NE_EINVAL, "ne_cconv_digits: null pointer");
    if (!aligned(out, 8)) return fail(NE_EINVAL, "ne_cconv_digits: out must be 8-byte aligned");
    CconvArgs a;
    fill_args(a, p, dg, g, out, flags, nf, N, fuse, r, faults);
    a.planes = planes;
    return dispatch<cconv::LD_PLANES>(a, batch, s);
}

extern "C" ne_status ne_set_cconv_split(int32_t variant) {
    static const int ok[] = {-1, 0, 23, 24, 34, 42, 43, 44, 443, 444};
    for (int v : ok)
        if (v == variant) {
            g_split = variant;
            return NE_OK;
        }
    return fail(NE_EINVAL, "ne_set_cconv_split: unknown variant %d", variant);
}
