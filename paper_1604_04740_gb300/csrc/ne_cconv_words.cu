// ne_cconv's S8SLICE mode: the tensor-path tiles split the entangled int64
// words themselves into their digit bytes while loading (Eq. 10 on the words
// of Eq. 16, with Eq. 17-20 / Eq. 24 fused into the epilogue).
#include "ne_cconv_launch.cuh"

using namespace ne;
using namespace ne::cconv_launch;

namespace ne {

// ne_cconv's S8SLICE mode: the tiles split the entangled words themselves
ne_status cconv_s8slice(ne_params p, ne_digits dg, const int64_t* words, const int8_t* g, int64_t* out,
                        uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t N, int32_t fuse, int32_t r,
                        const ne_faults& faults, int32_t* status, cudaStream_t s) {
    ne_status st = common_args(p, dg, batch, N, fuse, r, faults, "ne_cconv (S8SLICE)");
    if (st) return st;
    unsigned long long* nf = reinterpret_cast<unsigned long long*>(nflag);
    if (nf && cudaMemsetAsync(nf, 0, sizeof(*nf), s) != cudaSuccess) return check_launch("ne_cconv: reset");
    if (batch == 0) return NE_OK;
    if (!words || !g || !out) return fail(NE_EINVAL, "ne_cconv: null pointer");
    if (!aligned(words, 8) || !aligned(out, 8)) return fail(NE_EINVAL, "ne_cconv: eps and out must be 8-byte aligned");
    CconvArgs a;
    fill_args(a, p, dg, g, out, flags, nf, N, fuse, r, faults);
    uint64_t stored = 0;
    for (int i = 0; i < dg.S; i++) stored |= 0xffull << dg.shift[i];
    a.cwords = words;
    a.w_nsmask = ~stored;
    a.w_nswant = 0x8080808080808080ull & ~stored;
    a.status = status;
    return dispatch<cconv::LD_WORDS>(a, batch, s);
}

}  // namespace ne
