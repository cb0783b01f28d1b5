// Batched circular convolution on the int8 tensor path straight from the raw
// int32 streams: Eq. 16 and the digit split are computed while each tile
// loads its window, so the entangled words never reach memory (the one-launch
// form of Eq. 10 with Eq. 17-20 / Eq. 24 fused into the epilogue).
#include "ne_cconv_launch.cuh"

using namespace ne;
using namespace ne::cconv_launch;

extern "C" ne_status ne_cconv_entangled(ne_params p, ne_digits dg, const int32_t* c, const int8_t* g, int64_t* out,
                                        uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t N, int32_t fuse,
                                        int32_t r, int32_t plain, ne_faults faults, int32_t* status,
                                        cudaStream_t s) {
    ne_status st = common_args(p, dg, batch, N, fuse, r, faults, "ne_cconv_entangled");
    if (st) return st;
    if (plain && fuse != NE_FUSE_NONE) return fail(NE_EINVAL, "ne_cconv_entangled: the plain operation has no extraction");
    // the digit split in 32 bits needs the plan of a known input range: the
    // digit set of (l, lo, hi) itself (plain: one digit of values in [-128, 127])
    uint32_t off = 0;
    int byte_of[4] = {0, 0, 0, 0};
    if (plain && dg.S == 1 && dg.shift[0] == 0 && dg.lo <= dg.hi && dg.lo >= -128 && dg.hi <= 127) {
        off = 0x80u;                         // one digit: the raw int8-valued streams themselves
    } else {
        // the plan of (l, lo, hi); for the plain operation with 0 in [lo, hi] a
        // raw value is the word of Eq. 16 with a zero predecessor, so its digits
        // are in the plan too (the plain operation on the entangled digit set)
        ne_digits ref;
        FastPlan F;
        bool planned = dg.lo <= dg.hi && dg.l == p.l && ne_plan_digits(dg.l, dg.lo, dg.hi, &ref) == NE_OK &&
                       ref.S == dg.S && (!plain || (dg.lo <= 0 && 0 <= dg.hi));
        for (int i = 0; planned && i < dg.S; i++) planned = ref.shift[i] == dg.shift[i];
        if (!planned || !make_fast_plan(dg, p.l, &F))
            return fail(NE_EINVAL, "ne_cconv_entangled: dg must be the plan of (l, lo, hi) with words of at most "
                                   "4 digits (plain: or one digit of values in [-128, 127]); otherwise entangle "
                                   "with ne_entangle_digits");
        off = F.off;
        for (int i = 0; i < 4; i++) byte_of[i] = F.byte_of[i];
    }
    unsigned long long* nf = reinterpret_cast<unsigned long long*>(nflag);
    if (nf && cudaMemsetAsync(nf, 0, sizeof(*nf), s) != cudaSuccess) return check_launch("ne_cconv_entangled: reset");
    if (batch == 0) return NE_OK;
    if (!c || !g || !out) return fail(NE_EINVAL, "ne_cconv_entangled: null pointer");
    if (!aligned(c, 4) || !aligned(out, 8)) return fail(NE_EINVAL, "ne_cconv_entangled: c, out must be aligned");
    CconvArgs a;
    fill_args(a, p, dg, g, out, flags, nf, N, fuse, r, faults);
    a.craw = c;
    a.status = status;
    a.raw_off = off;
    a.raw_lo = dg.lo;
    a.raw_hi = dg.hi;
    a.raw_plain = plain ? 1 : 0;
    for (int i = 0; i < 4; i++) a.raw_byte[i] = byte_of[i];
    return dispatch<cconv::LD_RAW>(a, batch, s);
}
