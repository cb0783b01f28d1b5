// The operation of Eq. 10 on the M entangled streams in the form of the
// problem statement (Sec. II, Eq. 2 and Eq. 10): entangled words in, the
// operation with the shared operator, and optionally the extraction and check
// (Eq. 17-20, Eq. 24) or the recovery of a lost stream (Prop. 3) behind it.
//
//   NE_MODE_I64      the int64 multiply-add kernels on the CUDA cores: the
//                    operation writes delta into out, the fault hook and the
//                    extraction then run in place on out (HBM passes; the
//                    operation itself is ALU-bound)
//   NE_MODE_S8SLICE  the int8 tensor path: the tiles split every entangled
//                    word into the balanced base-256 digits of the plan dg
//                    while loading, multiply each digit slice exactly (int32
//                    accumulation), recombine in int64 and run the fault hook
//                    and the extraction in the epilogue; delta never reaches
//                    memory
#include "ne_common.cuh"

namespace {

using namespace ne;

ne_status common(const char* who, const ne_params& p, int32_t mode, int32_t fuse, int32_t r, uint32_t drop_mask,
                 const ne_faults& faults, uint32_t* skip) {
    if (fuse < NE_FUSE_NONE || fuse > NE_FUSE_RECOVER) return fail(NE_EINVAL, "%s: fuse=%d", who, fuse);
    if (mode != NE_MODE_I64 && mode != NE_MODE_S8SLICE) return fail(NE_EINVAL, "%s: mode=%d", who, mode);
    ne_status st;
    if (fuse == NE_FUSE_NONE && mode == NE_MODE_I64) {
        // the operation alone: any number of planes (the checksum comparator
        // runs M + 1, the plain operation the raw streams), l unused
        if (p.M < 1 || p.M > 32) return fail(NE_EINVAL, "%s: %d planes (1..32)", who, p.M);
    } else if ((st = validate_params(p))) {
        return st;
    }
    if ((st = validate_faults(faults, who))) return st;
    if (fuse != NE_FUSE_NONE && (r < 0 || r >= p.M)) return fail(NE_EINVAL, "%s: r=%d", who, r);
    if (p.M < 32 && (drop_mask >> p.M) != 0) return fail(NE_EINVAL, "%s: drop_mask names a plane >= M", who);
    const uint32_t lost = fuse == NE_FUSE_RECOVER ? (1u << r) : 0u;
    if (fuse == NE_FUSE_EXTRACT_CHECK && drop_mask)
        return fail(NE_EINVAL, "%s: the check reads every stream; drop streams with NE_FUSE_RECOVER", who);
    if (fuse == NE_FUSE_RECOVER && (drop_mask & ~lost))
        return fail(NE_EINVAL, "%s: recovery rebuilds one lost stream, r", who);
    if (mode == NE_MODE_S8SLICE && fuse == NE_FUSE_NONE && drop_mask)
        return fail(NE_EINVAL, "%s: the tensor path drops a stream only under NE_FUSE_RECOVER", who);
    *skip = drop_mask | lost;
    return NE_OK;
}

}  // namespace

extern "C" ne_status ne_gemm(ne_params p, const int64_t* eps, const int8_t* G, int64_t* out, uint32_t* flags,
                             uint64_t* nflag, int32_t rows, int32_t cols, int32_t k, int32_t mode, ne_digits dg,
                             int32_t fuse, int32_t r, uint32_t drop_mask, ne_faults faults, int32_t* status,
                             cudaStream_t s) {
    uint32_t skip = 0;
    ne_status st = common("ne_gemm", p, mode, fuse, r, drop_mask, faults, &skip);
    if (st) return st;
    if (mode == NE_MODE_S8SLICE)
        return gemm_s8slice(p, dg, eps, G, out, flags, nflag, rows, cols, k, fuse, r, faults, status, s);
    if (rows < 0 || cols < 0 || k < 0) return fail(NE_EINVAL, "ne_gemm: negative size");
    unsigned long long* nf = reinterpret_cast<unsigned long long*>(nflag);
    if (nf && cudaMemsetAsync(nf, 0, sizeof(*nf), s) != cudaSuccess) return check_launch("ne_gemm: reset count");
    if (rows == 0 || cols == 0) return NE_OK;
    if (!eps || !G || !out) return fail(NE_EINVAL, "ne_gemm: null pointer");
    if ((st = gemm_i64_launch(p.M, eps, G, out, rows, cols, k, skip, s))) return st;
    const int64_t n = (int64_t)rows * cols;
    if ((st = faults_launch(out, p.M, 1, n, faults, skip, s))) return st;
    if (fuse == NE_FUSE_NONE) return NE_OK;
    return extract_launch(p, out, out, 1, n, r, fuse == NE_FUSE_EXTRACT_CHECK && (flags || nf), flags, nf, s);
}

extern "C" ne_status ne_cconv(ne_params p, const int64_t* eps, const int8_t* g, int64_t* out, uint32_t* flags,
                              uint64_t* nflag, int64_t batch, int64_t N, int32_t mode, ne_digits dg, int32_t fuse,
                              int32_t r, uint32_t drop_mask, ne_faults faults, int32_t* status, cudaStream_t s) {
    uint32_t skip = 0;
    ne_status st = common("ne_cconv", p, mode, fuse, r, drop_mask, faults, &skip);
    if (st) return st;
    if (mode == NE_MODE_S8SLICE)
        return cconv_s8slice(p, dg, eps, g, out, flags, nflag, batch, N, fuse, r, faults, status, s);
    if (batch < 0 || N < 0) return fail(NE_EINVAL, "ne_cconv: negative size");
    unsigned long long* nf = reinterpret_cast<unsigned long long*>(nflag);
    if (nf && cudaMemsetAsync(nf, 0, sizeof(*nf), s) != cudaSuccess) return check_launch("ne_cconv: reset count");
    if (batch == 0 || N == 0) return NE_OK;
    if (!eps || !g || !out) return fail(NE_EINVAL, "ne_cconv: null pointer");
    if ((st = cconv_i64_launch(p.M, eps, g, out, batch, N, skip, s))) return st;
    if ((st = faults_launch(out, p.M, batch, N, faults, skip, s))) return st;
    if (fuse == NE_FUSE_NONE) return NE_OK;
    return extract_launch(p, out, out, batch, N, r, fuse == NE_FUSE_EXTRACT_CHECK && (flags || nf), flags, nf, s);
}
