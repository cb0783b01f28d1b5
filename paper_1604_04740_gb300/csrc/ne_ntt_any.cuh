// Jobs of the general-length transform convolution (ne_ntt_any.cu), shared
// with the ragged batch runner.
#pragma once

#include "ne_common.cuh"

namespace ne {

// One group: M streams of length N convolved with one filter of length N.
struct NJob {
    int64_t c_off;               // int32 element offset of the streams [M][N]
    int64_t g_off;               // byte offset of the filter [N]
    int64_t out_off;             // int64 element offset of the outputs [M][N]
    int64_t flag_off;            // uint32 word offset of the check bitmap
    int64_t ws_off;              // uint32 element offset of the workspace [M + 1][2][L]
    int64_t fault_begin, fault_end;   // the job's range in the (position-sorted) fault lists
    int64_t fault_key0;          // the list's position of the job's output 0 (0 in a batch)
    int32_t M, N, L, logL, l, r, fuse, plain, lo, hi;
    uint32_t gscale[2];          // 2^64 / L mod each prime: the filter transform's Montgomery scale
};

// Either a table of jobs or njobs copies of tmpl with the offsets advanced by
// the strides.
struct NJobs {
    const NJob* table;
    NJob tmpl;
    int64_t c_stride, g_stride, out_stride, flag_stride, ws_stride, fault_key_stride;
    int64_t njobs;
};

struct NttAnyArgs {
    NJobs jobs;
    const int32_t* c;
    const int8_t* g;
    int64_t* out;
    uint32_t* flags;
    unsigned long long* nflag;
    int flags_atomic;            // bitmap pre-zeroed: OR the set bits in
    int32_t* status;
    uint32_t* ws;
    const int64_t* fault_pos;    // fault hook (or null)
    const int32_t* fault_stream;
    const int32_t* fault_bit;
    uint32_t crt_inv, crt_invq;  // P1^-1 mod P2 and its Shoup quotient (set by ntt_any_run)
};

// transform length for N (N itself when a power of two, else the next power
// of two >= 2N - 1); *logL its logarithm
int ntt_any_length(int64_t N, int* logL);
// whether outputs of N-term convolutions of words from inputs with |c| <= cmax_abs
// stay inside the two-prime range
bool ntt_any_exact(int M, int l, int64_t N, int32_t cmax_abs, bool plain);
// per-job constants (gscale) once L is set
void ntt_any_job_constants(NJob& j);
// twiddle tables (once per device; synchronises s the first time)
ne_status ntt_any_init_tables(cudaStream_t s);
// the launches for a set of jobs: min_logL .. max_logL and max_M bound every
// job's L and M
ne_status ntt_any_run(NttAnyArgs& a, int min_logL, int max_logL, int max_M, int64_t max_units_load,
                      cudaStream_t s);

}  // namespace ne
