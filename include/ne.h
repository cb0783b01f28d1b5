/*
 * ne.h -- C ABI of the GB300 (sm_103a) numerical-entanglement library.
 *
 * Numerical entanglement (Anam & Andreopoulos, "Reliable Linear, Sesquilinear
 * and Bijective Operations on Integer Data Streams via Numerical
 * Entanglement") makes a linear/sesquilinear integer operation on M >= 3
 * streams fault tolerant without extra streams:
 *
 *   entangle   eps_m = c_m + 2^l c_{(m-1) mod M}                (Eq. 7, Eq. 16)
 *   operate    delta_m = eps_m op g, on every stream unchanged    (Eq. 10)
 *   extract    all M outputs from any M-1 of the delta_m        (Eq. 17-20)
 *   check      recreate the unused delta_r and compare           (Eq. 24)
 *   recover    a lost stream r is simply the unused one          (Prop. 3)
 *
 * All arithmetic is exact integer arithmetic on w = 64-bit words.
 *
 * Conventions for every entry point
 *  - Pointers named with a device type are DEVICE pointers; the caller owns
 *    all memory.  Only ne_*_host entry points take host pointers.
 *  - Calls are asynchronous on the CUDA stream `s` (0 = legacy default
 *    stream) and return a host-side status: NE_EINVAL / NE_ERANGE for
 *    arguments rejected before any launch, NE_ECUDA if a launch failed.
 *    Conditions found on the device are written to the caller's `status`
 *    word (device int32, nullable) and are visible after the stream syncs.
 *  - Stream planes are stored as [batch][M][n] (row-major): group b,
 *    stream m, position i is at index (b*M + m)*n + i.
 *  - Check results are bitmaps of uint32 words: position i of group b is bit
 *    (i % 32) of word b*ceil(n/32) + i/32 (bits past n in the last word are
 *    0).  When a count pointer `nflag` (device uint64) is given, the call
 *    first sets it to 0 and then adds the number of flagged positions.
 *  - No entry point allocates device memory.  ne_last_error() returns a
 *    message for the last failed call on the calling host thread.
 */
#ifndef NE_H
#define NE_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NE_OK = 0,
    NE_EINVAL = 1,    /* invalid argument (null pointer, size, alignment, M < 3, ...)       */
    NE_ERANGE = 2,    /* parameters violate Eq. 13, or data outside the planned digit range */
    NE_ECUDA = 3,     /* a CUDA runtime call or launch failed                               */
    NE_ETIMEOUT = 4,  /* a bounded device-side wait gave up                                 */
    NE_ENOMEM = 5     /* a caller-provided workspace is too small                           */
} ne_status;

/* The method's parameters: M streams (3 <= M <= 32), shift l, word width w
 * (always 64 here).  Valid when (M-1) l < w, i.e. Eq. 13 holds with k >= 1. */
typedef struct {
    int32_t M;
    int32_t l;
    int32_t w;
} ne_params;

/* Balanced base-256 digit planes of entangled words.  A word x is stored as
 * the S planes sigma_0..sigma_{S-1} (int8) with
 *     x = sum_s sigma_s * 2^shift[s],   shift[s] a multiple of 8, ascending,
 * where the digits not listed are identically zero for the inputs the plan
 * was made for (see ne_plan_digits).  Plane layout: [batch][M][S][n].
 * l, lo, hi record the shift and the stream-value range [lo, hi] the plan
 * was derived for (lo > hi: unknown); ne_entangle_digits uses them to check
 * its inputs instead of every digit. */
#define NE_MAX_DIGITS 8
typedef struct {
    int32_t S;
    int32_t shift[NE_MAX_DIGITS];
    int32_t l;
    int32_t lo;
    int32_t hi;
} ne_digits;

/* Transient faults injected into the words delta of a fused operation after
 * the operation and before its extraction -- the fault model of Sec. I: a
 * fault corrupts one stream's result of the operation.  Entry f XORs bit
 * (bit[f] mod 64) into delta_{stream[f]} at the flat output position pos[f]
 * of the call: group * N + i for the batched convolutions, i * cols + j for
 * the matrix product.  pos must be sorted ascending (an entry out of order may
 * be missed).  An entry whose stream lies outside [0, M) hits nothing; under
 * NE_FUSE_RECOVER an entry on the lost stream hits nothing (that stream is
 * never computed).  The three arrays are device arrays of count entries,
 * owned by the caller and only read; count = 0 injects nothing and the
 * pointers may then be null. */
typedef struct {
    const int64_t* pos;
    const int32_t* stream;
    const int32_t* bit;
    int64_t count;
} ne_faults;

/* l-selection policies for ne_choose_l */
#define NE_L_PAPER    0  /* max (M-2)l+k s.t. (M-1)l+k <= w, k <= l; ties -> larger (M-1)l+k */
#define NE_L_SMALLEST 1  /* smallest l with an admissible k whose Eq. 14 range covers the bound */
#define NE_L_BYTE     2  /* as NE_L_SMALLEST, l restricted to multiples of 8 */

/* fused epilogues of the digit-plane operations */
#define NE_FUSE_NONE          0  /* write delta_m (int64) for every computed stream            */
#define NE_FUSE_EXTRACT_CHECK 1  /* write d_hat (Eq. 17-20) and the Eq. 24 check flags        */
#define NE_FUSE_RECOVER       2  /* stream r is lost: skip it, write d_hat from the other M-1 */

/* ------------------------------------------------------------------------ */
/* Planning (host only, no device work)                                      */
/* ------------------------------------------------------------------------ */

/* Choose the shift l and the bookkeeping k of Sec. III-C: Eq. 13
 * ((M-1)l + k <= w) with k <= l, and the Eq. 14 output range
 * 2^((M-3)l+k) (2^(l-1)-1) >= out_bound for the bound-driven policies.
 * Returns NE_ERANGE if no (l, k) exists.  l, k: host out-pointers. */
ne_status ne_choose_l(int32_t M, int32_t w, int64_t out_bound, int32_t policy,
                      int32_t* l, int32_t* k);

/* Which balanced base-256 digits of eps = a + 2^l b can be non-zero when the
 * stream values a, b lie in [cmin, cmax] (the entanglement of Eq. 16).
 * Fills *dg with the digit positions that occur.  A range of at most 4096
 * values is enumerated exactly; a wider range lists every digit up to the
 * width of |eps| <= max|c| (2^l + 1).  NE_ERANGE if more than NE_MAX_DIGITS
 * digits would be needed. */
ne_status ne_plan_digits(int32_t l, int32_t cmin, int32_t cmax, ne_digits* dg);

/* ------------------------------------------------------------------------ */
/* Entanglement (Eq. 7 for M = 3; Eq. 15-16 for general M)                   */
/* ------------------------------------------------------------------------ */

/* eps[b][m][i] = c[b][m][i] + 2^l c[b][(m-1) mod M][i].
 * c: int32 [batch][M][n], eps: int64 [batch][M][n] (may not alias c). */
ne_status ne_entangle(ne_params p, const int32_t* c, int64_t* eps,
                      int64_t batch, int64_t n, cudaStream_t s);

/* Same entangled words, stored as digit planes: planes is int8
 * [batch][M][dg.S][n].  A word with a non-zero digit outside dg, or a
 * residue beyond the top digit, sets *status = NE_ERANGE (status nullable;
 * the call does not reset it). */
ne_status ne_entangle_digits(ne_params p, ne_digits dg, const int32_t* c, int8_t* planes,
                             int64_t batch, int64_t n, int32_t* status, cudaStream_t s);

/* Digit planes of the raw streams (no entanglement) with the digit set of an
 * entangled plan: planes is int8 [batch][M][dg.S][n] holding c itself, the
 * operand of the plain operation in the layout and digit count of the
 * entangled one.  dg must be the plan of (p.l, lo, hi) with lo <= 0 <= hi (a
 * raw value is then a word of Eq. 16 with a zero predecessor) and at most 4
 * digits, or one digit at shift 0 with [lo, hi] inside [-128, 127] (the
 * fewest digits of int8-valued streams); M <= 5; n a multiple of 8, c
 * 16-byte and planes 8-byte aligned.
 * An input outside [lo, hi] sets *status = NE_ERANGE (nullable). */
ne_status ne_split_digits_raw(ne_params p, ne_digits dg, const int32_t* c, int8_t* planes,
                              int64_t batch, int64_t n, int32_t* status, cudaStream_t s);

/* Digit planes of arbitrary int64 words (entangled words produced elsewhere,
 * or the raw and checksum streams of the ABFT comparator): x is int64
 * [batch][P][n], planes is int8 [batch][P][dg.S][n].  Out-of-plan words set
 * *status = NE_ERANGE as for ne_entangle_digits. */
ne_status ne_split_digits(ne_digits dg, const int64_t* x, int8_t* planes, int64_t batch, int32_t P,
                          int64_t n, int32_t* status, cudaStream_t s);

/* ------------------------------------------------------------------------ */
/* The LSB operation on each stream (Eq. 10), unaware of the entanglement    */
/* ------------------------------------------------------------------------ */

/* The operation of Eq. 10 in the form of the problem statement (Sec. II,
 * Eq. 2): the M entangled streams eps_m (int64 words of Eq. 16) times the
 * shared operator, each stream unchanged by the entanglement, with the
 * extraction and check or the recovery behind it.
 *  mode NE_MODE_I64:     int64 multiply-adds on the CUDA cores (exact while
 *        every partial sum fits 64 bits).  The operation writes delta into
 *        out; the fault hook and then the extraction (Eq. 17-20, with the
 *        check of Eq. 24) run in place on out, in the same call and stream.
 *        dg and status are not used.
 *  mode NE_MODE_S8SLICE: the int8 tensor path.  The kernel's loader splits
 *        every word into the balanced base-256 digits of the plan dg
 *        (ne_plan_digits of the range the streams were entangled from), each
 *        digit slice is multiplied exactly (int32 accumulation over chunks of
 *        at most 2^31 / 2^14 terms) and recombined in int64, and the fault hook
 *        and the extraction/check run in the epilogue: delta never reaches
 *        memory.  A word with a non-zero digit outside dg sets
 *        *status = NE_ERANGE (device int32, nullable).
 *  fuse: NE_FUSE_NONE (out = delta of every computed plane), NE_FUSE_EXTRACT_CHECK
 *        (out = d_hat, flags/nflag the Eq. 24 check of stream r, flags
 *        nullable) or NE_FUSE_RECOVER (stream r is lost: never read nor
 *        computed; out = d_hat from the other M-1, Prop. 3).
 *  drop_mask: planes that are not computed (a fail-stopped core): with
 *        NE_FUSE_NONE and NE_MODE_I64 any set of planes (their outputs are
 *        not written); with NE_FUSE_RECOVER 0 or the bit of r; otherwise 0.
 *  faults: transient faults XORed into delta before the extraction (ne_faults).
 * With NE_FUSE_NONE and NE_MODE_I64, p.M is just the number of planes (1..32,
 * l unused): the plain operation on raw streams widened to int64, or the M+1
 * planes of the checksum comparator.  Otherwise p must satisfy Eq. 13. */
#define NE_MODE_I64     0
#define NE_MODE_S8SLICE 1

/* Matrix product (the GEMM experiment of Sec. V): out[m] = eps[m] * G.
 * eps: int64 [M][rows][k]; G: int8 [k][cols]; out: int64 [M][rows][cols]
 * (must not overlap eps); positions i * cols + j for flags [ceil(rows cols /
 * 32)] and faults.  NE_MODE_S8SLICE: k <= 131056, M * dg.S <= 16. */
ne_status ne_gemm(ne_params p, const int64_t* eps, const int8_t* G, int64_t* out, uint32_t* flags, uint64_t* nflag,
                  int32_t rows, int32_t cols, int32_t k, int32_t mode, ne_digits dg, int32_t fuse, int32_t r,
                  uint32_t drop_mask, ne_faults faults, int32_t* status, cudaStream_t s);

/* Batched circular convolution (Eq. 2): out[b][m][i] = sum_j eps[b][m][j]
 * g[b][(i - j) mod N].  eps, out: int64 [batch][M][N] (no overlap); g: int8
 * [batch][N]; flags [batch][ceil(N/32)]; fault positions b * N + i.
 * NE_MODE_S8SLICE: N a multiple of 64 in [64, 65536], M * dg.S <= 16, eps
 * 16-byte aligned. */
ne_status ne_cconv(ne_params p, const int64_t* eps, const int8_t* g, int64_t* out, uint32_t* flags, uint64_t* nflag,
                   int64_t batch, int64_t N, int32_t mode, ne_digits dg, int32_t fuse, int32_t r,
                   uint32_t drop_mask, ne_faults faults, int32_t* status, cudaStream_t s);

/* The product on the int8 tensor path from digit planes already split (by
 * ne_entangle_digits, which writes 2 bytes per word of int8-valued streams
 * instead of 8): every digit plane is multiplied
 * by G with int32 accumulation over K chunks of at most 2^31 / 2^14 terms
 * (no int32 overflow for int8 x int8), and the digits are recombined exactly
 * in int64.  planes: int8 [M][dg.S][rows][k]; G: int8 [k][cols].
 *  fuse = NE_FUSE_NONE:          out = delta, int64 [M][rows][cols].
 *  fuse = NE_FUSE_EXTRACT_CHECK: out = d_hat of Eq. 17-20 using every stream
 *        but r, and flags/nflag receive the Eq. 24 check of stream r
 *        (positions flattened as i*cols + j; flags nullable).
 *  fuse = NE_FUSE_RECOVER:       stream r is not computed at all; out = d_hat
 *        from the other M-1 streams (Prop. 3); flags ignored.
 * faults: transient faults XORed into delta before the epilogue (see
 * ne_faults; positions i * cols + j).
 * rows, cols, k >= 0, k <= 131056; any sizes (a k that is not a multiple of
 * 16, or cols not of 4, take element-wise loads). */
ne_status ne_gemm_digits(ne_params p, ne_digits dg, const int8_t* planes, const int8_t* G,
                         int64_t* out, uint32_t* flags, uint64_t* nflag,
                         int32_t rows, int32_t cols, int32_t k,
                         int32_t fuse, int32_t r, ne_faults faults, cudaStream_t s);

/* The convolution on the int8 tensor path from digit planes already split:
 * the circulant of g is tiled
 * into Toeplitz blocks built in shared memory and multiplied with the digit
 * planes (int32 accumulation, exact int64 recombination), with the same
 * fused epilogues and fault hook as ne_gemm_digits (fault positions
 * group * N + i).  planes: int8 [batch][M][dg.S][N];
 * g: int8 [batch][N]; out: int64 [batch][M][N]; flags: [batch][N/32].
 * N a multiple of 64 with 64 <= N <= 4096. */
ne_status ne_cconv_digits(ne_params p, ne_digits dg, const int8_t* planes, const int8_t* g,
                          int64_t* out, uint32_t* flags, uint64_t* nflag,
                          int64_t batch, int64_t N, int32_t fuse, int32_t r, ne_faults faults,
                          cudaStream_t s);

/* ne_cconv_digits fused with the entanglement in front: the tiles read the
 * raw streams c (int32 [batch][M][N], 16-byte aligned) and form the words of
 * Eq. 16 and their digits while loading, so one launch goes from the raw
 * streams to the extracted outputs.  dg must be the digit plan of its
 * (l, lo, hi) with words of at most 4 digits (ne_plan_digits); every input
 * outside [lo, hi] sets *status = NE_ERANGE (device int32, nullable); under
 * NE_FUSE_RECOVER the lost stream's inputs are still read (as the
 * predecessor in the next stream's words) and range-checked.
 * plain = 1: the plain operation on the raw streams (NE_FUSE_NONE), with dg
 * either one digit at shift 0 and a range inside [-128, 127], or the plan of
 * (l, lo, hi) with lo <= 0 <= hi (the raw values split into the entangled
 * words' digit set: the same kernel doing the same int8 work).  Other
 * arguments as for ne_cconv_digits. */
ne_status ne_cconv_entangled(ne_params p, ne_digits dg, const int32_t* c, const int8_t* g, int64_t* out,
                             uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t N, int32_t fuse,
                             int32_t r, int32_t plain, ne_faults faults, int32_t* status, cudaStream_t s);

/* Linear convolution of long streams with a short kernel, the convolution of
 * the paper's second experiment (Sec. V; long streams processed as
 * overlapping blocks of about the kernel's length, Sec. IV-A), fused from the
 * raw streams to the extracted outputs in one launch on the int8 tensor path:
 *     out[b][m][i] = sum_{t<K} g[b][t] w[b][m][i - t],  0 <= i < n + K - 1,
 * with w the words of Eq. 16 (plain = 1: the raw values c) and w = 0 outside
 * [0, n) -- the full linear convolution of every entangled stream, then the
 * epilogue of ne_cconv_digits (fuse, r, flags/nflag, faults at positions
 * b * (n + K - 1) + i).  Every tile of 1024 outputs reads the K + 1023 inputs
 * it reaches (the overlap of overlap-save is the kernel's K - 1) and sums
 * only the kernel's Toeplitz blocks.  c: int32 [batch][M][n], 16-byte
 * aligned; g: int8 [batch][K]; out: int64 [batch][M][n + K - 1]; flags:
 * uint32 [batch][ceil((n + K - 1) / 32)].  1 <= K <= 131071, n + K - 1 <=
 * 2^30, M * dg.S <= 16.  dg and plain as for ne_cconv_entangled (an input
 * outside [lo, hi] sets *status = NE_ERANGE, the lost stream's included under
 * NE_FUSE_RECOVER); l must give an Eq. 14 range that covers the outputs'
 * bound K max|c| 128. */
ne_status ne_lconv(ne_params p, ne_digits dg, const int32_t* c, const int8_t* g, int64_t* out, uint32_t* flags,
                   uint64_t* nflag, int64_t batch, int64_t n, int64_t K, int32_t fuse, int32_t r, int32_t plain,
                   ne_faults faults, int32_t* status, cudaStream_t s);

/* Tuning knob (no counterpart in the paper; process-wide, for calls made
 * after it): how ne_cconv_digits and ne_cconv_entangled split a group of at
 * most 16 Toeplitz blocks between the int8 tensor pipe and the dp4a pipe of
 * the CUDA cores.  -1: the default (the split measured fastest per digit-plane
 * count); 0: tensor pipe only; HR in {23, 24, 34, 42, 43, 44}: 8 tensor
 * warps and H dp4a warps of R outputs per thread, which take H * R / 2 of
 * the blocks; 4HR in {443, 444}: the same with 4 tensor warps (groups of 16
 * blocks from raw streams or planes; others take HR).  NE_EINVAL for any
 * other value. */
ne_status ne_set_cconv_split(int32_t variant);

/* The same batched convolution through an exact number-theoretic transform
 * (the integer-exact form of the frequency-domain convolution of Sec. V),
 * fused from the raw streams to the extracted outputs: every word of Eq. 16
 * (c_m + 2^l c_{m-1}; plain = 1: c_m itself, no entanglement) is split into
 * the balanced base-256 digits of dg, each digit plane is convolved with g
 * modulo the prime 119 * 2^23 + 1 (exact: a digit plane's convolution is at
 * most N * 2^14 in magnitude), the digits are recombined in int64 and the
 * epilogue of ne_cconv_digits follows (fuse, r, flags, nflag and faults as
 * there; plain requires NE_FUSE_NONE).  A word with a non-zero digit outside
 * dg sets *status = NE_ERANGE (status: device int32, nullable); with the
 * range-checked split of a planned digit set the inputs are checked instead,
 * the lost stream's included under NE_FUSE_RECOVER.
 * c: int32 [batch][M][N]; g: int8 [batch][N]; out: int64 [batch][M][N].
 * N = 1024; M * dg.S <= 15. */
ne_status ne_cconv_ntt(ne_params p, ne_digits dg, const int32_t* c, const int8_t* g, int64_t* out,
                       uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t N, int32_t fuse,
                       int32_t r, int32_t plain, ne_faults faults, int32_t* status, cudaStream_t s);

/* Workspace bytes ne_cconv_ntt_any needs for batch groups of M streams of
 * length N (-1 for invalid sizes). */
int64_t ne_cconv_ntt_any_workspace(int32_t M, int64_t N, int64_t batch);

/* The transform convolution for any N in [2, 65536]: the words of Eq. 16
 * (plain = 1: the raw values) are transformed modulo two primes (77 * 2^19 + 1
 * and 69 * 2^19 + 1) at length N (a power of two) or at the next power of two
 * >= 2N - 1 (a linear convolution folded back), and the outputs rebuilt by the
 * Chinese remainder theorem, then the epilogue (and fault hook, positions
 * group * N + i) of ne_cconv_digits.
 * cmin, cmax: the range of the stream values; an input outside it sets
 * *status = NE_ERANGE (device int32, nullable; the lost stream's inputs are
 * checked too under NE_FUSE_RECOVER), and the host returns
 * NE_ERANGE when N * max|c| (2^l + 1) * 128 could leave the two-prime range.
 * workspace: device, 16-byte aligned, at least ne_cconv_ntt_any_workspace
 * bytes (caller-owned scratch).  The first call on a device also fills the
 * library's twiddle tables and synchronises s.  c: int32 [batch][M][N];
 * g: int8 [batch][N]; out: int64 [batch][M][N]; flags: [batch][ceil(N/32)];
 * batch <= 65535. */
ne_status ne_cconv_ntt_any(ne_params p, int32_t cmin, int32_t cmax, const int32_t* c, const int8_t* g,
                           int64_t* out, uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t N,
                           int32_t fuse, int32_t r, int32_t plain, ne_faults faults, int32_t* status,
                           void* workspace, int64_t workspace_bytes, cudaStream_t s);

/* ------------------------------------------------------------------------ */
/* Extraction, check and recovery (Eq. 17-20, Eq. 24, Prop. 3)               */
/* ------------------------------------------------------------------------ */

/* All M outputs from the streams other than r:
 *   T = (-1)^M sum_{m=0}^{M-2} (-1)^m 2^((M-2-m)l) delta_{(r+1+m) mod M}   (Eq. 17)
 *   d_{r-1} = low (M-1)l bits of T, sign-extended                          (Eq. 18)
 *   d_r = floor((-1)^M (T - d_{r-1}) / 2^((M-1)l))                         (Eq. 19)
 *   d_{r+m} = delta_{r+m} - 2^l d_{r+m-1},  m = 1..M-2                     (Eq. 20)
 * in 128-bit arithmetic (Remark 1); outputs are the low 64 bits.  The sign
 * (-1)^M and the index r-1 in Eq. 19 are the readings under which Eq. 17-19
 * reduce to Eq. 11 at M = 3.  delta, d_hat: int64 [batch][M][n].
 * If flags or nflag is non-null, also performs the check of ne_check. */
ne_status ne_extract(ne_params p, const int64_t* delta, int64_t* d_hat,
                     int64_t batch, int64_t n, int32_t r,
                     uint32_t* flags, uint64_t* nflag, cudaStream_t s);

/* Eq. 24: flag a position when delta_r != d_r + 2^l d_{r-1}, with d_r and
 * d_{r-1} of Eq. 18-19 computed exactly from the other streams.  Any fault
 * confined to one stream of a position is flagged (Prop. 4).  delta: int64
 * [batch][M][n]; flags/nflag as for ne_extract (at least one non-null).
 * With n even and delta 16-byte aligned the reads are staged in shared memory
 * by bulk copies; if such a copy fails to arrive within the kernel's bounded
 * wait, the positions it carried and those of every later unit of the same
 * block are reported flagged (they are not checked), *status is set to
 * NE_ETIMEOUT (status: device int32, nullable, otherwise left untouched), and
 * the block waits, again bounded, for its copies in flight before it returns. */
ne_status ne_check(ne_params p, const int64_t* delta, int64_t batch, int64_t n, int32_t r,
                   uint32_t* flags, uint64_t* nflag, int32_t* status, cudaStream_t s);

/* Test support (no counterpart in the paper; process-wide): the number of
 * polls of the first bounded wait of every block of ne_check's staged kernel
 * (default and maximum 2^22, the limit every other wait keeps, the drain
 * included).  0 makes that wait give up at once, so a test reaches the
 * timeout path without any fault: the block reports NE_ETIMEOUT, reports
 * every position of its units flagged, and drains its copies (which do
 * arrive) before it returns.  NE_EINVAL above the maximum. */
ne_status ne_check_set_wait_limit(uint32_t polls);

/* Prop. 3: stream r_lost is unavailable (never read, may hold anything);
 * all M outputs are rebuilt from the other M-1. */
ne_status ne_recover(ne_params p, const int64_t* delta, int64_t* d_hat,
                     int64_t batch, int64_t n, int32_t r_lost, cudaStream_t s);

/* ------------------------------------------------------------------------ */
/* Transient-fault injection (test harness for the fault model of Sec. I)    */
/* ------------------------------------------------------------------------ */

/* XOR one bit into entangled outputs: for f < count, flips bit bit[f] of
 * delta[(group[f]*P + stream[f])*n + pos[f]].  All four lists are device
 * int64 arrays; entries are validated on the device and out-of-range
 * entries are skipped and reported in *status (NE_EINVAL, nullable). */
ne_status ne_inject(int64_t* delta, int32_t P, int64_t batch, int64_t n,
                    const int64_t* group, const int64_t* pos, const int64_t* stream,
                    const int64_t* bit, int64_t count, int32_t* status, cudaStream_t s);

/* ------------------------------------------------------------------------ */
/* Row/column checksum ABFT of a product (the "ABFT RC-check" of Sec. V)     */
/* ------------------------------------------------------------------------ */
/*
 * The comparator the paper measures against for GEMM (after Huang and
 * Abraham): C_b = A_b B is bordered by the checksum row e^T C_b and the
 * checksum column C_b e, computed from the checksum row of A_b and the
 * checksum column of B; a row or column whose sum disagrees with its checksum
 * is flagged, and a single faulty entry is located and corrected.
 * A: int32 [batch][m][k]; B: int8 [k][n] (one operand for every product);
 * C: int64 [batch][m][n].  batch <= 65535.  All device pointers.
 */

/* Encoding: ac[b][t] = sum_i A_b[i][t] (int64 [batch][k]) and
 * br[t] = sum_j B[t][j] (int64 [k]). */
ne_status ne_abft_rc_encode(const int32_t* A, const int8_t* B, int64_t* ac, int64_t* br,
                            int64_t batch, int64_t m, int64_t k, int64_t n, cudaStream_t s);

/* Check.  work: int64 [batch][2 (m + n + 1)] (caller-owned scratch, written):
 * per product the border [C e (m) | e^T C (n) | e^T C e] computed as
 * A_b (B e), (e^T A_b) B and (e^T A_b)(B e), followed by the row and column
 * sums of C_b [m | n] and one word of border-consistency bits.  row_bad: uint32 [batch][ceil((m+1)/32)],
 * bit i < m: row i of C_b disagrees with its checksum, bit m: the checksum
 * row disagrees with the corner; col_bad: uint32 [batch][ceil((n+1)/32)],
 * likewise for the columns.  nbad (nullable): uint64 [2], the numbers of
 * flagged rows and columns over all products. */
ne_status ne_abft_rc_check(const int64_t* C, const int32_t* A, const int8_t* B, const int64_t* ac,
                           const int64_t* br, int64_t* work, uint32_t* row_bad, uint32_t* col_bad,
                           uint64_t* nbad, int64_t batch, int64_t m, int64_t k, int64_t n,
                           cudaStream_t s);

/* Correction after ne_abft_rc_check: in every product with exactly one
 * flagged row i and one flagged column j, the entry C_b[i][j] (i < m, j < n)
 * is corrected from its row checksum; a fault located in the border leaves
 * C_b unchanged.  ncorrected (nullable): uint64, the entries corrected. */
ne_status ne_abft_rc_correct(int64_t* C, const int64_t* work, const uint32_t* row_bad,
                             const uint32_t* col_bad, uint64_t* ncorrected, int64_t batch,
                             int64_t m, int64_t n, cudaStream_t s);

/* ------------------------------------------------------------------------ */
/* The other LSB operators of Eq. 2 on the entangled streams                 */
/* ------------------------------------------------------------------------ */
/*
 * Each call applies its operator to every entangled stream eps[b][m] (int64
 * [batch][M][n]) in wrapping 64-bit arithmetic -- exact whenever the true
 * results fit 64 bits, which the choice of l guarantees for in-range inputs --
 * and fuses the same epilogues as ne_gemm_digits behind it:
 *  fuse = NE_FUSE_NONE:          out = delta_m for every stream (r ignored).
 *  fuse = NE_FUSE_EXTRACT_CHECK: out = d_hat of Eq. 17-20 using every stream
 *        but r; flags (nullable) get the Eq. 24 check of stream r, one bit per
 *        output position, uint32 [batch][ceil(P/32)] with P the output
 *        positions per group; *nflag (nullable) their count.
 *  fuse = NE_FUSE_RECOVER:       stream r is neither read nor computed; out =
 *        d_hat from the other M-1 streams (Prop. 3).
 * out must not overlap eps.  The operand of group b is at g + b * g_stride
 * (g_stride = 0: one operand shared by every group).
 */
#define NE_OP_ADD 0
#define NE_OP_SUB 1
#define NE_OP_MUL 2

/* Element-wise +, -, x (Eq. 2): delta[b][m][i] = eps[b][m][i] op g_b[i];
 * out: int64 [batch][M][n].  For + and - the operand must be entangled with
 * itself first (ne_entangle_kernel_self, the footnote to Eq. 10) so that
 * the result is again a codeword of Eq. 16. */
ne_status ne_elementwise(ne_params p, int32_t op, const int64_t* eps, const int64_t* g, int64_t g_stride,
                         int64_t* out, uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t n,
                         int32_t fuse, int32_t r, cudaStream_t s);

/* The footnote to Eq. 10: ge[i] = 2^l g[i] + g[i] (int64, n entries). */
ne_status ne_entangle_kernel_self(int32_t l, const int64_t* g, int64_t* ge, int64_t n, cudaStream_t s);

/* Outer product (Eq. 2): delta[b][m][i][j] = eps[b][m][i] g_b[j], j < k;
 * out: int64 [batch][M][n][k]; output positions i*k + j (P = n*k). */
ne_status ne_outer(ne_params p, const int64_t* eps, const int64_t* g, int64_t g_stride, int64_t* out,
                   uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t n, int64_t k,
                   int32_t fuse, int32_t r, cudaStream_t s);

/* Permutation (Eq. 2, the bijection from the sequential index set to the
 * index set perm): delta[b][m][i] = eps[b][m][perm[i]]; perm: int32 [n],
 * one index set for every group (data-independent, as the method requires),
 * a permutation of 0..n-1 by contract.  An entry outside [0, n) is not
 * followed (position 0 is read instead) and sets *status = NE_EINVAL
 * (status: device int32, nullable). */
ne_status ne_permute(ne_params p, const int64_t* eps, const int32_t* perm, int64_t* out,
                     uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t n,
                     int32_t fuse, int32_t r, int32_t* status, cudaStream_t s);

/* Inner product (Eq. 2): delta[b][m] = sum_i eps[b][m][i] g_b[i];
 * out: int64 [batch][M]; one output position per group (flags [batch]). */
ne_status ne_inner(ne_params p, const int64_t* eps, const int64_t* g, int64_t g_stride, int64_t* out,
                   uint32_t* flags, uint64_t* nflag, int64_t batch, int64_t n,
                   int32_t fuse, int32_t r, cudaStream_t s);

/* Circular cross-correlation y[i] = sum_j x[(i + j) mod N] g[j] is the
 * circular convolution of x with g_rev[j] = g[(N - j) mod N]: this writes
 * g_rev (int8 [batch][N]) so that ne_cconv / ne_cconv_digits compute the
 * correlation form of the star operator of Eq. 2.  g_rev must not alias g. */
ne_status ne_reverse_operand(const int8_t* g, int8_t* g_rev, int64_t batch, int64_t N, cudaStream_t s);

/* ------------------------------------------------------------------------ */
/* Checksum ABFT comparator (Eq. 3-6, Sec. II-A)                             */
/* ------------------------------------------------------------------------ */

/* Eq. 4: x[b][m][i] = c[b][m][i] for m < M and x[b][M][i] = sum_m c[b][m][i]
 * (the checksum stream), widened to int64.  c: int32 [batch][M][n];
 * x: int64 [batch][M+1][n]. */
ne_status ne_abft_encode(int32_t M, const int32_t* c, int64_t* x,
                         int64_t batch, int64_t n, cudaStream_t s);

/* Eq. 6 per position: flag when sum_{m<M} d[b][m][i] != d[b][M][i].
 * d: int64 [batch][M+1][n]; flags/nflag as for ne_check. */
ne_status ne_abft_check(int32_t M, const int64_t* d, int64_t batch, int64_t n,
                        uint32_t* flags, uint64_t* nflag, cudaStream_t s);

/* Sec. II-A: rebuild the lost plane j of d in place as d[M] - sum_{m != j} d[m]. */
ne_status ne_abft_recover(int32_t M, int64_t* d, int64_t batch, int64_t n, int32_t j,
                          cudaStream_t s);

/* ------------------------------------------------------------------------ */
/* Ragged batches: many independent jobs in a few persistent launches       */
/* ------------------------------------------------------------------------ */
/*
 * Sec. IV notes that long streams and large products are processed as many
 * independent blocks; the entanglement of every block is independent.  A
 * batch runs any mix of such jobs -- products and circular convolutions,
 * with their own M, l and sizes -- through the same digit-plane tensor path:
 * one launch entangles every job into digit planes (and writes each
 * product's operand transposed), then one persistent launch walks the
 * product tiles and one the convolution tiles (an atomic tile counter each),
 * each tile running the operation with the fused extract/check (or fused
 * recovery) of its job; convolutions at or above the plan's ntt_min_n run
 * as exact transforms in the launches that follow.  Every launch reads only
 * device memory prepared by ne_batch_plan, so ne_batch_run can be captured
 * in a CUDA graph and replayed.
 */
#define NE_JOB_GEMM  0
#define NE_JOB_CCONV 1

#define NE_ORDER_JOB 0   /* tiles in job order                         */
#define NE_ORDER_LPT 1   /* costliest tiles first (longest-processing-time) */

typedef struct {
    int32_t kind;              /* NE_JOB_GEMM or NE_JOB_CCONV                                 */
    int32_t M;                 /* streams, 3..5                                               */
    int32_t l;                 /* shift; 0: chosen by the plan's l_policy from the job's bound */
    int32_t rows, cols, k;     /* GEMM: (rows x k) streams times a (k x cols) operator,
                                  any sizes >= 1 with k <= 131056                             */
    int32_t N;                 /* CCONV: signal length in [2, 65536]; a length that is not a
                                  multiple of 64 runs on the exact transforms                */
    int32_t r;                 /* checked stream (EXTRACT_CHECK) or lost stream (RECOVER)     */
    int32_t fuse;              /* NE_FUSE_EXTRACT_CHECK, NE_FUSE_RECOVER, or NE_FUSE_NONE
                                  (outputs are the words delta_m; no check)                  */
    int32_t cmin, cmax;        /* range of the stream values (bound and digit plan)           */
    int32_t plain;             /* 1: the plain operation on the M raw streams (no
                                  entanglement, outputs d_m; requires NE_FUSE_NONE) -- the
                                  unprotected path entanglement is compared with             */
    int64_t c_off;             /* int32 element offset of the job's streams [M][positions]    */
    int64_t op_off;            /* byte offset of the job's operator: G [k][cols] or g [N], a
                                  multiple of 4                                               */
    int64_t out_off;           /* int64 element offset of the job's outputs [M][positions]    */
    int64_t flag_off;          /* uint32 word offset of the job's check bitmap                */
    int64_t fault_begin;       /* the job's range [begin, end) in the fault lists             */
    int64_t fault_end;
} ne_job;

typedef struct {
    int32_t ctas_per_sm;       /* resident blocks per SM of the convolution-tile launch (1..4) */
    int32_t order;             /* NE_ORDER_JOB or NE_ORDER_LPT                                */
    int32_t cconv_blocks;      /* outputs per convolution tile, in blocks of 64: 4, 8 or 16   */
    int32_t l_policy;          /* NE_L_BYTE or NE_L_SMALLEST for jobs with l = 0              */
    int32_t ntt_min_n;         /* convolutions with N >= this (and outputs inside the two-prime
                                  range) run as exact transforms (ne_cconv_ntt_any's kernels)
                                  instead of tensor tiles; 0: only those whose N is not a
                                  multiple of 64 (the tiles take whole blocks of 64)           */
} ne_batch_config;

typedef struct {               /* what ne_batch_run needs to know on the host                 */
    int32_t njobs, ntiles, nsegs, grid;   /* grid: CTAs of the convolution-tile launch  */
    int32_t ngemm_tiles;       /* the first ngemm_tiles tiles are products (their own launch) */
    int32_t gemm_grid;         /* CTAs of the product-tile launch                             */
    int64_t flag_words;        /* total check-bitmap words (for clearing)                     */
    int64_t workspace_bytes;   /* device workspace the plan occupies                          */
    int64_t mma_ops;           /* int8 operations the tiles issue (2 x multiply-adds)         */
    int64_t useful_ops;        /* 2 x multiply-adds of the operations on the raw streams      */
    int32_t ntransform;        /* jobs on the transform path                                  */
    int32_t ntt_max_logL, ntt_max_M;
    int32_t ntt_min_logL;      /* log2 of the shortest transform length among them            */
    int64_t ntt_table_off;     /* byte offsets of the transform jobs' table and scratch       */
    int64_t ntt_ws_off;
    int64_t ntt_units;         /* the largest (M + 1) L of the transform jobs                 */
    int64_t table_bytes;       /* host bytes of the plan's tables (ne_batch_plan_staged)      */
} ne_batch_info;

/* Plan a batch: choose l and the digit plan of every job, lay out the digit
 * planes, cut entangle segments and operation tiles, order the tiles, and
 * write the tables to the device workspace (a copy ordered on stream s: run
 * the batch on s, or synchronise s before using the workspace elsewhere; the
 * host may reuse jobs at once.  workspace may be null to only size it:
 * info->workspace_bytes).  jobs is a host array.
 * Jobs are validated here (NE_EINVAL / NE_ERANGE with the job index in the
 * message).  The fault lists are sorted by position within each job's
 * range. */
ne_status ne_batch_plan(const ne_job* jobs, int32_t njobs, ne_batch_config cfg, void* workspace,
                        int64_t workspace_bytes, ne_batch_info* info, cudaStream_t s);

/* As ne_batch_plan, with the tables built in `staging`, a pinned host buffer
 * of at least info->table_bytes bytes (from a plan without a workspace), and
 * uploaded from it asynchronously on s: the call never waits for the copy
 * engines.  The caller keeps staging untouched until the upload has
 * completed (for instance until the batch run on s has).  workspace may be
 * null to only size the plan, as for ne_batch_plan. */
ne_status ne_batch_plan_staged(const ne_job* jobs, int32_t njobs, ne_batch_config cfg, void* workspace,
                               int64_t workspace_bytes, void* staging, int64_t staging_bytes, ne_batch_info* info,
                               cudaStream_t s);

/* Run a planned batch.  c: int32 stream arena, ops: int8 operator arena,
 * out: int64 output arena (d_hat of every job), flags: check bitmaps (all
 * info.flag_words are cleared first), nflag: total flagged positions
 * (nullable), faults: optional transient-fault lists (positions within the
 * job, stream, bit; all null when unused) applied to delta before the
 * extraction, status: NE_ERANGE if an input lies outside its job's range
 * (nullable, not reset).  No allocation, no host synchronisation. */
ne_status ne_batch_run(ne_batch_info info, const int32_t* c, const int8_t* ops, int64_t* out, uint32_t* flags,
                       uint64_t* nflag, const int64_t* fault_pos, const int32_t* fault_stream,
                       const int32_t* fault_bit, void* workspace, int32_t* status, cudaStream_t s);

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory themselves -- for example code that
 * runs inside another framework's memory pool or under a fixed device-memory
 * budget, or a hot loop where a cudaMalloc (which synchronises the device)
 * is not acceptable -- and therefore cannot hand ne_batch_run a workspace.
 *
 * ne_batch_run_static plans the batch (as ne_batch_plan) and runs it (as
 * ne_batch_run) with the scratch memory -- the plan's tables, every job's
 * digit planes and the transform jobs' table and scratch -- in one static
 * device array of NE_STATIC_WORKSPACE_BYTES bytes that the library owns.
 * The caller still passes every input and output (device pointers, as for
 * ne_batch_run; jobs and cfg are host data).  The call allocates no device
 * memory.
 *  - The array is part of the batch code's device module: it is held on
 *    every GPU where that module is loaded -- from the first launch of any
 *    batch kernel (ne_batch_run included) with CUDA's lazy module loading,
 *    or from the library's load with CUDA_MODULE_LOADING=EAGER -- until the
 *    process exits, whether or not ne_batch_run_static is ever called.
 *  - A batch whose scratch exceeds the array is rejected with NE_ENOMEM
 *    before any device work.
 *  - The first call on a device looks up the array's device address (one
 *    runtime query with that device current), and the first call that holds
 *    a transform job also fills the library's twiddle tables and
 *    synchronises s.
 *  - Do not call it under stream capture: every call plans the batch, which
 *    copies the tables from host memory that lives only during the call.
 *    To replay a batch from a CUDA graph, plan it with ne_batch_plan into a
 *    caller workspace and capture ne_batch_run.
 *  - The planning's table copy is ordered on s, before the run; consecutive
 *    calls on one stream therefore never see each other's tables.
 *  - All calls share the one array: calls whose work overlaps on the GPU
 *    (other streams, other host threads) overwrite each other's scratch and
 *    race.  The array keeps the last call's contents; everything a run needs
 *    zeroed is cleared by the run itself. */
#define NE_STATIC_WORKSPACE_BYTES (32LL << 20)
ne_status ne_batch_run_static(const ne_job* jobs, int32_t njobs, ne_batch_config cfg, const int32_t* c,
                              const int8_t* ops, int64_t* out, uint32_t* flags, uint64_t* nflag,
                              const int64_t* fault_pos, const int32_t* fault_stream, const int32_t* fault_bit,
                              int32_t* status, cudaStream_t s);

/* ------------------------------------------------------------------------ */

/* Serving runtime support (no counterpart in the paper): copy `count`
 * regions host -> device on stream s, region i being nbytes[i] bytes from
 * src_base + src_off[i] (host; pinned for the copies to be asynchronous) to
 * dst_base + dst_off[i] (device).  One cudaMemcpyAsync per region, issued in
 * order, so the copy engines move the bytes while the SMs compute; the three
 * arrays are host arrays read during the call. */
ne_status ne_copy_regions_h2d(void* dst_base, const void* src_base, const int64_t* dst_off, const int64_t* src_off,
                              const int64_t* nbytes, int64_t count, cudaStream_t s);

/* Message of the last failed call on this host thread ("" if none). */
const char* ne_last_error(void);

/* Library version string. */
const char* ne_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NE_H */
